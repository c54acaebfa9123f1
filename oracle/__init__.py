"""ctypes binding of the CPU FP64 oracle (``gmg_oracle.c``).

TEST INFRASTRUCTURE ONLY: the slow, plain reference that the CUDA solver is
checked against.  Only the tests, ``__graft_entry__.smoke()`` and the
benchmark's CPU-baseline leg may import this package.  It shares no code with
the CUDA library and never imports it.

Arrays are numpy float64 with all (n+1)^d grid nodes, x fastest (shape
``(n+1, n+1)`` in 2D and ``(n+1, n+1, n+1)`` in 3D, indexed ``[k, j, i]``).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "gmg_oracle.c")
_LIB = os.path.join(_HERE, "libgmg_oracle.so")
_lock = threading.Lock()
_lib = None

WJACOBI = 0
RBGS = 1
MCGS = 3          # the paper's 4-colour (2D) / 8-colour (3D) Gauss-Seidel
FW, SIMPLEX = 0, 1  # transfer: full weighting + multilinear P, or the paper's R and P


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (-O2, OpenMP, no FMA contraction)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call(
            ["gcc", "-O2", "-std=c11", "-fopenmp", "-ffp-contract=off", "-fPIC", "-shared",
             _SRC, "-o", tmp, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


class Cfg(ctypes.Structure):
    _fields_ = [("d", ctypes.c_int), ("n", ctypes.c_int), ("levels", ctypes.c_int),
                ("smoother", ctypes.c_int), ("omega", ctypes.c_double),
                ("nu1", ctypes.c_int), ("nu2", ctypes.c_int), ("coarse_sweeps", ctypes.c_int),
                ("transfer", ctypes.c_int)]


def lib():
    global _lib
    with _lock:
        if _lib is None:
            build()
            L = ctypes.CDLL(_LIB)
            P = ctypes.c_void_p
            I = ctypes.c_int
            D = ctypes.c_double
            for name, args, res in [
                ("orc_apply_stencil", [I, I, P, P], None),
                ("orc_residual", [I, I, P, P, P], None),
                ("orc_norm2", [I, I, P], D),
                ("orc_rbgs", [I, I, P, P, I], None),
                ("orc_wjacobi", [I, I, P, P, D, I], None),
                ("orc_restrict_fw", [I, I, P, P], None),
                ("orc_prolong_add", [I, I, P, P], None),
                ("orc_coarse_solve", [I, I, P, P, I], None),
                ("orc_vcycle", [ctypes.POINTER(Cfg), P, P], I),
                ("orc_scale_rhs", [I, I, P, P], None),
                ("orc_solve", [ctypes.POINTER(Cfg), P, P, D, I, P], I),
                ("orc_conv_fwd", [I, I, P, P, P, P, P], None),
                ("orc_conv_bwd", [I, I, P, P, P, P, P, P, P], None),
                ("orc_learned_smooth_error", [I, I, P, P, P], None),
                ("orc_cgc_error", [I, I, P, I], None),
                ("orc_learned_loss", [I, I, P, P, P, I], D),
                ("orc_learned_relax", [I, I, P, P, P, P], None),
                ("orc_conv_fwd_bf16", [I, I, P, P, P, P], None),
                ("orc_set_bf16_activations", [I], None),
                ("orc_vcycle_learned", [ctypes.POINTER(Cfg), P, P, P], I),
                ("orc_fmg", [ctypes.POINTER(Cfg), P, P], I),
                ("orc_mcgs", [I, I, P, P, I, I], None),
                ("orc_restrict_simplex", [I, I, P, P], None),
                ("orc_prolong_diag", [I, I, P, P], None),
            ]:
                fn = getattr(L, name)
                fn.argtypes = args
                fn.restype = res
            _lib = L
    return _lib


def _p(a: np.ndarray):
    assert a.dtype == np.float64 and a.flags["C_CONTIGUOUS"]
    return a.ctypes.data_as(ctypes.c_void_p)


def _dn(a: np.ndarray):
    d = a.ndim
    n = a.shape[0] - 1
    assert d in (2, 3) and all(s == n + 1 for s in a.shape)
    return d, n


def max_levels(n: int) -> int:
    """Number of grids from n intervals down to 2 intervals (one unknown)."""
    return int(np.log2(n))


def make_cfg(d, n, levels=0, smoother=RBGS, omega=0.8, nu1=2, nu2=2, coarse_sweeps=1,
             transfer=FW) -> Cfg:
    return Cfg(d, n, levels if levels > 0 else max_levels(n), smoother, omega, nu1, nu2,
               coarse_sweeps, transfer)


def apply_stencil(u):
    d, n = _dn(u)
    out = np.empty_like(u)
    lib().orc_apply_stencil(d, n, _p(u), _p(out))
    return out


def residual(b, u):
    d, n = _dn(u)
    r = np.empty_like(u)
    lib().orc_residual(d, n, _p(b), _p(u), _p(r))
    return r


def norm2(r):
    d, n = _dn(r)
    return lib().orc_norm2(d, n, _p(r))


def rbgs(b, u, sweeps):
    d, n = _dn(u)
    lib().orc_rbgs(d, n, _p(b), _p(u), sweeps)
    return u


def wjacobi(b, u, omega, sweeps):
    d, n = _dn(u)
    lib().orc_wjacobi(d, n, _p(b), _p(u), omega, sweeps)
    return u


def restrict_fw(r):
    d, n = _dn(r)
    nc = n // 2
    bc = np.empty((nc + 1,) * d)
    lib().orc_restrict_fw(d, n, _p(r), _p(bc))
    return bc


def prolong_add(uc, u):
    d, nc = _dn(uc)
    lib().orc_prolong_add(d, nc, _p(uc), _p(u))
    return u


def mcgs(b, u, sweeps, backward=False):
    d, n = _dn(u)
    lib().orc_mcgs(d, n, _p(b), _p(u), sweeps, 1 if backward else 0)
    return u


def restrict_simplex(r):
    d, n = _dn(r)
    nc = n // 2
    bc = np.empty((nc + 1,) * d)
    lib().orc_restrict_simplex(d, n, _p(r), _p(bc))
    return bc


def prolong_diag(uc, u):
    d, nc = _dn(uc)
    lib().orc_prolong_diag(d, nc, _p(uc), _p(u))
    return u


def coarse_solve(b, sweeps=1):
    d, n = _dn(b)
    u = np.empty_like(b)
    lib().orc_coarse_solve(d, n, _p(b), _p(u), sweeps)
    return u


def scale_rhs(f):
    d, n = _dn(f)
    b = np.empty_like(f)
    lib().orc_scale_rhs(d, n, _p(f), _p(b))
    return b


def vcycle(cfg: Cfg, b, u):
    rc = lib().orc_vcycle(ctypes.byref(cfg), _p(b), _p(u))
    if rc != 0:
        raise ValueError("oracle V-cycle: bad configuration")
    return u


def solve(cfg: Cfg, f, u, rtol=1e-10, maxit=100):
    """Returns (cycles, relres history); u is updated in place."""
    hist = np.zeros(maxit)
    it = lib().orc_solve(ctypes.byref(cfg), _p(f), _p(u), rtol, maxit, _p(hist))
    if it < 0:
        raise ValueError("oracle solve: bad configuration")
    return it, hist[:it].copy()


HIDDEN = 8


def taps(d):
    return 27 if d == 3 else 9


def _pf(a):
    assert a.dtype == np.float32 and a.flags["C_CONTIGUOUS"]
    return a.ctypes.data_as(ctypes.c_void_p)


def conv_fwd(W1, W2, x):
    """Returns (y, z) of the learned smoother's network on grid function x."""
    d, n = _dn(x)
    y = np.empty_like(x)
    z = np.empty((HIDDEN,) + x.shape)
    lib().orc_conv_fwd(d, n, _pf(W1), _pf(W2), _p(x), _p(z), _p(y))
    return y, z


def conv_bwd(W1, W2, x, gy):
    """Returns (gx, dW1, dW2) for upstream gradient gy."""
    d, n = _dn(x)
    gx = np.empty_like(x)
    dW1 = np.zeros((HIDDEN, taps(d)))
    dW2 = np.zeros((HIDDEN, taps(d)))
    lib().orc_conv_bwd(d, n, _pf(W1), _pf(W2), _p(x), _p(gy), _p(gx), _p(dW1), _p(dW2))
    return gx, dW1, dW2


def learned_smooth_error(W1, W2, e):
    d, n = _dn(e)
    lib().orc_learned_smooth_error(d, n, _pf(W1), _pf(W2), _p(e))
    return e


def cgc_error(e, cycles=30):
    d, n = _dn(e)
    lib().orc_cgc_error(d, n, _p(e), cycles)
    return e


def learned_loss(W1, W2, e0, coarse_cycles=30):
    d, n = _dn(e0)
    return lib().orc_learned_loss(d, n, _pf(W1), _pf(W2), _p(e0), coarse_cycles)


def learned_relax(W1, W2, b, u):
    d, n = _dn(u)
    lib().orc_learned_relax(d, n, _pf(W1), _pf(W2), _p(b), _p(u))
    return u


def conv_fwd_bf16(W1, W2, x):
    """The network with BF16 operands (x and relu(z) rounded to BF16)."""
    d, n = _dn(x)
    y = np.empty_like(x)
    lib().orc_conv_fwd_bf16(d, n, _pf(W1), _pf(W2), _p(x), _p(y))
    return y


def vcycle_learned(cfg: Cfg, weights, b, u, bf16_activations=False):
    """weights: list (one per level) of float32 arrays (2, 8, T) or None.
    bf16_activations: evaluate the network with BF16 operands."""
    lib().orc_set_bf16_activations(1 if bf16_activations else 0)
    arrs = [None if w is None else np.ascontiguousarray(w, dtype=np.float32) for w in weights]
    ptrs = (ctypes.c_void_p * len(arrs))(*[None if a is None else a.ctypes.data for a in arrs])
    rc = lib().orc_vcycle_learned(ctypes.byref(cfg), ptrs, _p(b), _p(u))
    lib().orc_set_bf16_activations(0)
    if rc != 0:
        raise ValueError("oracle learned V-cycle: bad configuration")
    return u


def fmg(cfg: Cfg, b, u):
    """FMG-V (Algorithm 2) on b = h^2 f; u (initial content ignored) is
    overwritten with the result."""
    rc = lib().orc_fmg(ctypes.byref(cfg), _p(b), _p(u))
    if rc != 0:
        raise ValueError("oracle FMG: bad configuration")
    return u
