"""Thin ctypes binding of ``libgmg.so`` (include/gmg.h).

Argument marshalling only: every step of the solve runs in the library's
CUDA kernels.  Tensors are torch float64 CUDA tensors of shape (n+1,)*d
(all grid nodes, x fastest); the calls are ordered on torch's current
stream.  There is no CPU fallback: without the built library every call
raises.
"""
from __future__ import annotations

import ctypes
import os
import threading

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "lib", "libgmg.so")

OK = 0
ERR_NOT_CONVERGED = 6
STATUS = {0: "OK", 1: "ERR_ARG", 2: "ERR_LAYOUT", 3: "ERR_ALLOC", 4: "ERR_CUDA",
          5: "ERR_NONFINITE", 6: "ERR_NOT_CONVERGED", 7: "ERR_DEVICE_TIMEOUT",
          8: "ERR_UNSUPPORTED"}
SMOOTHERS = {"wjacobi": 0, "rbgs": 1, "learned": 2, "mcgs": 3}
TRANSFERS = {"fw": 0, "paper": 1}
PRECISIONS = {"fp64": 0, "fp32": 1, "bf16": 2, "df": 3}
CYCLES = {"v": 0, "fmg": 1}


class GMGError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{STATUS.get(status, status)}: {msg}")
        self.status = status


class Config(ctypes.Structure):
    _fields_ = [("d", ctypes.c_int), ("n", ctypes.c_int), ("levels", ctypes.c_int),
                ("smoother", ctypes.c_int), ("omega", ctypes.c_double),
                ("nu1", ctypes.c_int), ("nu2", ctypes.c_int), ("cycle", ctypes.c_int),
                ("precision", ctypes.c_int), ("maxit", ctypes.c_int),
                ("inner_cycles", ctypes.c_int), ("coarse_sweeps", ctypes.c_int),
                ("transfer", ctypes.c_int)]


class KernelStat(ctypes.Structure):
    _fields_ = [("kernel", ctypes.c_char * 24), ("level", ctypes.c_int),
                ("launches", ctypes.c_int64), ("ms", ctypes.c_double),
                ("dp_ops", ctypes.c_double), ("bytes", ctypes.c_double)]


_lock = threading.Lock()
_lib = None

P = ctypes.c_void_p
I = ctypes.c_int
D = ctypes.c_double
PI = ctypes.POINTER(ctypes.c_int)
PD = ctypes.POINTER(ctypes.c_double)

# name -> (argtypes, restype); every symbol include/gmg.h declares.
SIGNATURES = {
    "gmg_abi_version": ([], I),
    "gmg_measure_fp64_rate": ([I, PD, P], I),
    "gmg_last_error": ([], ctypes.c_char_p),
    "gmg_config_init": ([ctypes.POINTER(Config), I, I], I),
    "gmg_create": ([ctypes.POINTER(Config), P, ctypes.POINTER(P)], I),
    "gmg_solve": ([P, P, P, D, PI, PD], I),
    "gmg_solve_host": ([P, P, P, D, PI, PD], I),
    "gmg_cycles": ([P, P, P, I, PD], I),
    "gmg_history": ([P, PD, I, PI], I),
    "gmg_residual_norm": ([P, P, P, PD], I),
    "gmg_residual_norm_noalloc": ([I, I, P, P, P, P], I),
    "gmg_destroy": ([P], I),
    "gmg_set_timing": ([P, I], I),
    "gmg_timing_report": ([P, ctypes.POINTER(KernelStat), I, PI,
                           ctypes.POINTER(ctypes.c_int64)], I),
    "gmg_timing_reset": ([P], I),
    "gmg_batch_create": ([I, PI, PI, ctypes.POINTER(Config), I, I, P, ctypes.POINTER(P)], I),
    "gmg_batch_solve": ([P, ctypes.POINTER(P), ctypes.POINTER(P), D, PI, PD, PI], I),
    "gmg_batch_set_timing": ([P, I], I),
    "gmg_batch_timing_report": ([P, ctypes.POINTER(KernelStat), I, PI,
                                 ctypes.POINTER(ctypes.c_int64)], I),
    "gmg_batch_destroy": ([P], I),
    "gmg_set_learned_weights": ([P, I, P], I),
    "gmg_fft_create": ([I, I, P, ctypes.POINTER(P)], I),
    "gmg_fft_solve": ([P, P, P], I),
    "gmg_fft_destroy": ([P], I),
    "gmg_learned_conv": ([I, I, P, P, P, I, P], I),
    "gmg_learned_loss_grad": ([I, I, P, P, I, PD, PD, P], I),
    "gmg_learned_train": ([I, I, I, I, I, I, D, ctypes.c_uint64, P, P, PD, P], I),
    "gmg_solve_strided": ([P, P, P, ctypes.POINTER(ctypes.c_int64), D, PI, PD], I),
    "gmg_create_batched": ([I, P, P, ctypes.POINTER(P)], I),
    "gmg_solve_batched": ([P, ctypes.POINTER(P), ctypes.POINTER(P), D, PI], I),
    "gmg_smoother_train": ([P, P, P, PD], I),
    "gmg_smoother_select": ([P, P, P, I, I, I, ctypes.POINTER(ctypes.c_uint), PD, PD], I),
    "gmg_smoother_save": ([P, P, ctypes.c_size_t, ctypes.POINTER(ctypes.c_size_t)], I),
    "gmg_smoother_load": ([P, P, ctypes.c_size_t], I),
}


class TrainConfig(ctypes.Structure):
    """gmg_train_config (include/gmg.h)."""
    _fields_ = [("n", ctypes.c_int), ("steps", ctypes.c_int), ("batch", ctypes.c_int),
                ("pair_cycles", ctypes.c_int), ("coarse_cycles", ctypes.c_int),
                ("lr", ctypes.c_double), ("seed", ctypes.c_uint64),
                ("omega_init", ctypes.c_double), ("level_mask", ctypes.c_uint),
                ("select_f", ctypes.c_void_p)]


def lib():
    """Load libgmg.so (raises if it has not been built)."""
    global _lib
    with _lock:
        if _lib is None:
            if not os.path.exists(LIB_PATH):
                raise RuntimeError(f"{LIB_PATH} is missing: build it with "
                                   "paper_1208_4247_gb300.build.build()")
            L = ctypes.CDLL(LIB_PATH)
            for name, (args, res) in SIGNATURES.items():
                fn = getattr(L, name)
                fn.argtypes = args
                fn.restype = res
            _lib = L
    return _lib


def _check(status: int, allow=()):
    if status != OK and status not in allow:
        raise GMGError(status, lib().gmg_last_error().decode())
    return status


def _stream_ptr(stream):
    import torch
    if stream is None:
        stream = torch.cuda.current_stream()
    return ctypes.c_void_p(stream.cuda_stream)


def _dptr(t, name, d, n):
    import torch
    if not (isinstance(t, torch.Tensor) and t.is_cuda and t.dtype == torch.float64):
        raise TypeError(f"{name} must be a float64 CUDA tensor")
    if tuple(t.shape) != (n + 1,) * d or not t.is_contiguous():
        raise ValueError(f"{name} must be contiguous with shape {(n + 1,) * d}")
    return ctypes.c_void_p(t.data_ptr())


class Solver:
    """GMG solver handle (gmg_create / gmg_solve / gmg_destroy)."""

    def __init__(self, d: int, n: int, levels: int = 0, smoother: str = "rbgs",
                 omega: float = 0.8, nu1: int = 2, nu2: int = 2, precision: str = "fp64",
                 maxit: int = 100, inner_cycles: int = 4, coarse_sweeps: int = 64,
                 cycle: str = "v", transfer: str = "fw", stream=None):
        self.d, self.n = d, n
        cfg = Config()
        _check(lib().gmg_config_init(ctypes.byref(cfg), d, n))
        cfg.levels = levels
        cfg.smoother = SMOOTHERS[smoother]
        cfg.omega = omega
        cfg.transfer = TRANSFERS[transfer]
        cfg.nu1, cfg.nu2 = nu1, nu2
        cfg.precision = PRECISIONS[precision]
        cfg.maxit = maxit
        cfg.inner_cycles = inner_cycles
        cfg.coarse_sweeps = coarse_sweeps
        cfg.cycle = CYCLES[cycle]
        self.cfg = cfg
        h = ctypes.c_void_p()
        _check(lib().gmg_create(ctypes.byref(cfg), _stream_ptr(stream), ctypes.byref(h)))
        self._h = h

    def solve(self, f, u, rtol: float = 1e-10):
        """Returns (cycles, final relative residual, converged)."""
        it = ctypes.c_int(0)
        rel = ctypes.c_double(0.0)
        st = _check(lib().gmg_solve(self._h, _dptr(f, "f", self.d, self.n),
                                    _dptr(u, "u", self.d, self.n), rtol, ctypes.byref(it),
                                    ctypes.byref(rel)), allow=(ERR_NOT_CONVERGED,))
        return it.value, rel.value, st == OK

    def solve_strided(self, f, u, rtol: float = 1e-10):
        """gmg_solve_strided: f, u float64 CUDA tensors of shape (n+1)^d whose
        x stride is 1 (e.g. views into padded arrays).  Returns as solve."""
        import torch
        for name, t in (("f", f), ("u", u)):
            if not (isinstance(t, torch.Tensor) and t.is_cuda and t.dtype == torch.float64):
                raise TypeError(f"{name} must be a float64 CUDA tensor")
            if tuple(t.shape) != (self.n + 1,) * self.d:
                raise ValueError(f"{name} must have shape {(self.n + 1,) * self.d}")
        if f.stride() != u.stride():
            raise ValueError("f and u must have the same strides")
        st_ = list(reversed(f.stride())) + [0] * (3 - self.d)
        strides = (ctypes.c_int64 * 3)(*st_)
        it = ctypes.c_int(0)
        rel = ctypes.c_double(0.0)
        st = _check(lib().gmg_solve_strided(self._h, ctypes.c_void_p(f.data_ptr()),
                                            ctypes.c_void_p(u.data_ptr()), strides, rtol,
                                            ctypes.byref(it), ctypes.byref(rel)),
                    allow=(ERR_NOT_CONVERGED,))
        return it.value, rel.value, st == OK

    def smoother_train(self, n: int, steps: int, batch: int = 8, pair_cycles: int = 1,
                       coarse_cycles: int = 12, lr: float = 3e-3, seed: int = 1,
                       omega_init: float = 0.0, levels=(0,), w_init=None, select_f=None):
        """gmg_smoother_train; returns the per-step mean loss (numpy).
        select_f (float64 CUDA tensor of the target problem, optional): keep
        the trained weights only on levels where they beat red-black GS."""
        import numpy as np
        sf = None if select_f is None else _dptr(select_f, "select_f", self.d, self.n)
        tc = TrainConfig(n, steps, batch, pair_cycles, coarse_cycles, lr, seed, omega_init,
                         sum(1 << l for l in levels), sf)
        loss = np.zeros(max(steps, 1), np.float64)
        w = None if w_init is None else np.ascontiguousarray(w_init, dtype=np.float32)
        _check(lib().gmg_smoother_train(self._h, ctypes.byref(tc),
                                        None if w is None else ctypes.c_void_p(w.ctypes.data),
                                        loss.ctypes.data_as(PD)))
        return loss[:steps]

    def smoother_select(self, f, candidates, cycles: int = 8, skip: int = 2):
        """gmg_smoother_select: candidates {level: weights (2, 8, 3^d) float32}.
        Returns (kept levels, contraction with red-black GS everywhere,
        contraction with the kept weights)."""
        import numpy as np
        count = max(candidates) + 1 if candidates else 0
        keep = [None] * count
        ptrs = (ctypes.c_void_p * max(count, 1))()
        for l, w in candidates.items():
            a = np.ascontiguousarray(w, dtype=np.float32)
            if a.size != 2 * 8 * (27 if self.d == 3 else 9):
                raise ValueError("weights must hold 2 x 8 x 3^d floats")
            keep[l] = a
            ptrs[l] = a.ctypes.data
        mask = ctypes.c_uint(0)
        rb = ctypes.c_double(0.0)
        rho = ctypes.c_double(0.0)
        _check(lib().gmg_smoother_select(self._h, _dptr(f, "f", self.d, self.n), ptrs, count,
                                         cycles, skip, ctypes.byref(mask), ctypes.byref(rb),
                                         ctypes.byref(rho)))
        del keep
        return [l for l in range(32) if (mask.value >> l) & 1], rb.value, rho.value

    def smoother_save(self) -> bytes:
        """gmg_smoother_save: the learned smoother of every level as a blob."""
        size = ctypes.c_size_t(0)
        _check(lib().gmg_smoother_save(self._h, None, 0, ctypes.byref(size)))
        buf = ctypes.create_string_buffer(max(size.value, 1))
        _check(lib().gmg_smoother_save(self._h, buf, size.value, ctypes.byref(size)))
        return buf.raw[:size.value]

    def smoother_load(self, blob: bytes):
        """gmg_smoother_load of a blob from smoother_save."""
        buf = ctypes.create_string_buffer(blob, len(blob))
        _check(lib().gmg_smoother_load(self._h, buf, len(blob)))

    def solve_host(self, f, u, rtol: float = 1e-10):
        """f, u: C-contiguous float64 numpy arrays (pinned or pageable host
        memory); u is overwritten with the solution."""
        import numpy as np
        for name, a in (("f", f), ("u", u)):
            if not (isinstance(a, np.ndarray) and a.dtype == np.float64
                    and a.flags["C_CONTIGUOUS"] and a.shape == (self.n + 1,) * self.d):
                raise ValueError(f"{name} must be a C-contiguous float64 array of shape "
                                 f"{(self.n + 1,) * self.d}")
        it = ctypes.c_int(0)
        rel = ctypes.c_double(0.0)
        st = _check(lib().gmg_solve_host(self._h, ctypes.c_void_p(f.ctypes.data),
                                         ctypes.c_void_p(u.ctypes.data), rtol,
                                         ctypes.byref(it), ctypes.byref(rel)),
                    allow=(ERR_NOT_CONVERGED,))
        return it.value, rel.value, st == OK

    def cycles(self, f, u, ncycles: int):
        """Exactly ncycles cycles; returns the relative residual after each."""
        out = (ctypes.c_double * max(ncycles, 1))()
        _check(lib().gmg_cycles(self._h, _dptr(f, "f", self.d, self.n),
                                _dptr(u, "u", self.d, self.n), ncycles, out))
        return list(out)[:ncycles]

    def residual_norm(self, f, u):
        """||h^2 f - A'u||_2 in FP64 (writes 0 to u's boundary nodes)."""
        out = ctypes.c_double(0.0)
        _check(lib().gmg_residual_norm(self._h, _dptr(f, "f", self.d, self.n),
                                       _dptr(u, "u", self.d, self.n), ctypes.byref(out)))
        return out.value

    def history(self):
        cnt = ctypes.c_int(0)
        _check(lib().gmg_history(self._h, None, 0, ctypes.byref(cnt)))
        buf = (ctypes.c_double * max(cnt.value, 1))()
        _check(lib().gmg_history(self._h, buf, cnt.value, ctypes.byref(cnt)))
        return list(buf)[:cnt.value]

    def set_timing(self, enable: bool = True):
        _check(lib().gmg_set_timing(self._h, 1 if enable else 0))

    def set_learned_weights(self, level: int, weights):
        """weights: float32 array (2, 8, 3^d) or None (red-black GS on this level)."""
        import numpy as np
        if weights is None:
            _check(lib().gmg_set_learned_weights(self._h, level, None))
            return
        w = np.ascontiguousarray(weights, dtype=np.float32)
        if w.size != 2 * 8 * (27 if self.d == 3 else 9):
            raise ValueError("weights must hold 2 x 8 x 3^d floats")
        _check(lib().gmg_set_learned_weights(self._h, level, ctypes.c_void_p(w.ctypes.data)))

    def timing_reset(self):
        _check(lib().gmg_timing_reset(self._h))

    def timing_report(self):
        """Returns (list of per-(kernel, level) dicts, total kernel launches)."""
        return timing_report(self._h)

    def close(self):
        if getattr(self, "_h", None):
            lib().gmg_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()


def timing_report(handle):
    cnt = ctypes.c_int(0)
    tot = ctypes.c_int64(0)
    _check(lib().gmg_timing_report(handle, None, 0, ctypes.byref(cnt), ctypes.byref(tot)))
    buf = (KernelStat * max(cnt.value, 1))()
    _check(lib().gmg_timing_report(handle, buf, cnt.value, ctypes.byref(cnt), ctypes.byref(tot)))
    rows = [dict(kernel=s.kernel.decode(), level=s.level, launches=s.launches, ms=s.ms,
                 dp_ops=s.dp_ops, bytes=s.bytes) for s in list(buf)[:cnt.value]]
    return rows, tot.value


class Batch:
    """Independent solves of uneven sizes advanced together (gmg_batch_*).

    dims, ns: per-solve d and n.  The inner precision ("fp32" / "bf16"),
    smoother, sweeps and inner cycles are shared; chunk = nodes per work item,
    ctas = CTAs per launch (0 = library defaults)."""

    def __init__(self, dims, ns, smoother: str = "wjacobi", omega: float = 0.8, nu1: int = 1,
                 nu2: int = 1, precision: str = "fp32", inner_cycles: int = 2, maxit: int = 200,
                 chunk: int = 0, ctas: int = 0, stream=None):
        self.dims = list(dims)
        self.ns = list(ns)
        self.count = len(self.dims)
        cfg = Config()
        _check(lib().gmg_config_init(ctypes.byref(cfg), 3, 2))
        cfg.smoother = SMOOTHERS[smoother]
        cfg.omega = omega
        cfg.nu1, cfg.nu2 = nu1, nu2
        cfg.precision = PRECISIONS[precision]
        cfg.inner_cycles = inner_cycles
        cfg.maxit = maxit
        darr = (ctypes.c_int * self.count)(*self.dims)
        narr = (ctypes.c_int * self.count)(*self.ns)
        h = ctypes.c_void_p()
        _check(lib().gmg_batch_create(self.count, darr, narr, ctypes.byref(cfg), chunk, ctas,
                                      _stream_ptr(stream), ctypes.byref(h)))
        self._h = h

    def solve(self, fs, us, rtol: float = 1e-10):
        """fs, us: lists of float64 CUDA tensors.  Returns (per-solve steps,
        per-solve relative residuals, batch steps, all converged)."""
        if len(fs) != self.count or len(us) != self.count:
            raise ValueError("need one f and one u per solve")
        fp = (ctypes.c_void_p * self.count)(
            *[_dptr(f, "f", d, n) for f, d, n in zip(fs, self.dims, self.ns)])
        up = (ctypes.c_void_p * self.count)(
            *[_dptr(u, "u", d, n) for u, d, n in zip(us, self.dims, self.ns)])
        it = (ctypes.c_int * self.count)()
        rel = (ctypes.c_double * self.count)()
        steps = ctypes.c_int(0)
        st = _check(lib().gmg_batch_solve(self._h, fp, up, rtol, it, rel, ctypes.byref(steps)),
                    allow=(ERR_NOT_CONVERGED,))
        return list(it), list(rel), steps.value, st == OK

    def set_timing(self, enable: bool = True):
        _check(lib().gmg_batch_set_timing(self._h, 1 if enable else 0))

    def timing_report(self):
        cnt = ctypes.c_int(0)
        tot = ctypes.c_int64(0)
        _check(lib().gmg_batch_timing_report(self._h, None, 0, ctypes.byref(cnt),
                                             ctypes.byref(tot)))
        buf = (KernelStat * max(cnt.value, 1))()
        _check(lib().gmg_batch_timing_report(self._h, buf, cnt.value, ctypes.byref(cnt),
                                             ctypes.byref(tot)))
        return [dict(kernel=s.kernel.decode(), level=s.level, launches=s.launches, ms=s.ms,
                     dp_ops=s.dp_ops, bytes=s.bytes) for s in list(buf)[:cnt.value]], tot.value

    def close(self):
        if getattr(self, "_h", None):
            lib().gmg_batch_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()


# ------------------------------------------------------------ learned smoother

def learned_taps(d: int) -> int:
    return 27 if d == 3 else 9


def jacobi_weights(d: int, omega: float):
    """Weights with relu(x) - relu(-x) = x: the network is omega * sigma
    (weighted Jacobi), the starting point of training."""
    import numpy as np
    T = learned_taps(d)
    w = np.zeros((2, 8, T), np.float32)
    w[0, 0, T // 2], w[0, 1, T // 2] = 1.0, -1.0
    w[1, 0, T // 2], w[1, 1, T // 2] = omega, -omega
    return w


def learned_conv(weights, x, tensor_cores: bool = False):
    """y = N(x) for a float64 CUDA tensor x (all nodes, zero boundary)."""
    import numpy as np
    import torch
    d = x.dim()
    n = x.shape[0] - 1
    w = np.ascontiguousarray(weights, dtype=np.float32)
    y = torch.zeros_like(x)
    _check(lib().gmg_learned_conv(d, n, ctypes.c_void_p(w.ctypes.data), _dptr(x, "x", d, n),
                                  _dptr(y, "y", d, n), 1 if tensor_cores else 0,
                                  _stream_ptr(None)))
    return y


def learned_loss_grad(weights, e0, coarse_cycles: int = 30, want_grad: bool = True):
    """(loss, grad (2, 8, T) float64 or None) of the two-grid contraction."""
    import numpy as np
    d = e0.dim()
    n = e0.shape[0] - 1
    w = np.ascontiguousarray(weights, dtype=np.float32)
    loss = ctypes.c_double(0.0)
    g = np.zeros((2, 8, learned_taps(d)))
    _check(lib().gmg_learned_loss_grad(
        d, n, ctypes.c_void_p(w.ctypes.data), _dptr(e0, "e0", d, n), coarse_cycles,
        ctypes.byref(loss), g.ctypes.data_as(PD) if want_grad else None, _stream_ptr(None)))
    return loss.value, (g if want_grad else None)


def learned_train(d: int, n: int, steps: int, batch: int, w_init, lr: float = 1e-3,
                  pair_cycles: int = 1, coarse_cycles: int = 12, seed: int = 100):
    """Train on the GPU; returns (weights (2, 8, T) float32, loss history)."""
    import numpy as np
    w0 = np.ascontiguousarray(w_init, dtype=np.float32)
    out = np.zeros_like(w0)
    hist = np.zeros(steps)
    _check(lib().gmg_learned_train(d, n, steps, batch, pair_cycles, coarse_cycles, lr, seed,
                                   ctypes.c_void_p(w0.ctypes.data),
                                   ctypes.c_void_p(out.ctypes.data), hist.ctypes.data_as(PD),
                                   _stream_ptr(None)))
    return out, hist


def measure_fp64_rate(kind: int = 0, stream=None) -> float:
    """gmg_measure_fp64_rate: FP64 instructions/s (0: DFMA, 1: DADD)."""
    out = ctypes.c_double(0.0)
    _check(lib().gmg_measure_fp64_rate(kind, ctypes.byref(out), _stream_ptr(stream)))
    return out.value


class FFTSolver:
    """Direct sine-transform (cuFFT DST-I) solve of the same FD system."""

    def __init__(self, d: int, n: int, stream=None):
        self.d, self.n = d, n
        h = ctypes.c_void_p()
        _check(lib().gmg_fft_create(d, n, _stream_ptr(stream), ctypes.byref(h)))
        self._h = h

    def solve(self, f, u):
        _check(lib().gmg_fft_solve(self._h, _dptr(f, "f", self.d, self.n),
                                   _dptr(u, "u", self.d, self.n)))

    def close(self):
        if getattr(self, "_h", None):
            lib().gmg_fft_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()
