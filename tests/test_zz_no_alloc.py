"""gmg_residual_norm_noalloc: the allocation-free residual norm for callers
that cannot allocate device memory (allocator / memory-pool callbacks,
real-time loops that forbid cudaMalloc) and so cannot create a handle.

Checked through the C ABI against the handle path's gmg_residual_norm and
against the oracle's residual and norm, on two calls in a row with different
data, and on a large grid followed by a small one (the static scratch keeps
the previous call's contents, which the small call must not read).  Bad
pointers are rejected before any launch.  This file is collected last on
purpose.
"""
import ctypes

import numpy as np
import pytest

import oracle
from paper_1208_4247_gb300 import build, gmg, inputs

GMG_ERR_ARG, GMG_ERR_LAYOUT = 1, 2


def _lib():
    build.build()
    return gmg.lib()


def test_rejects_grids_beyond_static_scratch():
    L = _lib()
    st = L.gmg_residual_norm_noalloc(3, 512, None, None, None, None)
    assert st == GMG_ERR_ARG  # before any device work
    assert b"static scratch" in L.gmg_last_error()


def test_rejects_misaligned_pointer():
    L = _lib()
    a = np.zeros(64)
    base = a.ctypes.data
    st = L.gmg_residual_norm_noalloc(2, 4, ctypes.c_void_p(base + 4), ctypes.c_void_p(base),
                                     ctypes.c_void_p(base), None)
    assert st == GMG_ERR_LAYOUT
    assert b"8-byte aligned" in L.gmg_last_error()


def test_rejects_host_pointer():
    L = _lib()
    f = np.zeros((5, 5))
    u = np.zeros((5, 5))
    out = np.zeros(1)
    st = L.gmg_residual_norm_noalloc(2, 4, ctypes.c_void_p(f.ctypes.data),
                                     ctypes.c_void_p(u.ctypes.data),
                                     ctypes.c_void_p(out.ctypes.data), None)
    assert st == GMG_ERR_LAYOUT
    assert b"device pointer" in L.gmg_last_error()


def _case(d, n, seed):
    f = inputs.rhs_uniform(d, n, seed)
    rng = np.random.default_rng(seed)
    u = np.zeros((n + 1,) * d)
    u[(slice(1, -1),) * d] = 1e-3 * rng.standard_normal((n - 1,) * d)
    # the oracle's unscaled residual norm ||h^2 f - A'u||
    ref = oracle.norm2(oracle.residual(oracle.scale_rhs(f), u))
    return f, u, ref


def _noalloc(L, torch, d, n, f, u, out):
    fd = torch.from_numpy(f).cuda()
    ud = torch.from_numpy(u).cuda()
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    st = L.gmg_residual_norm_noalloc(d, n, ctypes.c_void_p(fd.data_ptr()),
                                     ctypes.c_void_p(ud.data_ptr()),
                                     ctypes.c_void_p(out.data_ptr()), stream)
    assert st == 0, L.gmg_last_error()
    return float(out.item()), fd, ud


@pytest.mark.gpu
@pytest.mark.parametrize("d,n", [(3, 256), (2, 1024), (3, 16)])
def test_noalloc_norm_matches_handle_norm_twice(d, n):
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    L = _lib()
    out = torch.zeros(1, dtype=torch.float64, device="cuda")
    with gmg.Solver(d, n) as S:
        for call, seed in enumerate((21, 22)):
            f, u, ref_orc = _case(d, n, seed)
            got, fd, ud = _noalloc(L, torch, d, n, f, u, out)
            ref = S.residual_norm(fd, ud.clone())
            assert got == pytest.approx(ref, rel=1e-12), (call, got, ref)
            assert got == pytest.approx(ref_orc, rel=1e-12), (call, got, ref_orc)


@pytest.mark.gpu
def test_noalloc_small_after_large_reads_only_its_own_partials():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    L = _lib()
    out = torch.zeros(1, dtype=torch.float64, device="cuda")
    # 3D n = 256 fills 32640 partial sums; 3D n = 16 then writes 15 of them
    results = []
    for d, n, seed in ((3, 256, 31), (3, 16, 32), (2, 64, 33)):
        f, u, ref_orc = _case(d, n, seed)
        got, fd, ud = _noalloc(L, torch, d, n, f, u, out)
        with gmg.Solver(d, n) as S:
            ref = S.residual_norm(fd, ud.clone())
        results.append((d, n, got, ref, ref_orc))
    for d, n, got, ref, ref_orc in results:
        assert got == pytest.approx(ref, rel=1e-12), (d, n, got, ref)
        assert got == pytest.approx(ref_orc, rel=1e-12), (d, n, got, ref_orc)
