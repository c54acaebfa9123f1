"""gmg_residual_norm_noalloc: the allocation-free residual norm for callers
that cannot allocate device memory (allocator / memory-pool callbacks,
real-time loops that forbid cudaMalloc) and so cannot create a handle.

Checked through the C ABI against the handle path's gmg_residual_norm, on two
calls in a row with different data (the static scratch keeps the previous
call's contents).  This file is collected last on purpose.
"""
import ctypes

import numpy as np
import pytest

from paper_1208_4247_gb300 import build, gmg, inputs


def test_rejects_grids_beyond_static_scratch():
    build.build()
    L = gmg.lib()
    st = L.gmg_residual_norm_noalloc(3, 512, None, None, None, None)
    assert st == 1  # GMG_ERR_ARG, before any device work
    assert b"static scratch" in L.gmg_last_error()


@pytest.mark.gpu
@pytest.mark.parametrize("d,n", [(3, 256), (2, 1024), (3, 16)])
def test_noalloc_norm_matches_handle_norm_twice(d, n):
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    build.build()
    L = gmg.lib()
    out = torch.zeros(1, dtype=torch.float64, device="cuda")
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    with gmg.Solver(d, n) as S:
        for call, seed in enumerate((21, 22)):
            f = torch.from_numpy(inputs.rhs_uniform(d, n, seed)).cuda()
            rng = np.random.default_rng(seed)
            un = np.zeros((n + 1,) * d)
            un[(slice(1, -1),) * d] = 1e-3 * rng.standard_normal((n - 1,) * d)
            u = torch.from_numpy(un).cuda()
            st = L.gmg_residual_norm_noalloc(d, n, ctypes.c_void_p(f.data_ptr()),
                                            ctypes.c_void_p(u.data_ptr()),
                                            ctypes.c_void_p(out.data_ptr()), stream)
            assert st == 0, L.gmg_last_error()
            got = float(out.item())
            ref = S.residual_norm(f, u.clone())
            assert got == pytest.approx(ref, rel=1e-12), (call, got, ref)
