"""The problem statement's entry points on the GPU: the strided solve, the
batched form built from per-solve configurations, and training and
persistence of the learned smoother."""
import ctypes

import numpy as np
import pytest

from paper_1208_4247_gb300 import inputs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch_cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1208_4247_gb300 import build
    build.build()
    return torch


@pytest.mark.parametrize("d,n,pad", [(3, 32, (1, 2, 3)), (2, 64, (0, 5, 0)), (3, 16, (0, 0, 4))])
def test_strided_solve_equals_dense_solve(torch_cuda, d, n, pad):
    """f, u as views into padded arrays: the strided solve gives the dense
    solve's result bit for bit, writes u's boundary as 0 and leaves the
    padding untouched."""
    torch = torch_cuda
    from paper_1208_4247_gb300.gmg import Solver
    f = torch.from_numpy(inputs.rhs_uniform(d, n, 17)).cuda()
    u = torch.zeros_like(f)
    shape = tuple(n + 1 + p for p in (pad if d == 3 else pad[1:]))
    fp = torch.full(shape, 7.0, dtype=torch.float64, device="cuda")
    up = torch.full(shape, 7.0, dtype=torch.float64, device="cuda")
    view = tuple(slice(0, n + 1) for _ in range(d))
    fp[view] = f
    up[view] = 0.0
    with Solver(d, n) as S:
        it, rel, conv = S.solve(f, u, 1e-10)
        it2, rel2, conv2 = S.solve_strided(fp[view], up[view], 1e-10)
    assert conv and conv2 and it == it2 and rel == rel2
    assert torch.equal(up[view], u)
    mask = torch.ones(shape, dtype=torch.bool, device="cuda")
    mask[view] = False
    assert bool((up[mask] == 7.0).all()) and bool((fp[mask] == 7.0).all())


def test_create_batched_equals_batch_create(torch_cuda):
    """gmg_create_batched / gmg_solve_batched from per-solve configurations
    run the same batch as gmg_batch_create / gmg_batch_solve."""
    torch = torch_cuda
    from paper_1208_4247_gb300 import gmg
    mix = [(2, 64), (3, 16), (2, 128), (3, 32)]
    fs = [torch.from_numpy(inputs.rhs_uniform(d, n, 20 + i)).cuda() for i, (d, n) in enumerate(mix)]
    kw = dict(smoother="wjacobi", omega=0.8, nu1=1, nu2=1, precision="fp32")
    us = [torch.zeros_like(f) for f in fs]
    with gmg.Batch([d for d, _ in mix], [n for _, n in mix], inner_cycles=2, **kw) as B:
        it_ref, _, _, conv = B.solve(fs, us, 1e-10)
    assert conv
    L = gmg.lib()
    cfgs = (gmg.Config * len(mix))()
    for c, (d, n) in zip(cfgs, mix):
        L.gmg_config_init(ctypes.byref(c), d, n)
        c.smoother, c.omega, c.nu1, c.nu2 = gmg.SMOOTHERS["wjacobi"], 0.8, 1, 1
        c.precision, c.inner_cycles, c.maxit = gmg.PRECISIONS["fp32"], 2, 200
    h = ctypes.c_void_p()
    gmg._check(L.gmg_create_batched(len(mix), cfgs, gmg._stream_ptr(None), ctypes.byref(h)))
    vs = [torch.zeros_like(f) for f in fs]
    fp = (ctypes.c_void_p * len(mix))(*[f.data_ptr() for f in fs])
    vp = (ctypes.c_void_p * len(mix))(*[v.data_ptr() for v in vs])
    its = (ctypes.c_int * len(mix))()
    try:
        gmg._check(L.gmg_solve_batched(h, fp, vp, 1e-10, its))
    finally:
        L.gmg_batch_destroy(h)
    assert list(its) == list(it_ref)
    for u, v in zip(us, vs):
        assert torch.equal(u, v)


def test_smoother_save_load_round_trip(torch_cuda):
    """The blob of gmg_smoother_save restores the same smoother in a new
    handle (cycles agree bit for bit); a truncated blob is rejected and
    leaves the handle unchanged."""
    torch = torch_cuda
    from paper_1208_4247_gb300.gmg import GMGError, Solver, jacobi_weights
    d, n = 3, 32
    f = torch.from_numpy(inputs.rhs_grf(d, n, 5)).cuda()
    w0 = jacobi_weights(d, 6 / 7)
    w1 = w0.copy()
    w1[1, :2] *= 0.9
    u1 = torch.zeros_like(f)
    with Solver(d, n, smoother="learned", nu1=1, nu2=1) as S:
        S.set_learned_weights(0, w0)
        S.set_learned_weights(2, w1)
        blob = S.smoother_save()
        S.cycles(f, u1, 3)
    levels = 5
    assert len(blob) == 4 * levels + 2 * (2 * 8 * 27 * 4)
    u2 = torch.zeros_like(f)
    with Solver(d, n, smoother="learned", nu1=1, nu2=1) as S:
        S.smoother_load(blob)
        with pytest.raises(GMGError):
            S.smoother_load(blob[:-4])
        assert S.smoother_save() == blob
        S.cycles(f, u2, 3)
    assert torch.equal(u1, u2)


def test_smoother_train_installs_weights(torch_cuda):
    """gmg_smoother_train trains from the weighted-Jacobi start and installs
    the weights on the masked levels; the learned solve then converges."""
    torch = torch_cuda
    from paper_1208_4247_gb300.gmg import Solver
    d, n = 3, 32
    f = torch.from_numpy(inputs.rhs_grf(d, n, 5)).cuda()
    u = torch.zeros_like(f)
    with Solver(d, n, smoother="learned", nu1=1, nu2=1) as S:
        loss = S.smoother_train(n=32, steps=4, batch=2, levels=(0, 1))
        assert loss.shape == (4,) and np.all(np.isfinite(loss)) and np.all(loss > 0)
        blob = S.smoother_save()
        flags = [int.from_bytes(blob[o:o + 4], "little") for o in
                 (0, 4 + 2 * 8 * 27 * 4, 2 * (4 + 2 * 8 * 27 * 4))]
        assert flags == [1, 1, 0]
        it, rel, conv = S.solve(f, u, 1e-10)
    assert conv and rel <= 1e-10


def test_measured_fp64_rate_is_plausible(torch_cuda):
    """gmg_measure_fp64_rate: the FP64 pipe's measured DFMA and DADD rates
    lie within a factor of two of the nominal 2 instructions per clock per SM
    at the SM clock range of the part (152 SMs, up to 2.07 GHz)."""
    from paper_1208_4247_gb300.gmg import measure_fp64_rate
    nominal = 2 * 152 * 2.07e9
    for kind in (0, 1):
        r = measure_fp64_rate(kind)
        assert 0.5 * nominal <= r <= 1.1 * nominal, (kind, r / nominal)
