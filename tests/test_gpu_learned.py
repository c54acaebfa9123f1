"""Learned smoother on the GPU against the CPU FP64 oracle.

* network forward: FP32 accumulation with BF16 weights vs the oracle's FP64
  evaluation of the same (BF16-representable) weights: <= 2e-6 relative
  (about 30 FP32 roundoffs of the largest term);
* two-grid loss and its gradient: loss within 1e-5, gradient against central
  finite differences of the oracle's FP64 loss within 2e-3 relative or
  3e-4 of the gradient's scale (the backward runs in FP32);
* the fused tensor-core network (BF16 sigma and hidden activations) vs the
  oracle's BF16-operand network: <= 1e-4 relative (L2), and one learned
  V-cycle (which uses it on every level) vs the oracle's learned V-cycle:
  <= 1e-3 (below one BF16 ulp, 2^-8);
* training lowers the loss, the learned cycle solves to an FP64 relative
  residual of 1e-10, and a trained network contracts more per cycle than its
  untrained (weighted-Jacobi) start.
"""
import numpy as np
import pytest

import oracle
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


def bf16_round(w):
    """Round-to-nearest-even to BF16 (torch's CPU conversion), as float32."""
    import torch
    t = torch.from_numpy(np.ascontiguousarray(w, np.float32))
    return t.to(torch.bfloat16).to(torch.float32).numpy().reshape(np.shape(w))


def random_weights(d, rng, scale=0.3):
    from paper_1208_4247_gb300.gmg import jacobi_weights
    w = jacobi_weights(d, 0.8) + scale * rng.standard_normal((2, 8, 27 if d == 3 else 9))
    return bf16_round(w.astype(np.float32))


def interior_noise(d, n, rng):
    x = np.zeros((n + 1,) * d)
    x[(slice(1, -1),) * d] = rng.standard_normal((n - 1,) * d)
    return x


@pytest.mark.parametrize("d,n", [(3, 16), (3, 33 - 1), (2, 64)])
def test_conv_forward_matches_oracle(torch_cuda, d, n):
    torch = torch_cuda
    from paper_1208_4247_gb300.gmg import learned_conv
    rng = np.random.default_rng(1)
    w = random_weights(d, rng)
    x = interior_noise(d, n, rng)
    y = learned_conv(w, torch.from_numpy(x).cuda()).cpu().numpy()
    yo, _ = oracle.conv_fwd(w[0].copy(), w[1].copy(), x)
    assert np.max(np.abs(y - yo)) <= 2e-6 * np.max(np.abs(yo))
    assert np.all(y[0] == 0) and np.all(y[:, -1] == 0)
    # the tensor-core kernel against the BF16-operand network: the FP32 sums
    # round a few hidden values to the neighbouring BF16 value (one BF16 ulp,
    # 2^-8 relative), which moves single outputs by ~1e-4 relative
    yt = learned_conv(w, torch.from_numpy(x).cuda(), tensor_cores=True).cpu().numpy()
    yb = oracle.conv_fwd_bf16(w[0].copy(), w[1].copy(), x)
    assert np.max(np.abs(yt - yb)) <= 1e-3 * np.max(np.abs(yb))
    assert np.linalg.norm(yt - yb) <= 1e-4 * np.linalg.norm(yb)
    assert np.all(yt[0] == 0) and np.all(yt[:, -1] == 0)


@pytest.mark.parametrize("d,n", [(3, 8), (2, 16)])
def test_loss_and_gradient_match_oracle(torch_cuda, d, n):
    torch = torch_cuda
    from paper_1208_4247_gb300.gmg import learned_loss_grad
    rng = np.random.default_rng(2)
    w = random_weights(d, rng, 0.1)
    e0 = interior_noise(d, n, rng)
    loss, g = learned_loss_grad(w, torch.from_numpy(e0).cuda(), coarse_cycles=30)
    lo = oracle.learned_loss(w[0].copy(), w[1].copy(), e0, 30)
    assert loss == pytest.approx(lo, rel=1e-5)

    def L(wp):
        return oracle.learned_loss(wp[0].copy(), wp[1].copy(), e0, 30)

    # central differences with the float32 displacement actually applied (a
    # small step keeps them from crossing ReLU kinks): along random directions
    # and along single weights
    for _ in range(3):
        v = rng.standard_normal(w.shape)
        wp = (w + 1e-4 * v).astype(np.float32)
        wm = (w - 1e-4 * v).astype(np.float32)
        dw = wp.astype(np.float64) - wm.astype(np.float64)
        pred = np.sum(g * dw)
        # the backward runs in FP32: its error scales with |g| |dw|, not with
        # the (cancelling) directional derivative itself
        assert pred == pytest.approx(L(wp) - L(wm), rel=2e-3,
                                     abs=3e-4 * np.linalg.norm(g) * np.linalg.norm(dw))
    for _ in range(6):
        idx = tuple(rng.integers(0, s) for s in w.shape)
        wp, wm = w.copy(), w.copy()
        wp[idx] += np.float32(2.0 ** -12)
        wm[idx] -= np.float32(2.0 ** -12)
        fd = (L(wp) - L(wm)) / (float(wp[idx]) - float(wm[idx]))
        assert g[idx] == pytest.approx(fd, rel=2e-3, abs=3e-4 * np.max(np.abs(g)))


@pytest.mark.parametrize("d,n", [(3, 32), (2, 64)])
def test_learned_vcycle_matches_oracle(torch_cuda, d, n):
    torch = torch_cuda
    from paper_1208_4247_gb300.gmg import Solver
    rng = np.random.default_rng(3)
    L = oracle.max_levels(n)
    ws = [random_weights(d, rng, 0.05) if l < L - 2 else None for l in range(L)]
    f = inputs.rhs_uniform(d, n, 5)
    u = interior_noise(d, n, rng) * 1e-2
    uo = u.copy()
    oracle.vcycle_learned(oracle.make_cfg(d, n, 0, oracle.RBGS, 0.8, 1, 1, 1), ws,
                          oracle.scale_rhs(f), uo, bf16_activations=True)
    ud = torch.from_numpy(u).cuda()
    with Solver(d, n, smoother="learned", nu1=1, nu2=1) as S:
        for l, w in enumerate(ws):
            S.set_learned_weights(l, w)
        S.cycles(torch.from_numpy(f).cuda(), ud, 1)
    ug = ud.cpu().numpy()
    # each smoothing inherits the network's ~1e-4 (rare one-ulp BF16 hidden
    # roundings); the cycle applies it on every level: bound 1e-3 < 2^-8
    assert np.linalg.norm(ug - uo) <= 1e-3 * np.linalg.norm(uo)


def _contraction(torch, S, f, cycles=8):
    u = torch.zeros_like(f)
    rel = S.cycles(f, u, cycles)
    return (rel[-1] / rel[2]) ** (1.0 / (cycles - 3))


def test_training_lowers_loss_and_beats_untrained_start(torch_cuda):
    torch = torch_cuda
    from paper_1208_4247_gb300.gmg import Solver, jacobi_weights, learned_train
    d, n = 3, 32
    w0 = jacobi_weights(d, 6 / 7)
    w, hist = learned_train(d, n, steps=60, batch=4, w_init=w0, lr=3e-3, seed=7)
    assert np.all(np.isfinite(hist))
    assert np.mean(hist[-10:]) < 0.9 * np.mean(hist[:5])
    # measured V(1,1) contraction on a 65^3 GRF problem: trained vs untrained start
    nn = 64
    f = torch.from_numpy(inputs.rhs_grf(3, nn, 5)).cuda()
    L = oracle.max_levels(nn)
    with Solver(3, nn, smoother="learned", nu1=1, nu2=1) as S:
        for l in range(L - 1):
            S.set_learned_weights(l, w0)
        rho0 = _contraction(torch, S, f)
        for l in range(L - 1):
            S.set_learned_weights(l, w)
        rho1 = _contraction(torch, S, f)
        u = torch.zeros_like(f)
        it, rel, conv = S.solve(f, u, 1e-10)
    assert rho1 < rho0
    assert conv
    fn = f.cpu().numpy()
    ug = u.cpu().numpy()
    b = oracle.scale_rhs(fn)
    assert oracle.norm2(oracle.residual(b, ug)) / oracle.norm2(b) <= 1e-10
    uo = np.zeros_like(fn)
    oracle.solve(oracle.make_cfg(3, nn, 0, oracle.RBGS, 0.8, 2, 2, 1), fn, uo, 1e-13, 100)
    assert np.linalg.norm(ug - uo) <= 1e-9 * np.linalg.norm(uo)


def _blob_levels(blob, nlev, T):
    """Levels whose flag is 1 in a gmg_smoother_save blob."""
    import struct
    kept, off = [], 0
    for l in range(nlev):
        flag = struct.unpack_from("<i", blob, off)[0]
        off += 4
        if flag:
            kept.append(l)
            off += 4 * 2 * 8 * T
    assert off == len(blob)
    return kept


def test_trained_smoother_gains_over_red_black(torch_cuda):
    """What the trained network gains over the method without it: trained on
    the GPU (65^3 error samples), installed through the library's fallback
    rule on a 65^3 GRF problem, the learned V(1,1) cycle contracts the
    residual faster than the red-black V(1,1) cycle on the same problem, and
    the solve still reaches the oracle's FP64 solution."""
    torch = torch_cuda
    from paper_1208_4247_gb300.gmg import Solver
    d, n = 3, 64
    f = torch.from_numpy(inputs.rhs_grf(d, n, 5)).cuda()
    L = oracle.max_levels(n)
    with Solver(d, n, nu1=1, nu2=1) as R:
        rho_rb = _contraction(torch, R, f)
    with Solver(d, n, smoother="learned", nu1=1, nu2=1) as S:
        S.smoother_train(n, steps=300, batch=8, coarse_cycles=12, lr=2e-3, seed=100,
                         levels=range(L - 2), select_f=f)
        kept = _blob_levels(S.smoother_save(), L, 27)
        rho_l = _contraction(torch, S, f)
        u = torch.zeros_like(f)
        it, rel, conv = S.solve(f, u, 1e-10)
    assert kept, kept
    assert rho_l < 0.95 * rho_rb, (rho_l, rho_rb, kept)
    assert conv
    fn = f.cpu().numpy()
    ug = u.cpu().numpy()
    b = oracle.scale_rhs(fn)
    assert oracle.norm2(oracle.residual(b, ug)) / oracle.norm2(b) <= 1e-10
    uo = np.zeros_like(fn)
    oracle.solve(oracle.make_cfg(d, n, 0, oracle.RBGS, 0.8, 2, 2, 1), fn, uo, 1e-13, 100)
    assert np.linalg.norm(ug - uo) <= 1e-9 * np.linalg.norm(uo)


def test_poor_weights_fall_back_to_red_black(torch_cuda):
    """Finite but poor weights (weighted Jacobi, omega = 0.3) on every level:
    the fallback rejects every level, and the cycle is then the red-black
    V(1,1) cycle bit for bit."""
    torch = torch_cuda
    from paper_1208_4247_gb300.gmg import Solver, jacobi_weights
    d, n = 3, 64
    f = torch.from_numpy(inputs.rhs_grf(d, n, 5)).cuda()
    L = oracle.max_levels(n)
    w = jacobi_weights(d, 0.3)
    rng = np.random.default_rng(8)
    u0 = torch.from_numpy(interior_noise(d, n, rng)).cuda()
    with Solver(d, n, smoother="learned", nu1=1, nu2=1) as S:
        kept, rho_rb, rho = S.smoother_select(f, {l: w for l in range(L)})
        assert kept == [] and rho == rho_rb
        assert _blob_levels(S.smoother_save(), L, 27) == []
        ul = u0.clone()
        S.cycles(f, ul, 3)
    with Solver(d, n, nu1=1, nu2=1) as R:
        ur = u0.clone()
        R.cycles(f, ur, 3)
    assert torch.equal(ul, ur)
