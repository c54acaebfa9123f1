"""The cuFFT DST-I direct solve of the FD system: exact on sine modes, equal
to the dense direct solve on small grids and to the converged oracle
multigrid solution (1e-9 relative) at the 257^3 workload."""
import numpy as np
import pytest

import oracle
import dense_mg as dm
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


@pytest.mark.parametrize("d,n", [(2, 16), (3, 8), (2, 64), (3, 32)])
def test_sine_mode_and_dense(torch_cuda, d, n):
    torch = torch_cuda
    from paper_1208_4247_gb300.gmg import FFTSolver
    x = np.arange(n + 1) / n
    ks = [3, 1, 2][:d]
    modes = [np.sin(k * np.pi * x) for k in ks]
    phi = modes[0][None, :] * modes[1][:, None] if d == 2 else \
        modes[0][None, None, :] * modes[1][None, :, None] * modes[2][:, None, None]
    phi = np.ascontiguousarray(phi)
    lam = sum(4 * np.sin(k * np.pi / (2 * n)) ** 2 for k in ks)
    f = phi * n ** 2  # h^2 f = phi
    with FFTSolver(d, n) as F:
        u = torch.zeros((n + 1,) * d, dtype=torch.float64, device="cuda")
        F.solve(torch.from_numpy(f).cuda(), u)
        ug = u.cpu().numpy()
        inner = (slice(1, -1),) * d
        np.testing.assert_allclose(ug[inner], phi[inner] / lam, rtol=0, atol=1e-13 / lam)
        if (n - 1) ** d <= 2000:
            rng = np.random.default_rng(0)
            g = dm.from_vec(rng.uniform(-1, 1, (n - 1) ** d), d, n)
            F.solve(torch.from_numpy(g).cuda(), u)
            ref = np.linalg.solve(dm.lap(d, n), dm.to_vec(g) / n ** 2)
            np.testing.assert_allclose(dm.to_vec(u.cpu().numpy()), ref, rtol=0,
                                       atol=1e-12 * np.max(np.abs(ref)))


def test_matches_converged_multigrid_257(torch_cuda):
    torch = torch_cuda
    from paper_1208_4247_gb300.gmg import FFTSolver
    d, n = 3, 256
    f = inputs.rhs_uniform(d, n, 2)
    uo = np.zeros_like(f)
    oracle.solve(oracle.make_cfg(d, n, 0, oracle.RBGS, 0.8, 2, 2, 1), f, uo, 1e-13, 100)
    with FFTSolver(d, n) as F:
        u = torch.zeros_like(torch.from_numpy(f)).cuda()
        F.solve(torch.from_numpy(f).cuda(), u)
    ug = u.cpu().numpy()
    assert np.linalg.norm(ug - uo) <= 1e-9 * np.linalg.norm(uo)
    b = oracle.scale_rhs(f)
    assert oracle.norm2(oracle.residual(b, ug)) / oracle.norm2(b) <= 1e-11
