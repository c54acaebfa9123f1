"""The double-float refinement form (GMG_DF_IR, one inner cycle per step):
each step is the FP64 V-cycle in exact arithmetic, so every step must meet
the plain form's per-cycle bar against the CPU FP64 oracle (node by node
within 1e-12 of max |u|, and in the Euclidean norm), and whole solves take
the oracle's cycle count to a relative residual of 1e-10 with matching
residual histories."""
import numpy as np
import pytest

import oracle
from paper_1208_4247_gb300 import inputs

pytestmark = pytest.mark.gpu

TOL_CYCLE = 1e-12


@pytest.fixture(scope="module")
def torch_cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1208_4247_gb300 import build
    build.build()
    return torch


def _dev(torch, a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def _rel(a, b):
    return np.linalg.norm((a - b).ravel()) / np.linalg.norm(b.ravel())


def _max_rel(a, b):
    return np.max(np.abs(a - b)) / np.max(np.abs(b))


def _floor(d, u, b):
    return np.finfo(float).eps * 2 * d * np.linalg.norm(u.ravel()) / np.linalg.norm(b.ravel())


CYCLE_CASES = [
    # d, n, smoother, omega, nu1, nu2
    (2, 4, "rbgs", 0.8, 2, 2),
    (2, 64, "rbgs", 0.8, 2, 2),
    (2, 256, "wjacobi", 0.8, 2, 2),
    (2, 1024, "rbgs", 0.8, 1, 1),
    (3, 4, "rbgs", 0.8, 2, 2),
    (3, 16, "wjacobi", 6 / 7, 1, 1),
    (3, 32, "rbgs", 0.8, 0, 2),
    (3, 64, "rbgs", 0.8, 2, 2),
    (3, 128, "rbgs", 0.8, 2, 2),
    (3, 128, "wjacobi", 6 / 7, 2, 2),
    (3, 256, "rbgs", 0.8, 2, 2),
    (3, 512, "rbgs", 0.8, 2, 2),
]


def _rhs(d, n):
    if d == 3 and n == 512:
        return inputs.rhs_sine_plus_gauss(d, n, 3)
    return inputs.rhs_uniform(d, n, 2 if (d, n) == (3, 256) else 7)


@pytest.mark.parametrize("case", CYCLE_CASES, ids=lambda c: "-".join(map(str, c)))
def test_df_step_is_the_fp64_cycle(torch_cuda, case):
    torch = torch_cuda
    from paper_1208_4247_gb300.gmg import Solver
    d, n, sm, om, nu1, nu2 = case
    f = _rhs(d, n)
    rng = np.random.default_rng(29)
    u = np.zeros_like(f)
    u[(slice(1, -1),) * d] = rng.standard_normal((n - 1,) * d)
    cfg = oracle.make_cfg(d, n, 0, oracle.RBGS if sm == "rbgs" else oracle.WJACOBI, om, nu1,
                          nu2, 1)
    b = oracle.scale_rhs(f)
    fd = _dev(torch, f)
    with Solver(d, n, smoother=sm, omega=om, nu1=nu1, nu2=nu2, precision="df",
                inner_cycles=1) as S:
        for c in range(3):
            ud = _dev(torch, u)
            rel_gpu = S.cycles(fd, ud, 1)[0]
            ug = ud.cpu().numpy()
            del ud
            uo = u.copy()
            oracle.vcycle(cfg, b, uo)
            assert _rel(ug, uo) <= TOL_CYCLE, (c, _rel(ug, uo))
            assert _max_rel(ug, uo) <= TOL_CYCLE, (c, _max_rel(ug, uo))
            rel_orc = oracle.norm2(oracle.residual(b, uo)) / oracle.norm2(oracle.residual(b, u))
            assert rel_gpu == pytest.approx(rel_orc, rel=1e-6)
            u = ug


SOLVE_CASES = [
    (2, 256, "wjacobi", 0.8, 2, 2, "sine_uniform"),
    (3, 64, "rbgs", 0.8, 2, 2, "uniform"),
    (3, 128, "rbgs", 0.8, 1, 1, "uniform"),
    (3, 256, "rbgs", 0.8, 2, 2, "uniform"),
    (3, 512, "rbgs", 0.8, 2, 2, "sine_gauss"),
]


@pytest.mark.parametrize("case", SOLVE_CASES, ids=lambda c: "-".join(map(str, c)))
def test_df_solve_takes_the_oracle_cycles(torch_cuda, case):
    torch = torch_cuda
    from paper_1208_4247_gb300.gmg import Solver
    d, n, sm, om, nu1, nu2, kind = case
    f = {"sine_uniform": lambda: inputs.rhs_sine_plus_uniform(d, n, 1),
         "uniform": lambda: inputs.rhs_uniform(d, n, 2),
         "sine_gauss": lambda: inputs.rhs_sine_plus_gauss(d, n, 3)}[kind]()
    uo = np.zeros_like(f)
    cfg = oracle.make_cfg(d, n, 0, oracle.RBGS if sm == "rbgs" else oracle.WJACOBI, om, nu1,
                          nu2, 1)
    it_o, hist_o = oracle.solve(cfg, f, uo, rtol=1e-10, maxit=100)
    fd = _dev(torch, f)
    ud = torch.zeros_like(fd)
    with Solver(d, n, smoother=sm, omega=om, nu1=nu1, nu2=nu2, precision="df",
                inner_cycles=1) as S:
        it_g, rel_g, conv = S.solve(fd, ud, rtol=1e-10)
        hist_g = np.array(S.history())
    assert conv and it_g == it_o, (it_g, it_o)
    b = oracle.scale_rhs(f)
    np.testing.assert_allclose(hist_g, hist_o, rtol=1e-6, atol=_floor(d, uo, b))
    ug = ud.cpu().numpy()
    assert _rel(ug, uo) <= 1e-10
    assert _max_rel(ug, uo) <= 1e-10
    assert oracle.norm2(oracle.residual(b, ug)) / oracle.norm2(b) <= 1e-10
