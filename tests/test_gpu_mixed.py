"""Mixed-precision form: FP32 and BF16-storage V-cycles inside FP64 iterative
refinement, against the CPU FP64 oracle.

Bars: the FP64 relative residual of the result (evaluated by the oracle)
<= 1e-10 and ||u - u_oracle|| / ||u_oracle|| <= 1e-9 (oracle solved to
1e-12).  Element-wise check of the inner kernels: one refinement step from
u = 0 with a single inner cycle is one V-cycle in the inner precision, and
must match the oracle's FP64 V-cycle within that precision's tolerance:
FP32 (unit roundoff 6e-8) 2e-5, BF16 storage (unit roundoff 3.9e-3) 3e-2 --
about 300 / 8 roundoffs of the stored values, covering the rounding of q,
e and r at every level.
"""
import numpy as np
import pytest

import oracle
from paper_1208_4247_gb300 import inputs

pytestmark = pytest.mark.gpu

INNER_TOL = {"fp32": 2e-5, "bf16": 3e-2}


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


@pytest.mark.parametrize("prec", ["fp32", "bf16"])
@pytest.mark.parametrize("d,n,sm,om", [(3, 64, "rbgs", 0.8), (2, 128, "wjacobi", 0.8),
                                       (3, 32, "wjacobi", 6 / 7)])
def test_one_inner_cycle_matches_fp64_cycle(torch_cuda, prec, d, n, sm, om):
    torch = torch_cuda
    from paper_1208_4247_gb300.gmg import Solver
    f = inputs.rhs_uniform(d, n, 3)
    smo = oracle.RBGS if sm == "rbgs" else oracle.WJACOBI
    uo = np.zeros_like(f)
    oracle.vcycle(oracle.make_cfg(d, n, 0, smo, om, 2, 2, 1), oracle.scale_rhs(f), uo)
    ud = torch.zeros_like(_dev(torch, f))
    with Solver(d, n, smoother=sm, omega=om, precision=prec, inner_cycles=1) as S:
        S.cycles(_dev(torch, f), ud, 1)
    assert _rel(ud.cpu().numpy(), uo) <= INNER_TOL[prec]


@pytest.mark.parametrize("prec,k", [("fp32", 5), ("fp32", 3), ("bf16", 2), ("bf16", 1)])
@pytest.mark.parametrize("d,n,sm,om,nu", [(3, 128, "rbgs", 0.8, 2), (2, 256, "wjacobi", 0.8, 1),
                                          (3, 64, "wjacobi", 6 / 7, 1)])
def test_refinement_reaches_fp64_accuracy(torch_cuda, prec, k, d, n, sm, om, nu):
    torch = torch_cuda
    from paper_1208_4247_gb300.gmg import Solver
    f = inputs.rhs_sine_plus_gauss(d, n, 3) if d == 3 else inputs.rhs_uniform(d, n, 4)
    uo = np.zeros_like(f)
    smo = oracle.RBGS if sm == "rbgs" else oracle.WJACOBI
    oracle.solve(oracle.make_cfg(d, n, 0, smo, om, 2, 2, 1), f, uo, rtol=1e-12, maxit=100)
    fd = _dev(torch, f)
    ud = torch.zeros_like(fd)
    with Solver(d, n, smoother=sm, omega=om, nu1=nu, nu2=nu, precision=prec,
                inner_cycles=k) as S:
        it, rel, conv = S.solve(fd, ud, rtol=1e-10)
        hist = S.history()
    assert conv and rel <= 1e-10
    assert all(b < a for a, b in zip(hist, hist[1:]))
    ug = ud.cpu().numpy()
    b = oracle.scale_rhs(f)
    assert oracle.norm2(oracle.residual(b, ug)) / oracle.norm2(b) <= 1e-10
    assert _rel(ug, uo) <= 1e-9


@pytest.fixture(scope="module")
def oracle_513():
    """f of the 3D 513^3 workload (3 pi^2 prod sin + 0.01 N(0,1), seed 3) and
    the oracle's FP64 solution (RB-GS V(2,2) to 1e-12), computed once."""
    d, n = 3, 512
    f = inputs.rhs_sine_plus_gauss(d, n, 3)
    uo = np.zeros_like(f)
    oracle.solve(oracle.make_cfg(d, n, 0, oracle.RBGS, 0.8, 2, 2, 1), f, uo, rtol=1e-12, maxit=60)
    return f, uo


# k = 3 (FP32) and k = 1 (BF16) are the inner-cycle counts the benchmark's
# autotuner picks on this workload; k = 5 / 2 are the neighbours it rejects
@pytest.mark.parametrize("prec,k", [("fp32", 3), ("bf16", 1), ("fp32", 5), ("bf16", 2)])
def test_full_size_513(torch_cuda, oracle_513, prec, k):
    """The 3D 513^3 workload, RB-GS V(2,2) inner cycles: FP64 residual
    <= 1e-10 and error vs the oracle's FP64 solution <= 1e-9 (globally and
    node by node)."""
    torch = torch_cuda
    from paper_1208_4247_gb300.gmg import Solver
    d, n = 3, 512
    f, uo = oracle_513
    fd = _dev(torch, f)
    ud = torch.zeros_like(fd)
    with Solver(d, n, precision=prec, inner_cycles=k) as S:
        it, rel, conv = S.solve(fd, ud, rtol=1e-10)
    assert conv
    ug = ud.cpu().numpy()
    del ud, fd
    b = oracle.scale_rhs(f)
    assert oracle.norm2(oracle.residual(b, ug)) / oracle.norm2(b) <= 1e-10
    assert _rel(ug, uo) <= 1e-9
    assert np.max(np.abs(ug - uo)) <= 1e-9 * np.max(np.abs(uo))


def test_fused_sweep_equals_two_half_sweeps(torch_cuda, monkeypatch):
    """GMG_FUSED_RB=1: the fused z-streaming FP32 sweep gives the same V-cycle
    bit for bit (it performs the same updates in the same order per node)."""
    torch = torch_cuda
    from paper_1208_4247_gb300.gmg import Solver
    d, n = 3, 128
    f = torch.from_numpy(inputs.rhs_uniform(d, n, 6)).cuda()
    out = []
    for flag in ("0", "1"):
        monkeypatch.setenv("GMG_FUSED_RB", flag)
        u = torch.zeros_like(f)
        with Solver(d, n, precision="fp32", inner_cycles=2) as S:
            S.cycles(f, u, 2)
        out.append(u.cpu().numpy())
    assert np.array_equal(out[0], out[1])


@pytest.mark.parametrize("prec", ["fp32", "bf16"])
@pytest.mark.parametrize("d,n,sm", [(3, 4, "rbgs"), (3, 8, "wjacobi"), (3, 16, "rbgs"),
                                    (2, 8, "rbgs"), (2, 64, "wjacobi"), (2, 32, "rbgs")])
def test_small_grids_colour_split(torch_cuda, prec, d, n, sm):
    """Tiny grids, where the whole inner hierarchy (colour-split FP32/BF16)
    runs in the single-CTA tail or a single vector group covers a row: the
    refinement still reaches a FP64 residual of 1e-10 and the oracle's
    solution to 1e-9."""
    torch = torch_cuda
    from paper_1208_4247_gb300.gmg import Solver
    f = inputs.rhs_uniform(d, n, 16)
    om = 0.8 if d == 2 else 6 / 7
    smo = oracle.RBGS if sm == "rbgs" else oracle.WJACOBI
    uo = np.zeros_like(f)
    oracle.solve(oracle.make_cfg(d, n, 0, smo, om, 2, 2, 1), f, uo, rtol=1e-13, maxit=200)
    fd = _dev(torch, f)
    ud = torch.zeros_like(fd)
    with Solver(d, n, smoother=sm, omega=om, precision=prec, inner_cycles=2, maxit=200) as S:
        it, rel, conv = S.solve(fd, ud, rtol=1e-10)
    assert conv and rel <= 1e-10
    ug = ud.cpu().numpy()
    b = oracle.scale_rhs(f)
    assert oracle.norm2(oracle.residual(b, ug)) / oracle.norm2(b) <= 1e-10
    assert _rel(ug, uo) <= 1e-9


def test_sweep_refinement_best_entry_matches_oracle(torch_cuda):
    """The sweep over smoother x sweeps x inner cycles (autotune.sweep_refinement)
    on a 65^3 grid returns converged entries, and its fastest setting solves to
    the oracle's FP64 solution within 1e-9."""
    torch = torch_cuda
    from paper_1208_4247_gb300.autotune import sweep_refinement
    from paper_1208_4247_gb300.gmg import Solver
    d, n = 3, 64
    fn = inputs.rhs_sine_plus_gauss(d, n, 3)
    f = _dev(torch, fn)
    u = torch.zeros_like(f)
    rows, best = sweep_refinement(d, n, f, u, "fp32", (("rbgs", 0.8), ("wjacobi", 6 / 7)),
                                  (1, 2), ks=(1, 2, 3))
    assert len(rows) == 12 and best is not None
    assert all(r["ms"] > 0 for r in rows if r["converged"])
    assert sum(r["converged"] for r in rows) >= 6
    with Solver(d, n, precision="fp32", inner_cycles=best["k"], smoother=best["smoother"],
                omega=best["omega"], nu1=best["nu"], nu2=best["nu"], maxit=200) as S:
        u.zero_()
        it, rel, conv = S.solve(f, u, 1e-10)
    assert conv and it == best["steps"]
    ug = u.cpu().numpy()
    uo = np.zeros_like(fn)
    oracle.solve(oracle.make_cfg(d, n, 0, oracle.RBGS, 0.8, 2, 2, 1), fn, uo, rtol=1e-13,
                 maxit=100)
    assert _rel(ug, uo) <= 1e-9
