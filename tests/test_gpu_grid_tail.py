"""The grid tail (GMG_GRID_TAIL_N, off by default): the middle and small
levels of a V-cycle (n <= 128) in one cooperative launch with grid barriers
between the steps, the smallest levels in one CTA.  Its arithmetic is the
level kernels' node for node, so the iterates must equal those of the
per-level kernels plus the single-CTA tail bit for bit, in every precision
and at every threshold."""
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


def _cycles(torch, monkeypatch, d, n, prec, env, cycles=2, nu=2):
    from paper_1208_4247_gb300.gmg import Solver
    for k in ("GMG_GRID_TAIL_N", "GMG_GRID_TAIL_CTA_N", "GMG_GRID_TAIL_CLUSTER"):
        monkeypatch.delenv(k, raising=False)
    for k, v in env.items():
        monkeypatch.setenv(k, v)
    f = torch.from_numpy(inputs.rhs_uniform(d, n, 8)).cuda()
    u = torch.zeros_like(f)
    kw = dict(precision=prec, nu1=nu, nu2=nu)
    if prec != "fp64":
        kw["inner_cycles"] = 1 if prec == "df" else 2
    with Solver(d, n, **kw) as S:
        rel = S.cycles(f, u, cycles)
    return u.cpu().numpy(), rel


CASES = [
    (3, 256, "df"), (3, 256, "fp64"), (3, 256, "fp32"), (3, 256, "bf16"),
    (3, 128, "df"), (3, 64, "fp64"), (3, 512, "fp32"), (2, 1024, "fp64"), (2, 1024, "df"),
]


@pytest.mark.parametrize("case", CASES, ids=lambda c: "-".join(map(str, c)))
def test_grid_tail_bit_identical(torch_cuda, monkeypatch, case):
    d, n, prec = case
    ref, rel_ref = _cycles(torch_cuda, monkeypatch, d, n, prec, {"GMG_GRID_TAIL_N": "0"})
    got, rel = _cycles(torch_cuda, monkeypatch, d, n, prec, {"GMG_GRID_TAIL_N": "128"})
    assert np.array_equal(got, ref)
    assert rel == rel_ref


@pytest.mark.parametrize("cta_n,top", [(2, 128), (16, 128), (32, 64), (8, 32)])
def test_grid_tail_thresholds(torch_cuda, monkeypatch, cta_n, top):
    """Where the grid part starts and where one CTA takes over changes no bit
    (double-float 3D 257^3, V(1,1) and V(2,2))."""
    for nu in (1, 2):
        ref, _ = _cycles(torch_cuda, monkeypatch, 3, 256, "df", {"GMG_GRID_TAIL_N": "0"}, nu=nu)
        got, _ = _cycles(torch_cuda, monkeypatch, 3, 256, "df",
                         {"GMG_GRID_TAIL_N": str(top), "GMG_GRID_TAIL_CTA_N": str(cta_n)}, nu=nu)
        assert np.array_equal(got, ref), (cta_n, top, nu)


@pytest.mark.parametrize("cluster,top,prec", [(8, 32, "df"), (16, 64, "df"), (16, 32, "fp32"),
                                              (8, 64, "fp64")])
def test_cluster_tail_bit_identical(torch_cuda, monkeypatch, cluster, top, prec):
    """The same steps run by one thread-block cluster (hardware cluster
    barrier between the steps, GMG_GRID_TAIL_CLUSTER): bit for bit the
    per-level kernels' iterates (3D 257^3, two cycles)."""
    ref, rel_ref = _cycles(torch_cuda, monkeypatch, 3, 256, prec, {"GMG_GRID_TAIL_N": "0"})
    got, rel = _cycles(torch_cuda, monkeypatch, 3, 256, prec,
                       {"GMG_GRID_TAIL_N": str(top), "GMG_GRID_TAIL_CLUSTER": str(cluster)})
    assert np.array_equal(got, ref)
    assert rel == rel_ref
