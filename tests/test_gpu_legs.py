"""Fused leg kernels on the GPU (csrc/legs.cu): the down leg (pre-smoothing
half sweeps, red residual, full-weighting restriction) and the up leg
(black prolongation + correction, post-smoothing half sweeps) as one
z-streamed pass each over the large 3D levels of the FP32 and double-float
inner hierarchies, planes staged by TMA.  They must reproduce the unfused
cycle bit for bit (GMG_FUSED_LEGS=0 at handle creation selects it), also
with other z-segment splits of the CTAs and with sweep counts that leave a
level unfused; the forms' own tests (test_gpu_df, test_gpu_mixed) check the
fused solves against the oracle."""
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


def _steps(torch, monkeypatch, prec, n, nu1, nu2, k, steps, legs, segs=None, timing=False):
    from paper_1208_4247_gb300.gmg import Solver
    monkeypatch.setenv("GMG_FUSED_LEGS", "1" if legs else "0")
    if segs is None:
        monkeypatch.delenv("GMG_LEG_SEGS", raising=False)
    else:
        monkeypatch.setenv("GMG_LEG_SEGS", str(segs))
    f = torch.from_numpy(inputs.rhs_uniform(3, n, 11)).cuda()
    rng = np.random.default_rng(5)
    u0 = np.zeros((n + 1,) * 3)
    u0[1:-1, 1:-1, 1:-1] = rng.standard_normal((n - 1,) * 3)
    u = torch.from_numpy(u0).cuda()
    with Solver(3, n, nu1=nu1, nu2=nu2, precision=prec, inner_cycles=k) as S:
        if timing:
            S.set_timing(True)
        rel = S.cycles(f, u, steps)
        names = {r["kernel"] for r in S.timing_report()[0]} if timing else set()
    return u.cpu().numpy(), rel, names


CASES = [
    # precision, n, nu1, nu2, inner cycles, steps
    ("fp32", 128, 2, 2, 3, 2),
    ("fp32", 256, 2, 2, 2, 2),
    ("fp32", 512, 2, 2, 3, 1),
    ("fp32", 256, 1, 1, 2, 2),
    ("fp32", 256, 2, 1, 2, 2),
    ("df", 128, 2, 2, 1, 2),
    ("df", 256, 2, 2, 1, 3),
    ("df", 512, 2, 2, 1, 1),
    ("df", 256, 1, 2, 1, 2),
    ("df", 256, 2, 2, 2, 2),
]


@pytest.mark.parametrize("case", CASES, ids=lambda c: "-".join(map(str, c)))
def test_fused_legs_equal_unfused_cycles(torch_cuda, monkeypatch, case):
    prec, n, nu1, nu2, k, steps = case
    uf, rf, names = _steps(torch_cuda, monkeypatch, prec, n, nu1, nu2, k, steps, True,
                           timing=True)
    uu, ru, names_u = _steps(torch_cuda, monkeypatch, prec, n, nu1, nu2, k, steps, False,
                             timing=True)
    assert any(s.startswith("leg_down") for s in names), names
    assert any(s.startswith("leg_up") for s in names), names
    assert not any(s.startswith("leg_") for s in names_u)
    assert np.array_equal(uf, uu)
    assert rf == ru


@pytest.mark.parametrize("segs", [1, 3, 7])
def test_segment_splits_give_the_same_bits(torch_cuda, monkeypatch, segs):
    ref, _, _ = _steps(torch_cuda, monkeypatch, "df", 256, 2, 2, 1, 2, False)
    got, _, _ = _steps(torch_cuda, monkeypatch, "df", 256, 2, 2, 1, 2, True, segs=segs)
    assert np.array_equal(got, ref)
    ref, _, _ = _steps(torch_cuda, monkeypatch, "fp32", 256, 2, 2, 2, 1, False)
    got, _, _ = _steps(torch_cuda, monkeypatch, "fp32", 256, 2, 2, 2, 1, True, segs=segs)
    assert np.array_equal(got, ref)
