"""The fixed-point scaled residual (csrc/fx.cuh) built for the host and
checked against binary128 (tests/fx_host_check.cpp): within 2^-48 of sigma
(plus the subnormal floats' spacing) on converging, random-magnitude,
exactly cancelling and zero-operand cases in 2D and 3D; the FP64 fallback
only for special operands and results below the float range."""
import os
import shutil
import subprocess

import pytest

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(ROOT, "paper_1208_4247_gb300", "csrc")


@pytest.fixture(scope="module")
def report(tmp_path_factory):
    gxx = shutil.which("g++")
    cuda_inc = "/usr/local/cuda/include"
    if not gxx or not os.path.exists(os.path.join(cuda_inc, "cuda_runtime.h")):
        pytest.skip("needs g++ and the CUDA headers")
    exe = str(tmp_path_factory.mktemp("fx") / "fx_host_check")
    r = subprocess.run([gxx, "-std=c++17", "-O2", "-ffp-contract=off", "-I", CSRC, "-I", cuda_inc,
                        os.path.join(HERE, "fx_host_check.cpp"), "-o", exe, "-lquadmath"],
                       capture_output=True, text=True)
    if r.returncode != 0:
        pytest.skip("binary128 (libquadmath) not available: " + r.stderr[-200:])
    out = subprocess.run([exe], check=True, capture_output=True, text=True, timeout=600).stdout
    rows = {}
    for line in out.strip().splitlines():
        name, cases, fails, worst = line.split()
        rows[name] = (int(cases), int(fails), float(worst))
    return rows


@pytest.mark.parametrize("name", ["converging3d", "random3d", "cancel3d", "zeros3d",
                                  "converging2d", "random2d", "special"])
def test_fixed_point_sigma(report, name):
    cases, fails, worst = report[name]
    assert cases >= 6
    assert fails == 0, (name, fails)
    assert worst <= 1.01, (name, worst)
