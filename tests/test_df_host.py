"""The double-float arithmetic of the library (csrc/df.cuh) built for the
host and checked against exact references (tests/df_host_check.cpp): the
integer-pipe float <-> double conversions bit for bit against the C casts,
TwoSum exactness, the double-word addition / product / compensated sums /
exact-constant division by 6 within their error bounds, and the triple-float
Gauss-Seidel value within 2^-60 (binary128 references)."""
import os
import shutil
import subprocess

import pytest

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(ROOT, "paper_1208_4247_gb300", "csrc")

BOUNDS = {  # check -> largest error the library's comments state (units of the report)
    "widen": 0.0, "split": 0.0, "two_sum": 0.0, "df_add": 4.0, "df_add_fast": 4.0,
    "df_mul": 6.0, "df_sum46": 16.0, "df_sixth": 3.0, "triple_fma": 1.0, "triple_to_double": 1.0,
}


@pytest.fixture(scope="module")
def report(tmp_path_factory):
    gxx = shutil.which("g++")
    cuda_inc = "/usr/local/cuda/include"
    if not gxx or not os.path.exists(os.path.join(cuda_inc, "cuda_runtime.h")):
        pytest.skip("needs g++ and the CUDA headers")
    exe = str(tmp_path_factory.mktemp("df") / "df_host_check")
    subprocess.run([gxx, "-std=c++17", "-O2", "-ffp-contract=off", "-I", CSRC, "-I", cuda_inc,
                    os.path.join(HERE, "df_host_check.cpp"), "-o", exe], check=True)
    out = subprocess.run([exe], check=True, capture_output=True, text=True, timeout=600).stdout
    rows = {}
    for line in out.strip().splitlines():
        name, cases, fails, worst = line.split()
        rows[name] = (int(cases), int(fails), float(worst))
    return rows


@pytest.mark.parametrize("name", sorted(BOUNDS))
def test_df_arithmetic(report, name):
    cases, fails, worst = report[name]
    assert cases > 1000
    assert fails == 0, (name, fails, worst)
    assert worst <= BOUNDS[name], (name, worst)
