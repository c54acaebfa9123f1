"""The fused leg kernels' CTA algorithm (csrc/legs.cuh) emulated on the host
(tests/legs_host_check.cpp): one thread, plain box copies in place of the
TMA loads, random stale shared memory and random padding entries.  Every
case must equal the unfused sequence (half sweeps, red residual and
full-weighting restriction; black prolongation and half sweeps) bit for bit,
with every box start 16-byte aligned and every box inside the shared-memory
window; the build uses AddressSanitizer where the compiler has it, so a read
outside the shared-memory buffer or a level array fails the run."""
import os
import shutil
import subprocess

import pytest

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(ROOT, "paper_1208_4247_gb300", "csrc")


def _build(gxx, cuda_inc, exe, asan):
    flags = ["-fsanitize=address", "-fno-omit-frame-pointer"] if asan else []
    cmd = [gxx, "-std=c++17", "-O1", "-g", "-ffp-contract=off", *flags, "-I", CSRC, "-I",
           cuda_inc, os.path.join(HERE, "legs_host_check.cpp"), "-o", exe]
    return subprocess.run(cmd, capture_output=True, text=True).returncode == 0


@pytest.fixture(scope="module")
def rows(tmp_path_factory):
    gxx = shutil.which("g++")
    cuda_inc = "/usr/local/cuda/include"
    if not gxx or not os.path.exists(os.path.join(cuda_inc, "cuda_runtime.h")):
        pytest.skip("needs g++ and the CUDA headers")
    exe = str(tmp_path_factory.mktemp("legs") / "legs_host_check")
    if not _build(gxx, cuda_inc, exe, True):
        assert _build(gxx, cuda_inc, exe, False), "legs_host_check.cpp does not build"
    out = subprocess.run([exe], check=True, capture_output=True, text=True, timeout=900).stdout
    res = {}
    for line in out.strip().splitlines():
        name, mism, bad = line.split()
        res[name] = (int(mism), int(bad))
    return res


def test_every_case_ran(rows):
    assert len(rows) == 16
    kinds = {(k.split("_")[0], k.split("_")[1]) for k in rows}
    assert kinds == {("f32", "down"), ("f32", "up"), ("df", "down"), ("df", "up")}


def test_fused_legs_equal_unfused_bit_for_bit(rows):
    for name, (mism, bad) in rows.items():
        assert mism == 0, (name, mism)
        assert bad == 0, (name, bad)
