"""The kernels' branch-free deterministic math equals the plain forms the CPU
oracle follows, on every input of the ranges the sampler uses (compiled and
run as a small CUDA program)."""
import os
import shutil
import subprocess

import pytest

pytestmark = pytest.mark.gpu

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)


def test_detmath_exhaustive(tmp_path):
    nvcc = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    exe = str(tmp_path / "detmath_check")
    cmd = [nvcc, "-gencode", "arch=compute_103a,code=sm_103a", "-O3", "-std=c++17", "--fmad=false",
           "-I" + os.path.join(ROOT, "paper_2210_10513_gb300", "csrc"), "-I" + os.path.join(ROOT, "include"),
           os.path.join(HERE, "cuda", "detmath_check.cu"), "-o", exe]
    subprocess.run(cmd, check=True, capture_output=True)
    out = subprocess.run([exe], check=True, capture_output=True, text=True, timeout=300).stdout
    vals = dict(line.split() for line in out.strip().splitlines())
    assert int(vals["div_mismatches"]) == 0
    assert int(vals["exp_mismatches"]) == 0
    for name in ("race", "mult", "k"):
        assert int(vals[name + "_div_compared"]) > 10 ** 9
        assert int(vals[name + "_div_mismatches"]) == 0, name
    assert int(vals["u64_compared"]) > 5 * 10 ** 9 and int(vals["u64_mismatches"]) == 0
    print(vals)
