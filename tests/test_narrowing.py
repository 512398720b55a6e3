"""The integer FP64 -> FP32 / BF16 rounding of the mixed-precision copies
(narrow_f64_bits in csrc/spfd_internal.cuh) against the host's FP64 -> FP32
conversion and a bfloat16 rounding written from the format's definition, on
3 M values (every exponent, subnormal results, exact ties, NaN and the
infinities).  Host code only: compiled with nvcc, run on the CPU."""

import os
import shutil
import subprocess

import pytest

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)


def _nvcc():
    cand = os.path.join(os.environ.get("CUDA_HOME", "/usr/local/cuda"), "bin", "nvcc")
    return cand if os.path.exists(cand) else shutil.which("nvcc")


def test_narrowing_matches_references(tmp_path):
    nvcc = _nvcc()
    if not nvcc:
        pytest.skip("nvcc not available")
    exe = str(tmp_path / "narrowing_check")
    cmd = [nvcc, "-O2", "-std=c++17", "-gencode", "arch=compute_103a,code=sm_103a",
           "-I" + os.path.join(ROOT, "include"),
           "-I" + os.path.join(ROOT, "paper_2010_12879_gb300", "csrc"),
           os.path.join(HERE, "narrowing_check.cu"), "-o", exe]
    b = subprocess.run(cmd, capture_output=True, text=True)
    assert b.returncode == 0, b.stderr[-2000:]
    r = subprocess.run([exe], capture_output=True, text=True, timeout=300)
    assert r.returncode == 0, r.stdout[-2000:]
    assert r.stdout.startswith("ok ")
