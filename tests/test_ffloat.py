"""Float-float arithmetic for FP64-accurate stencils on the FP32 pipe
(csrc/ffloat.cuh): exact double <-> float-pair conversions by integer
operations, correct rounding back to double, error-free transforms, the pair
sum and product within their bounds, and one row of the fermion operator
within 1e-13 of long double arithmetic. A host program built from the header
(tests/c/ffloat_check.cu) runs 2.5M checks. Runs on the CPU; needs nvcc."""
import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_float_float_arithmetic(tmp_path):
    nvcc = os.environ.get("NVCC") or shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(nvcc) and shutil.which(nvcc) is None:
        pytest.skip("nvcc not found")
    exe = str(tmp_path / "ffloat_check")
    r = subprocess.run([nvcc, "-O2", "-std=c++17", "-gencode", "arch=compute_103a,code=sm_103a",
                        "-I", os.path.join(ROOT, "paper_1804_07195_gb300", "csrc"),
                        os.path.join(ROOT, "tests", "c", "ffloat_check.cu"), "-o", exe],
                       capture_output=True, text=True, timeout=300)
    assert r.returncode == 0, r.stderr
    r = subprocess.run([exe], capture_output=True, text=True, timeout=300)
    assert r.returncode == 0, r.stdout + r.stderr
    assert " 0 failures" in r.stdout
