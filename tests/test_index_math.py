"""The stencil kernels find a site's cell and time slice by multiply-high
division (common.cuh). A host program built from the same header checks the
multiplier and shift against integer division over the whole index range the
library accepts (tests/c/index_math_check.cu). Runs on the CPU; needs nvcc."""
import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_fast_division_is_exact(tmp_path):
    nvcc = os.environ.get("NVCC") or shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(nvcc) and shutil.which(nvcc) is None:
        pytest.skip("nvcc not found")
    exe = str(tmp_path / "index_math_check")
    src = os.path.join(ROOT, "tests", "c", "index_math_check.cu")
    inc = os.path.join(ROOT, "paper_1804_07195_gb300", "csrc")
    r = subprocess.run([nvcc, "-O2", "-std=c++17", "-gencode", "arch=compute_103a,code=sm_103a", "-I", inc, src,
                        "-o", exe], capture_output=True, text=True, timeout=300)
    assert r.returncode == 0, r.stderr
    r = subprocess.run([exe], capture_output=True, text=True, timeout=300)
    assert r.returncode == 0, r.stdout + r.stderr
    assert "0 failures" in r.stdout
