"""The C ABI from C: tests/c/hmc_example.c links against libhmc.so and the CUDA
runtime, reads phi and b from a file, applies M and solves (M M^dagger) x = b
with FP64 CG. Without a GPU the program must report hmc_create's error status
and exit cleanly; on a GPU its outputs match the oracle."""
import os
import shutil
import subprocess

import numpy as np
import pytest

import workloads as W
from oracle import fermion as of
from oracle.lattice import Lattice as OLat

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def cuda_home():
    for c in (os.environ.get("CUDA_HOME"), "/usr/local/cuda"):
        if c and os.path.exists(os.path.join(c, "include", "cuda_runtime_api.h")):
            return c
    return None


def build_example(tmp_path):
    cc = shutil.which("gcc") or shutil.which("cc")
    cuda = cuda_home()
    if cc is None or cuda is None:
        pytest.skip("no C compiler or CUDA toolkit headers")
    from paper_1804_07195_gb300 import build
    lib = build.build()
    libdir = os.path.dirname(lib)
    cudalib = os.path.join(cuda, "lib64")
    exe = str(tmp_path / "hmc_example")
    cmd = [cc, "-std=c11", "-O2", "-I", os.path.join(ROOT, "include"), "-I", os.path.join(cuda, "include"),
           os.path.join(ROOT, "tests", "c", "hmc_example.c"), "-o", exe, "-L", libdir, "-lhmc",
           "-L", cudalib, "-lcudart", f"-Wl,-rpath,{libdir}", f"-Wl,-rpath,{cudalib}"]
    r = subprocess.run(cmd, capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
    return exe


def run_example(exe, w, tmp_path):
    n, m, nt = w.lat.n, w.lat.m, w.lat.nt
    inp, out = tmp_path / "in.bin", tmp_path / "out.bin"
    np.concatenate([w.phi, w.b.view(np.float64)]).astype(np.float64).tofile(inp)
    r = subprocess.run([exe, str(n), str(m), str(nt), str(inp), str(out)], capture_output=True, text=True,
                       timeout=300)
    return r, out


def test_c_caller_without_gpu_reports_the_status(tmp_path):
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present; the GPU test covers this program")
    exe = build_example(tmp_path)
    w = W.small(3, 2, 6, seed=31, U=2.0, beta=4.0)
    r, _ = run_example(exe, w, tmp_path)
    assert r.returncode == 0, r.stderr
    lines = r.stdout.splitlines()
    assert lines[0] == "abi 1"
    status = int(lines[1].split()[1])
    assert status == -2, r.stdout  # HMC_ERR_CUDA: no device


@pytest.mark.gpu
def test_c_caller_matches_the_oracle(tmp_path):
    import torch
    if not torch.cuda.is_available():
        pytest.skip("needs a GPU")
    exe = build_example(tmp_path)
    w = W.small(3, 2, 6, seed=31, U=2.0, beta=4.0)
    r, out = run_example(exe, w, tmp_path)
    assert r.returncode == 0, r.stderr
    assert "create 0" in r.stdout and "apply_M 0" in r.stdout and "solve_cg 0" in r.stdout, r.stdout
    N = w.lat.nsites
    res = np.fromfile(out, dtype=np.float64).view(np.complex128)
    mb, x = res[:N], res[N:]
    ol = OLat.from_params(w.lat)
    ref = of.apply_M(ol, w.phi, 0.3, w.b)
    assert np.abs(mb - ref).max() <= 1e-12 * np.abs(ref).max()
    resid = w.b - of.apply_MMdag(ol, w.phi, 0.3, x)
    assert np.linalg.norm(resid) <= 1e-11 * np.linalg.norm(w.b)
