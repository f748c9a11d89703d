"""The float-float operator stencils (csrc/operator_ff.cuh: M and M^dagger of
Eq. ferm_op on the FP32 pipe with FP64 accuracy), run over whole lattices by a
host program built from the same header, against the oracle element by
element within 1e-13 of the largest entry (ten times tighter than the FP64
parity bar): lattices with n or m of 1 to 3 (every wrap, coinciding bonds),
odd nt and n != m, with and without a staggered mass. CPU only; needs nvcc."""
import os
import shutil
import subprocess

import numpy as np
import pytest

import workloads as W
from oracle import fermion as of
from oracle.lattice import Lattice as OLat

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def exe(tmp_path_factory):
    nvcc = os.environ.get("NVCC") or shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(nvcc) and shutil.which(nvcc) is None:
        pytest.skip("nvcc not found")
    out = str(tmp_path_factory.mktemp("ff") / "ff_stencil_check")
    r = subprocess.run([nvcc, "-O2", "-std=c++17", "-gencode", "arch=compute_103a,code=sm_103a",
                        "-I", os.path.join(ROOT, "paper_1804_07195_gb300", "csrc"),
                        os.path.join(ROOT, "tests", "c", "ff_stencil_check.cu"), "-o", out],
                       capture_output=True, text=True, timeout=300)
    assert r.returncode == 0, r.stderr
    return out


@pytest.mark.parametrize("shape", [(1, 1, 2), (2, 1, 4), (1, 3, 5), (3, 3, 8), (4, 5, 6), (7, 3, 10), (6, 6, 16)])
@pytest.mark.parametrize("ms", [0.0, 0.37])
def test_float_float_stencil_matches_the_oracle(exe, tmp_path, shape, ms):
    w = W.small(*shape, seed=500 + sum(shape))
    p = w.lat
    ol = OLat.from_params(p)
    inp, outp = tmp_path / "in.bin", tmp_path / "out.bin"
    with open(inp, "wb") as f:
        np.array([p.n, p.m, p.nt], dtype=np.int32).tofile(f)
        np.array([p.delta, p.kappa, ms], dtype=np.float64).tofile(f)
        w.phi.astype(np.float64).tofile(f)
        w.b.astype(np.complex128).tofile(f)
    r = subprocess.run([exe, str(inp), str(outp)], capture_output=True, text=True, timeout=120)
    assert r.returncode == 0, r.stderr
    out = np.fromfile(outp, dtype=np.complex128)
    N = p.nsites
    gotM, gotD = out[:N], out[N:]
    refM = of.apply_M(ol, w.phi, ms, w.b)
    refD = of.apply_Mdag(ol, w.phi, ms, w.b)
    assert np.abs(gotM - refM).max() <= 1e-13 * np.abs(refM).max()
    assert np.abs(gotD - refD).max() <= 1e-13 * np.abs(refD).max()
