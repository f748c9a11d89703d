"""The C-ABI library builds, loads without a GPU and exports every function
that include/hmc.h declares; the Python binding declares the same set."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def header_functions():
    txt = open(os.path.join(ROOT, "include", "hmc.h")).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    return sorted(set(re.findall(r"\b(hmc_[A-Za-z0-9_]+)\s*\(", txt)))


@pytest.fixture(scope="module")
def lib():
    from paper_1804_07195_gb300 import build
    path = build.build()
    return ctypes.CDLL(path)


def test_header_declares_the_hot_path_calls():
    names = header_functions()
    for f in ("hmc_apply_M", "hmc_apply_Mdag", "hmc_solve_cg", "hmc_solve_fgmres", "hmc_force",
              "hmc_md_trajectory"):
        assert f in names


def test_every_declared_symbol_is_exported(lib):
    missing = [f for f in header_functions() if not hasattr(lib, f)]
    assert not missing, missing


def test_binding_covers_the_header():
    from paper_1804_07195_gb300 import _abi
    assert sorted(_abi.PROTOTYPES) == header_functions()


def test_host_only_calls(lib):
    from paper_1804_07195_gb300 import _abi
    L = _abi.load()
    assert L.hmc_abi_version() == 1
    assert L.hmc_status_string(0) == b"ok"
    assert L.hmc_status_string(-3) == b"solver did not converge"
    # invalid lattices are rejected before any CUDA call
    h = ctypes.c_void_p()
    bad = _abi.hmc_lattice(0, 3, 8, 1.0, 2.0, 4.0)
    assert L.hmc_create(ctypes.byref(h), ctypes.byref(bad), None) == _abi.HMC_ERR_INVALID
    bad = _abi.hmc_lattice(3, 3, 1, 1.0, 2.0, 4.0)
    assert L.hmc_create(ctypes.byref(h), ctypes.byref(bad), None) == _abi.HMC_ERR_INVALID
    assert L.hmc_destroy(None) == _abi.HMC_ERR_INVALID
    assert L.hmc_apply_M(None, None, 0.0, None, None, 64) == _abi.HMC_ERR_INVALID


def test_product_never_imports_the_oracle():
    pkg = os.path.join(ROOT, "paper_1804_07195_gb300")
    for dirpath, _, files in os.walk(pkg):
        for f in files:
            if f.endswith((".py", ".cu", ".cuh", ".h")):
                src = open(os.path.join(dirpath, f)).read()
                assert "oracle" not in re.findall(r"(?:import|from)\s+(\w+)", src), f


@pytest.mark.parametrize("params", [
    (4096, 4096, 32, 1.0, 2.0, 4.0),          # exactly 2^30 sites: above the index range
    (1 << 20, 1 << 20, 1 << 20, 1.0, 2.0, 4.0),  # n*m*nt overflows 32 bits
    (5, (1 << 30) + 1, 1 << 30, 1.0, 2.0, 4.0),  # 2*n*m*nt overflows signed 64 bits
    ((1 << 31) - 1, (1 << 31) - 1, (1 << 31) - 1, 1.0, 2.0, 4.0),  # every factor at the int limit
    (3, 3, 8, float("nan"), 2.0, 4.0),
    (3, 3, 8, 1.0, float("inf"), 4.0),
    (3, 3, 8, 1.0, 2.0, 0.0),
    (3, 3, 8, 1.0, 0.0, 4.0),                 # U = 0: the Gaussian term 1/(delta U) is undefined
    (3, 3, 8, 1.0, -1.0, 4.0),
    (3, -1, 8, 1.0, 2.0, 4.0),
])
def test_invalid_lattices_are_rejected_before_any_cuda_call(lib, params):
    from paper_1804_07195_gb300 import _abi
    L = _abi.load()
    h = ctypes.c_void_p()
    lat = _abi.hmc_lattice(*params)
    assert L.hmc_create(ctypes.byref(h), ctypes.byref(lat), None) == _abi.HMC_ERR_INVALID
    assert not h.value


def test_largest_accepted_lattice_passes_validation(lib):
    """2 * 4096 * 4096 * 31 sites (just under 2^30) passes the size check: without
    a GPU the create call then fails in CUDA, not as an invalid argument."""
    torch = pytest.importorskip("torch")
    if torch.cuda.is_available():
        pytest.skip("would allocate tens of GB on the device")
    from paper_1804_07195_gb300 import _abi
    L = _abi.load()
    h = ctypes.c_void_p()
    lat = _abi.hmc_lattice(4096, 4096, 31, 1.0, 2.0, 4.0)
    assert L.hmc_create(ctypes.byref(h), ctypes.byref(lat), None) in (_abi.HMC_ERR_CUDA, _abi.HMC_ERR_NOMEM)
    assert not h.value


def test_every_status_has_its_own_message(lib):
    from paper_1804_07195_gb300 import _abi
    L = _abi.load()
    codes = [_abi.HMC_OK, _abi.HMC_ERR_INVALID, _abi.HMC_ERR_CUDA, _abi.HMC_ERR_NOT_CONVERGED,
             _abi.HMC_ERR_NAN, _abi.HMC_ERR_TIMEOUT, _abi.HMC_ERR_NOMEM]
    msgs = [L.hmc_status_string(c) for c in codes]
    assert all(m and m != b"unknown status" for m in msgs) and len(set(msgs)) == len(codes)
    assert L.hmc_status_string(-99) == b"unknown status"
    assert L.hmc_last_error(None) == b""


# 16-byte aligned stand-ins for device pointers: every lattice below is rejected
# before the first CUDA call, so none of them is ever dereferenced
FAKE_PHI, FAKE_IN, FAKE_OUT = 0x10000, 0x20000000, 0x40000000


@pytest.mark.parametrize("params", [
    (5, (1 << 30) + 1, 1 << 30, 1.0, 2.0, 4.0),
    (4096, 4096, 32, 1.0, 2.0, 4.0),
    (3, 3, 8, float("nan"), 2.0, 4.0),
    (3, 3, 8, 1.0, 2.0, float("inf")),
    (3, 3, 8, 1.0, 0.0, 4.0),
    (0, 3, 8, 1.0, 2.0, 4.0),
])
def test_noalloc_rejects_what_create_rejects(lib, params):
    """The allocation-free entry point validates its lattice with the same
    checks as hmc_create (overflow-safe sizes, finite couplings), before any
    CUDA call."""
    from paper_1804_07195_gb300 import _abi
    L = _abi.load()
    lat = _abi.hmc_lattice(*params)
    h = ctypes.c_void_p()
    assert L.hmc_create(ctypes.byref(h), ctypes.byref(lat), None) == _abi.HMC_ERR_INVALID
    st = L.hmc_apply_MMdag_noalloc(ctypes.byref(lat), ctypes.c_void_p(FAKE_PHI), 0.0, 0.0,
                                   ctypes.c_void_p(FAKE_IN), ctypes.c_void_p(FAKE_OUT), None)
    assert st == _abi.HMC_ERR_INVALID


@pytest.mark.parametrize("shift_bytes", [0, 16, 16 * 8])
def test_noalloc_rejects_overlapping_vectors(lib, shift_bytes):
    """in and out that share any byte (not only identical pointers) are rejected."""
    torch = pytest.importorskip("torch")
    if torch.cuda.is_available():
        pytest.skip("CPU-only check with stand-in pointers")
    from paper_1804_07195_gb300 import _abi
    L = _abi.load()
    lat = _abi.hmc_lattice(3, 3, 8, 1.0, 2.0, 4.0)
    st = L.hmc_apply_MMdag_noalloc(ctypes.byref(lat), ctypes.c_void_p(FAKE_PHI), 0.0, 0.0,
                                   ctypes.c_void_p(FAKE_IN), ctypes.c_void_p(FAKE_IN + shift_bytes), None)
    assert st == _abi.HMC_ERR_INVALID
