"""The Python binding is marshalling only and never falls back to the CPU:
CPU tensors are refused before any library call, vector precisions map to the
ABI's 64/32 codes, and without a GPU a context cannot be made. CPU only."""
import pytest

torch = pytest.importorskip("torch")

import paper_1804_07195_gb300 as hmc  # noqa: E402


def test_cpu_tensors_are_refused():
    for t in (torch.zeros(8, dtype=torch.float64), torch.zeros(8, dtype=torch.complex128)):
        with pytest.raises(ValueError, match="CUDA tensor"):
            hmc._ptr(t, t.dtype, 8, "x")
    assert hmc._ptr(None) is None


def test_precision_codes():
    assert hmc._prec(torch.zeros(2, dtype=torch.complex128)) == 64
    assert hmc._prec(torch.zeros(2, dtype=torch.complex64)) == 32
    with pytest.raises(TypeError):
        hmc._prec(torch.zeros(2, dtype=torch.float64))


def test_no_context_without_a_gpu():
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    with pytest.raises(RuntimeError):
        hmc.Context(hmc.Lattice(3, 3, 8, 1.0, 2.0, 4.0))
    with pytest.raises((RuntimeError, ValueError)):
        hmc.apply_MMdag_noalloc(hmc.Lattice(3, 3, 8, 1.0, 2.0, 4.0), torch.zeros(144, dtype=torch.float64), 0.0,
                                torch.zeros(144, dtype=torch.complex128))


def test_missing_library_raises(tmp_path, monkeypatch):
    """Without the built libhmc.so the package raises; nothing else computes."""
    from paper_1804_07195_gb300 import _abi
    monkeypatch.setattr(_abi, "_lib", None)
    with pytest.raises(RuntimeError, match="no CPU fallback"):
        _abi.load(str(tmp_path / "libhmc.so"))
