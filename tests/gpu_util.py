"""Shared helpers of the GPU parity tests (no arithmetic of the method)."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")


def need_gpu():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


def ctx_for(params):
    import paper_1804_07195_gb300 as hmc
    from paper_1804_07195_gb300 import build
    build.build()
    lat = hmc.Lattice(params.n, params.m, params.nt, params.kappa, params.U, params.beta)
    return hmc.Context(lat)


def dev(a):
    return torch.tensor(np.ascontiguousarray(a), device="cuda")


def host(t):
    return t.detach().cpu().numpy()


def rel_max(got, ref):
    return float(np.abs(got - ref).max() / max(np.abs(ref).max(), 1e-300))
