"""Single-particle correlators and their energies (Section 8.1).

The particle propagator is M[phi]^{-1}; on a configuration its column for a
source b is M^{-1} b = M^dagger (M M^dagger)^{-1} b (one CG solve and one
M^dagger). For the band at lattice momentum k the source is the orbital
o_k = (A_k + B_k)/sqrt(2) on time slice t0 (A_k, B_k the plane waves on the two
sublattices); the correlator is
    C_k(tau) = < sum_x conj(o_k(x)) [M^{-1} o_k](x, t0 + tau) >,
averaged over configurations and source slices t0, with the anti-periodic
sign when t0 + tau wraps. For large tau it falls as exp(-E_k tau); E_k is taken
from an exponential fit in a window of tau (the windows of Section 8.1:
tau kappa in [0.2, 1] at Gamma and [0.6, 2] at M).
"""
from __future__ import annotations

import math
from typing import Sequence, Tuple

import numpy as np


def band_orbital(n: int, m: int, k1: float, k2: float = 0.0) -> np.ndarray:
    """Coefficients of o_k over the 2nm sites of one time slice (A cells then B
    cells, cell index j*n + i)."""
    V = n * m
    o = np.zeros(2 * V, complex)
    for j in range(m):
        for i in range(n):
            ph = np.exp(1j * (k1 * i + k2 * j)) / math.sqrt(2 * V)
            o[j * n + i] = ph
            o[V + j * n + i] = ph
    return o


def slice_indices(n: int, m: int, nt: int, t: int) -> np.ndarray:
    """Canonical indices of the 2nm sites of time slice t, in band_orbital order."""
    V = n * m
    idx = np.empty(2 * V, dtype=np.int64)
    for s in range(2):
        for c in range(V):
            idx[s * V + c] = (s * nt + t) * V + c
    return idx


def correlator(ctx, lat, phi, orbital: np.ndarray, t0s: Sequence[int], tol: float = 1e-12) -> np.ndarray:
    """C(tau) on one configuration, averaged over the source slices t0s. The
    vectors live on phi's device (the GPU: the context's solves run there)."""
    import torch
    n, m, nt = lat.n, lat.m, lat.nt
    N = lat.nsites
    dev = phi.device
    o = torch.tensor(orbital, device=dev)
    out = torch.zeros(nt, dtype=torch.complex128, device=dev)
    ctx.load_field(phi)
    idx = torch.tensor(np.stack([slice_indices(n, m, nt, t) for t in range(nt)]), device=dev)  # (nt, 2V)
    for t0 in t0s:
        b = torch.zeros(N, dtype=torch.complex128, device=dev)
        b[idx[t0]] = o
        y, _ = ctx.solve_cg(None, 0.0, b, tol=tol)
        col = ctx.apply_Mdag(None, 0.0, y)
        per_t = col[idx] @ o.conj()                 # projection on every slice t
        tau = torch.arange(nt, device=dev)
        t = (t0 + tau) % nt
        sign = torch.where(t0 + tau >= nt, -1.0, 1.0).to(torch.complex128)
        out += sign * per_t[t]
    return (out / len(t0s)).cpu().numpy()


def fit_energy(C: np.ndarray, delta: float, window: Tuple[float, float]) -> float:
    """E from a fit of log|C(tau)| = a - E tau over tau in [window] (physical
    units, tau = t delta), by least squares."""
    t = np.arange(len(C)) * delta
    sel = (t >= window[0] - 1e-12) & (t <= window[1] + 1e-12)
    y = np.log(np.abs(C[sel].real))
    A = np.vstack([np.ones(sel.sum()), t[sel]]).T
    coef, *_ = np.linalg.lstsq(A, y, rcond=None)
    return float(-coef[1])


def bootstrap_energy(Cs: np.ndarray, delta: float, window: Tuple[float, float], nboot: int = 200,
                     block: int = 1, seed: int = 0) -> Tuple[float, float]:
    """Energy of the mean correlator and its bootstrap error over configurations
    (resampled in blocks of `block` consecutive ones against autocorrelation)."""
    Cs = np.asarray(Cs)
    nb = len(Cs) // block
    blocks = Cs[: nb * block].reshape(nb, block, -1).mean(axis=1)
    E = fit_energy(blocks.mean(axis=0), delta, window)
    g = np.random.default_rng(seed)
    boots = [fit_energy(blocks[g.integers(0, nb, nb)].mean(axis=0), delta, window) for _ in range(nboot)]
    return E, float(np.std(boots, ddof=1))
