"""Exact application and inversion of A = M M^dagger + sigma for a constant
field phi = theta, by Fourier transform (Eq. ferm_op, Section 2).

For constant phi the operator is translation invariant in space and, with the
anti-periodic time boundary, diagonalised by the plane waves
e^{i(omega t + k1 i + k2 j)} with omega_l = (2l + 1) pi / nt and
k1 = 2 pi j1 / n, k2 = 2 pi j2 / m. In each (k, omega) block M is
[[a, -dk f], [-dk conj(f), -conj(a)]] with a = -1 + z e^{-i omega},
z = e^{i theta} - delta m_s, dk = delta kappa and |f|^2 = 3 + 2 cos k1 +
2 cos k2 + 2 cos(k1 - k2); its M M^dagger is (|a|^2 + dk^2 |f|^2) times the 2x2
identity. So A acts on each sublattice's component alone, as multiplication by
lambda(k, omega) = |a|^2 + dk^2 |f|^2 + sigma of its Fourier coefficients.

This restates the operator through its spectrum with numpy's FFT as the only
library step; it shares nothing with the stencil in fermion.py, which it pins at
sizes where no dense matrix fits.
"""
from __future__ import annotations

import numpy as np

from .lattice import Lattice


def mode_eigenvalues(lat: Lattice, ms: float, sigma: float = 0.0, theta: float = 0.0) -> np.ndarray:
    """lambda(omega_l, k1, k2) on the grid (nt, m, n) in numpy FFT order along
    each axis: index l along time is omega_l = (2l + 1) pi / nt, index j2 along
    the second cell axis is k2 = 2 pi j2 / m, index j1 along the first is
    k1 = 2 pi j1 / n. Eq. ferm_op in plane waves."""
    omega = (2 * np.arange(lat.nt) + 1) * np.pi / lat.nt
    k2 = 2 * np.pi * np.arange(lat.m) / lat.m
    k1 = 2 * np.pi * np.arange(lat.n) / lat.n
    z = np.exp(1j * theta) - lat.delta * ms
    a2 = np.abs(-1.0 + z * np.exp(-1j * omega)) ** 2
    K2, K1 = np.meshgrid(k2, k1, indexing="ij")
    f2 = 3 + 2 * np.cos(K1) + 2 * np.cos(K2) + 2 * np.cos(K1 - K2)
    dk = lat.delta * lat.kappa
    return a2[:, None, None] + dk * dk * f2[None, :, :] + sigma


def _multiply(lat: Lattice, v: np.ndarray, factor: np.ndarray) -> np.ndarray:
    """Multiply the Fourier coefficients of each sublattice component of v by
    `factor`. The anti-periodic frequencies are (2l + 1) pi / nt: removing the
    half-step twist e^{i pi t / nt} leaves a periodic function of t, which the
    ordinary FFT expands in e^{2 pi i l t / nt}."""
    x = np.asarray(v, dtype=np.complex128).reshape(2, lat.nt, lat.m, lat.n)
    twist = np.exp(1j * np.pi * np.arange(lat.nt) / lat.nt)[None, :, None, None]
    c = np.fft.fftn(x / twist, axes=(1, 2, 3))
    return (np.fft.ifftn(c * factor[None], axes=(1, 2, 3)) * twist).reshape(-1)


def apply_A(lat: Lattice, ms: float, sigma: float, v: np.ndarray, theta: float = 0.0) -> np.ndarray:
    """(M M^dagger + sigma) v for phi = theta everywhere. Eq. ferm_op in plane waves."""
    return _multiply(lat, v, mode_eigenvalues(lat, ms, sigma, theta))


def solve_A(lat: Lattice, ms: float, sigma: float, b: np.ndarray, theta: float = 0.0) -> np.ndarray:
    """(M M^dagger + sigma)^{-1} b for phi = theta everywhere. Eq. ferm_op in plane waves."""
    return _multiply(lat, b, 1.0 / mode_eigenvalues(lat, ms, sigma, theta))


def condition_number(lat: Lattice, ms: float, sigma: float = 0.0, theta: float = 0.0) -> float:
    """lambda_max / lambda_min of A: the factor by which a relative residual
    can grow into the relative error of a solution. Eq. ferm_op in plane waves."""
    lam = mode_eigenvalues(lat, ms, sigma, theta)
    return float(lam.max() / lam.min())
