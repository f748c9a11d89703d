"""Pins of the free-field closed form (constant phi, Eq. ferm_op diagonalised
by plane waves) against the explicit dense matrix and LU, and, through it, of
the oracle's stencil and CG at sizes where no dense matrix fits. CPU only."""
import numpy as np
import pytest

from oracle import fermion, free_field, solvers
from oracle.lattice import Lattice

SMALL = [(2, 1, 4), (1, 1, 5), (4, 2, 6), (3, 5, 4), (3, 3, 8)]


def lat_of(n, m, nt, U=2.0, beta=4.0):
    return Lattice(n, m, nt, 1.0, U, beta)


def rand_vec(N, seed):
    g = np.random.default_rng(seed)
    return (g.normal(size=N) + 1j * g.normal(size=N)) * np.sqrt(0.5)


@pytest.mark.parametrize("shape", SMALL)
@pytest.mark.parametrize("theta,ms,sigma", [(0.0, 0.0, 0.0), (0.7, 0.5, 0.0), (-2.1, 0.0, 0.3)])
def test_closed_form_equals_dense_matrix(shape, theta, ms, sigma):
    """The FFT application and inverse equal the dense M M^dagger + sigma built
    entry by entry, and its solution by LU, for lattices with n != m, a single
    cell, odd and even nt, and a complex time hop (theta != 0)."""
    lat = lat_of(*shape)
    D = fermion.dense_M(lat, np.full(lat.N, theta), ms)
    Amat = D @ D.conj().T + sigma * np.eye(lat.N)
    v = rand_vec(lat.N, sum(shape))
    assert np.abs(free_field.apply_A(lat, ms, sigma, v, theta) - Amat @ v).max() <= 1e-13 * np.abs(Amat @ v).max()
    x = np.linalg.solve(Amat, v)
    assert np.abs(free_field.solve_A(lat, ms, sigma, v, theta) - x).max() <= 1e-12 * np.abs(x).max()
    # the mode eigenvalues, each twice, are the spectrum
    lam = free_field.mode_eigenvalues(lat, ms, sigma, theta).ravel()
    assert np.allclose(np.sort(np.concatenate([lam, lam])), np.linalg.eigvalsh(Amat), atol=1e-12, rtol=0)


def test_a_mode_is_an_eigenvector():
    """A single plane wave e^{i(omega_l t + k1 i + k2 j)} on sublattice A alone
    is mapped to lambda times itself by the dense matrix (the block is a
    multiple of the identity, so no B component appears)."""
    lat = lat_of(3, 2, 6)
    theta, ms = 0.4, 0.3
    D = fermion.dense_M(lat, np.full(lat.N, theta), ms)
    Amat = D @ D.conj().T
    s, t, i, j = lat.coords()
    l, j1, j2 = 2, 1, 1
    omega = (2 * l + 1) * np.pi / lat.nt
    wave = np.where(s == 0, np.exp(1j * (omega * t + 2 * np.pi * j1 * i / lat.n + 2 * np.pi * j2 * j / lat.m)), 0)
    lam = free_field.mode_eigenvalues(lat, ms, 0.0, theta)[l, j2, j1]
    assert np.abs(Amat @ wave - lam * wave).max() <= 1e-13


def test_condition_number_at_a_dirac_point():
    """m_s = 0, phi = 0, 3 | n, m: lambda_min = 4 sin^2(pi / 2 nt) (the Dirac
    point at the lowest Matsubara frequency), lambda_max = 4 cos^2(pi / 2 nt)
    + 9 (delta kappa)^2."""
    lat = lat_of(6, 6, 16)
    dk = lat.delta * lat.kappa
    lmin = 4 * np.sin(np.pi / 32) ** 2
    lmax = 4 * np.cos(np.pi / 32) ** 2 + 9 * dk * dk
    assert abs(free_field.condition_number(lat, 0.0) - lmax / lmin) <= 1e-9 * lmax / lmin


@pytest.mark.parametrize("theta,ms,sigma", [(0.0, 0.0, 0.0), (0.3, 0.5, 0.05)])
def test_stencil_at_36x36x64_equals_closed_form(theta, ms, sigma):
    """The oracle's stencil M M^dagger + sigma on 36x36, nt = 64 (165,888 sites)
    against the closed form, element by element."""
    lat = Lattice(36, 36, 64, 1.0, 3.5, 8.0)
    v = rand_vec(lat.N, 36)
    ref = free_field.apply_A(lat, ms, sigma, v, theta)
    got = fermion.apply_MMdag(lat, np.full(lat.N, theta), ms, v, sigma)
    assert np.abs(got - ref).max() <= 1e-13 * np.abs(ref).max()


def test_cg_at_36x36x64_reaches_the_exact_solution():
    """The oracle's FP64 CG at true residual 1e-10 is within kappa * 1e-10 of
    the closed-form solution (the relative error is at most the condition
    number times the relative residual)."""
    lat = Lattice(36, 36, 64, 1.0, 3.5, 8.0)
    theta, ms, sigma = 0.3, 0.5, 0.05
    b = rand_vec(lat.N, 37)
    phi = np.full(lat.N, theta)
    res = solvers.cg(lambda v: fermion.apply_MMdag(lat, phi, ms, v, sigma), b, tol=1e-10)
    x = free_field.solve_A(lat, ms, sigma, b, theta)
    kappa = free_field.condition_number(lat, ms, sigma, theta)
    rel_res = np.linalg.norm(free_field.apply_A(lat, ms, sigma, res.x, theta) - b) / np.linalg.norm(b)
    assert res.converged and rel_res <= 1.01e-10
    assert np.linalg.norm(res.x - x) / np.linalg.norm(x) <= kappa * rel_res


def test_spectral_edge_at_the_papers_setting(paper):
    """At the setting of the paper's solver-time fit (N_t = 256, beta kappa = 8,
    m_s = 0) the free-field upper edge 4 cos^2(pi / 2 nt) + 9 (delta kappa)^2
    (omega nearest pi, k = 0, the same on any torus) lies inside the fitted
    lambda_max = 4.1 +- 0.2 of Section 6.1. The fit was made on interacting
    configurations of a nanotube, so this is a consistency check of the
    operator's scale, not a sharp pin."""
    lat = Lattice(3, 3, 256, 1.0, 3.5, 8.0)
    lam = free_field.mode_eigenvalues(lat, 0.0)
    dk = lat.delta * lat.kappa
    edge = 4 * np.cos(np.pi / 512) ** 2 + 9 * dk * dk
    assert abs(lam.max() - edge) < 1e-12
    assert abs(edge - paper["solver_time_fit"]["lambda_max"]) <= 0.2
