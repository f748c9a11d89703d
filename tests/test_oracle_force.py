"""Pins of the oracle's action and force (Eqs. hamiltonian, p_dot, eta_xi,
f_chi_i, def_xi_i) against finite differences, library log-determinants and
the identities of the Hasenbusch splitting. CPU only."""
import numpy as np
import pytest

import workloads as W
from oracle import action, fermion
from oracle.lattice import Lattice


def setup(shape=(3, 2, 6), seed=21, masses=()):
    w = W.small(*shape, seed=seed, masses=masses)
    lat = Lattice.from_params(w.lat)
    return w, lat, action.SolveA(lat, "dense")


def central_dir(f, x, d, h=1e-5):
    return (f(x + h * d) - f(x - h * d)) / (2 * h)


@pytest.mark.parametrize("ms", [0.0, 0.6])
def test_logdet_gradient_vs_finite_differences(ms):
    w, lat, _ = setup()
    g = action.grad_logdet_MMdag(lat, w.phi, ms)
    f = lambda p: action.logdet_MMdag(lat, p, ms)
    rng = np.random.default_rng(0)
    for _ in range(3):
        d = rng.normal(size=lat.N)
        d /= np.linalg.norm(d)
        assert abs(central_dir(f, w.phi, d) - g @ d) < 1e-7 * max(1.0, np.abs(g).sum())
    for k in (0, lat.N // 2 - 1, lat.N // 2, lat.N - 1):   # A at t=0 and B at nt-1 wrap
        e = np.zeros(lat.N)
        e[k] = 1.0
        assert abs(central_dir(f, w.phi, e) - g[k]) < 1e-7


@pytest.mark.parametrize("ms", [0.0, 0.4])
def test_pseudofermion_force_vs_finite_differences(ms):
    w, lat, solve = setup()
    chi = w.b
    g = action.grad_pf_action(lat, w.phi, ms, chi, solve)
    f = lambda p: action.pf_action(lat, p, ms, chi, solve)
    rng = np.random.default_rng(1)
    for _ in range(3):
        d = rng.normal(size=lat.N)
        d /= np.linalg.norm(d)
        fd = central_dir(f, w.phi, d)
        assert abs(fd - g @ d) <= 1e-6 * max(1.0, abs(fd))


def test_stochastic_identity_mean_force_is_logdet_gradient():
    """chi = M rho with rho ~ exp(-rho^dagger rho) samples exp(-S)/det(M M^dagger), so
    E[dS/dphi] = -d log det(M M^dagger)/dphi."""
    w, lat, solve = setup(shape=(2, 1, 4), seed=4)
    rng = np.random.default_rng(9)
    ns = 4000
    acc = np.zeros((ns, lat.N))
    D = fermion.dense_M(lat, w.phi, 0.0)
    AA = D @ D.conj().T
    Ainv = np.linalg.inv(AA)
    for k in range(ns):
        rho = (rng.normal(size=lat.N) + 1j * rng.normal(size=lat.N)) * np.sqrt(0.5)
        chi = D @ rho
        eta = Ainv @ chi
        xi = D.conj().T @ eta
        acc[k] = action.force_kernel(lat, w.phi, eta, xi)
    mean = acc.mean(axis=0)
    err = acc.std(axis=0) / np.sqrt(ns)
    ref = -action.grad_logdet_MMdag(lat, w.phi, 0.0)
    assert np.all(np.abs(mean - ref) < 5 * err + 1e-12)


def test_hasenbusch_start_action_equals_rho_norm():
    """S_i(phi_start) = rho_i^dagger rho_i exactly, by construction of chi_i (Section 5.1)."""
    masses = (0.3, 1.0)
    w, lat, solve = setup(masses=masses)
    chis = action.make_chi(lat, w.phi, masses, w.rho, solve)
    for i in range(len(masses) + 1):
        S = action.term_action(lat, w.phi, masses, chis, i, solve)
        rr = float(np.real(np.vdot(w.rho[i], w.rho[i])))
        assert abs(S - rr) < 1e-11 * rr


def test_hasenbusch_equal_masses_give_zero_force():
    """mu_i = mu_{i-1} gives xi_i = chi_i and F_{chi_i} = 0 (Section 5.1)."""
    masses = (0.5, 0.5)
    w, lat, solve = setup(masses=masses)
    chis = action.make_chi(lat, w.phi, masses, w.rho, solve)
    phi1 = w.phi + 0.1 * np.random.default_rng(2).normal(size=lat.N)
    g1 = action.term_grad(lat, phi1, masses, chis, 1, solve)
    assert np.abs(g1).max() < 1e-12
    assert np.abs(action.term_grad(lat, phi1, masses, chis, 0, solve)).max() > 1e-3


def test_hasenbusch_force_is_linear_in_the_mass_gap():
    """For nearly equal neighbouring masses the term's force grows in
    proportion to mu_1 - mu_0 (Section 7.2: the small force of the Hasenbusch
    tuner): doubling a small gap doubles the force, to first order."""
    w, lat, solve = setup(masses=(0.4, 0.4))
    phi1 = w.phi + 0.1 * np.random.default_rng(2).normal(size=lat.N)

    def force(eps):
        masses = (0.4, 0.4 + eps)
        chis = action.make_chi(lat, w.phi, masses, w.rho, solve)
        return action.term_grad(lat, phi1, masses, chis, 1, solve)

    f1, f2 = force(1e-3), force(2e-3)
    assert np.linalg.norm(f1) > 1e-6
    assert abs(np.linalg.norm(f2) / np.linalg.norm(f1) - 2.0) < 1e-2
    assert np.linalg.norm(f2 - 2 * f1) < 1e-2 * np.linalg.norm(f2)


@pytest.mark.parametrize("i", [0, 1, 2])
def test_hasenbusch_term_force_vs_finite_differences(i):
    masses = (0.3, 1.0)
    w, lat, solve = setup(masses=masses)
    chis = action.make_chi(lat, w.phi, masses, w.rho, solve)
    phi1 = w.phi + 0.05 * np.random.default_rng(7).normal(size=lat.N)  # away from the start point
    g = action.term_grad(lat, phi1, masses, chis, i, solve)
    f = lambda p: action.term_action(lat, p, masses, chis, i, solve)
    rng = np.random.default_rng(i)
    for _ in range(2):
        d = rng.normal(size=lat.N)
        d /= np.linalg.norm(d)
        fd = central_dir(f, phi1, d)
        assert abs(fd - g @ d) <= 2e-6 * max(1.0, abs(fd))


def test_hasenbusch_determinant_telescopes():
    """The terms' operators multiply to M M^dagger: sum over terms of
    log det(M_{mu_{i-1}} M_{mu_{i-1}}^dagger) - log det(M_{mu_i} M_{mu_i}^dagger), plus the top
    log det(M_{mu_{n-1}} M_{mu_{n-1}}^dagger), equals log det(M M^dagger) (Section 5.1)."""
    masses = (0.2, 0.7, 1.5)
    w, lat, _ = setup(masses=masses)
    ld = lambda ms: action.logdet_MMdag(lat, w.phi, ms)
    total = ld(masses[-1]) + sum(ld(action.lower_mass(masses, i)) - ld(masses[i])
                                  for i in range(len(masses)))
    assert abs(total - ld(0.0)) < 1e-9
