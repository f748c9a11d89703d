"""Pins of the oracle's fermion operator (Eq. ferm_op) against closed forms,
library routines and invariants. CPU only."""
import numpy as np
import pytest

import workloads as W
from oracle import action, fermion
from oracle.lattice import A, B, Lattice

SHAPES = [(2, 1, 4), (1, 3, 6), (3, 3, 8), (4, 5, 6), (6, 6, 16)]


def lat_of(n, m, nt, U=2.0, beta=4.0):
    return Lattice(n, m, nt, 1.0, U, beta)


@pytest.mark.parametrize("shape", SHAPES)
@pytest.mark.parametrize("ms", [0.0, 0.37])
def test_stencil_equals_dense_matrix(shape, ms):
    w = W.small(*shape, seed=11)
    lat = Lattice.from_params(w.lat)
    D = fermion.dense_M(lat, w.phi, ms)
    x = w.b
    ref = np.abs(D @ x).max()
    assert np.abs(D @ x - fermion.apply_M(lat, w.phi, ms, x)).max() <= 1e-14 * ref
    # the adjoint stencil is the conjugate transpose of the dense matrix
    assert np.abs(D.conj().T @ x - fermion.apply_Mdag(lat, w.phi, ms, x)).max() <= 1e-14 * ref
    AA = D @ D.conj().T + 0.25 * np.eye(lat.N)
    assert np.abs(AA @ x - fermion.apply_MMdag(lat, w.phi, ms, x, 0.25)).max() <= 1e-13 * ref


@pytest.mark.parametrize("shape", SHAPES)
def test_sparse_matrix_equals_dense_matrix(shape):
    w = W.small(*shape, seed=12)
    lat = Lattice.from_params(w.lat)
    for ms in (0.0, 0.6):
        assert np.abs(fermion.sparse_M(lat, w.phi, ms).toarray() - fermion.dense_M(lat, w.phi, ms)).max() < 1e-15


def test_sparse_lu_solve_matches_dense_lu():
    w = W.small(4, 5, 6, seed=13)
    lat = Lattice.from_params(w.lat)
    x1 = action.SolveA(lat, "splu")(w.phi, 0.3, w.b)
    x2 = action.SolveA(lat, "dense")(w.phi, 0.3, w.b)
    assert np.linalg.norm(x1 - x2) < 1e-11 * np.linalg.norm(x2)


@pytest.mark.parametrize("shape", SHAPES[:4])
def test_every_site_has_three_bonds(shape):
    lat = lat_of(*shape)
    D = fermion.dense_M(lat, np.zeros(lat.N), 0.0)
    s, _, _, _ = lat.coords()
    hop = D.copy()
    idx = np.arange(lat.N)
    tp, _ = lat.time_partner()
    hop[idx, idx] = 0
    hop[idx, tp] = 0
    # rows: the spatial hopping sums to -3 delta kappa, entries only across sublattices
    assert np.allclose(hop.sum(axis=1), -3 * lat.delta * lat.kappa)
    assert np.all(hop[np.ix_(s == A, s == A)] == 0) and np.all(hop[np.ix_(s == B, s == B)] == 0)
    assert np.allclose(hop, hop.T)


@pytest.mark.parametrize("shape", [(3, 3, 8), (2, 1, 4), (4, 2, 6), (1, 1, 5)])
@pytest.mark.parametrize("theta", [0.0, 0.7, -2.1])
@pytest.mark.parametrize("ms", [0.0, 0.5])
def test_free_field_spectrum_closed_form(shape, theta, ms):
    """phi = theta constant: spectrum of M M^dagger from plane waves (anti-periodic
    Matsubara frequencies, |f(k)|^2 of the honeycomb, time hop z = e^{i theta} - delta m_s)."""
    lat = lat_of(*shape)
    D = fermion.dense_M(lat, np.full(lat.N, theta), ms)
    ev = np.linalg.eigvalsh(D @ D.conj().T)
    assert np.allclose(np.sort(ev), fermion.free_spectrum(lat, ms, theta), atol=1e-12, rtol=0)


@pytest.mark.parametrize("L,nt", [(3, 4), (6, 8), (3, 16)])
def test_lowest_mode_antiperiodic(L, nt):
    """m_s = 0, phi = 0, 3 | L: a Dirac point exists, and the lowest eigenvalue is
    |1 - e^{-i pi/nt}|^2 = 4 sin^2(pi/(2 nt)); a periodic time boundary would give 0."""
    lat = lat_of(L, L, nt)
    D = fermion.dense_M(lat, np.zeros(lat.N), 0.0)
    ev = np.linalg.eigvalsh(D @ D.conj().T)
    assert abs(ev.min() - 4 * np.sin(np.pi / (2 * nt)) ** 2) < 1e-12
    # largest: (1 + z)^2 + 9 (delta kappa)^2 at omega = pi, k = 0, here z = 1
    dk = lat.delta * lat.kappa
    assert ev.max() <= 4 * np.cos(np.pi / (2 * nt)) ** 2 + 9 * dk * dk + 1e-12
    assert abs(ev.max() - (4 * np.cos(np.pi / (2 * nt)) ** 2 + 9 * dk * dk)) < 1e-12


@pytest.mark.parametrize("shape", [(2, 1, 4), (3, 2, 6)])
def test_time_gauge_invariance(shape):
    """At m_s = 0, the unitary D = diag(e^{i beta_t}) maps M[phi] to M[phi'] with
    phi'_A(x,t) = phi_A(x,t) + beta_t - beta_{t-1}, phi'_B(x,t) = phi_B(x,t) + beta_{t+1} - beta_t
    (time indices mod nt). The spectrum of M M^dagger must not change. This fixes
    which time slice's phi sits on which time link, for both sublattices."""
    w = W.small(*shape, seed=5)
    lat = Lattice.from_params(w.lat)
    g = np.random.default_rng(3)
    beta = g.uniform(-np.pi, np.pi, lat.nt)
    s, t, _, _ = lat.coords()
    shift = np.where(s == A, beta[t] - beta[(t - 1) % lat.nt], beta[(t + 1) % lat.nt] - beta[t])
    D0 = fermion.dense_M(lat, w.phi, 0.0)
    D1 = fermion.dense_M(lat, w.phi + shift, 0.0)
    e0 = np.linalg.eigvalsh(D0 @ D0.conj().T)
    e1 = np.linalg.eigvalsh(D1 @ D1.conj().T)
    assert np.allclose(e0, e1, atol=1e-12)
    # and a shift that puts B's phase on the other link does change it
    wrong = np.where(s == A, shift, beta[t] - beta[(t - 1) % lat.nt])
    D2 = fermion.dense_M(lat, w.phi + wrong, 0.0)
    e2 = np.linalg.eigvalsh(D2 @ D2.conj().T)
    assert not np.allclose(e0, e2, atol=1e-6)


def test_logdet_free_field_closed_form():
    lat = lat_of(3, 3, 8)
    for ms in (0.0, 0.8):
        ld = action.logdet_MMdag(lat, np.full(lat.N, 0.3), ms)
        assert abs(ld - np.log(fermion.free_spectrum(lat, ms, 0.3)).sum()) < 1e-10
