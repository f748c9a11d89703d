"""Exact diagonalisation pins (Section 8.1): on the 2x1 honeycomb torus at
U/kappa = 4 the quasi-particle energies equal the exact values the paper
prints, E_Gamma/kappa = 3.429 and E_M/kappa = 1.565; at U = 0 they are the
free band energies |f(k)| = 3 and 1. CPU only."""
import numpy as np

from oracle import ed, fermion
from oracle.lattice import Lattice


def test_exact_energies_of_the_4_site_model(paper):
    lat = Lattice(2, 1, 4, 1.0, paper["ed_U_over_kappa"], paper["ed_beta_kappa"])
    assert round(ed.quasiparticle_energy(lat, 0.0), 3) == paper["ed_E_Gamma_over_kappa"]
    assert round(ed.quasiparticle_energy(lat, np.pi), 3) == paper["ed_E_M_over_kappa"]


def test_free_limit_gives_band_energies():
    lat = Lattice(2, 1, 4, 1.0, 1e-300, 8.0)
    assert abs(ed.quasiparticle_energy(lat, 0.0) - 3.0) < 1e-12
    assert abs(ed.quasiparticle_energy(lat, np.pi) - 1.0) < 1e-12


def test_hopping_matrix_matches_the_operator_convention():
    """The ED hopping matrix is the spatial part of M (Eq. ferm_op) up to
    -delta kappa, with the same bond multiplicities."""
    lat = Lattice(2, 1, 4, 1.0, 4.0, 8.0)
    K = ed.hopping_matrix(lat)
    assert np.allclose(np.sort(np.linalg.eigvalsh(K)), [-3, -1, 1, 3])
    D = fermion.dense_M(lat, np.zeros(lat.N), 0.0)
    # time slice 0 block of the spatial hopping
    s, t, i, j = lat.coords()
    sl = np.where(t == 0)[0]
    hop = D[np.ix_(sl, sl)] + np.diag(np.where(s[sl] == 0, 1.0, -1.0))
    assert np.allclose(hop, -lat.delta * lat.kappa * K)
