"""Correlator helpers (Section 8.1) on the free field, with the oracle's dense
propagator: the band projection of M^{-1} falls as a single exponential whose
fitted energy approaches the free band energy |f(k)| (3 at Gamma, 1 at M on the
2x1 torus) as delta -> 0. CPU only."""
import numpy as np
import pytest

from oracle import fermion
from oracle.lattice import Lattice
from paper_1804_07195_gb300 import correlators as cr


def free_correlator(lat, k1):
    G = np.linalg.inv(fermion.dense_M(lat, np.zeros(lat.N), 0.0))
    o = cr.band_orbital(lat.n, lat.m, k1)
    C = np.zeros(lat.nt, complex)
    for t0 in range(lat.nt):
        src = cr.slice_indices(lat.n, lat.m, lat.nt, t0)
        col = G[:, src] @ o
        for tau in range(lat.nt):
            t = (t0 + tau) % lat.nt
            sign = -1.0 if t0 + tau >= lat.nt else 1.0
            C[tau] += sign * np.vdot(o, col[cr.slice_indices(lat.n, lat.m, lat.nt, t)])
    return C / lat.nt


@pytest.mark.parametrize("k1,E", [(0.0, 3.0), (np.pi, 1.0)])
def test_free_band_energies(paper, k1, E):
    win = paper["fit_windows"]["Gamma" if k1 == 0.0 else "M"]
    errs = []
    for nt in (32, 64):
        lat = Lattice(2, 1, nt, 1.0, 4.0, 8.0)
        C = free_correlator(lat, k1)
        errs.append(abs(cr.fit_energy(C, lat.delta, win) - E))
    assert errs[1] < 0.02
    assert errs[1] < 0.5 * errs[0]   # discretisation error shrinks with delta


def test_bootstrap_of_identical_samples_has_no_spread():
    lat = Lattice(2, 1, 32, 1.0, 4.0, 8.0)
    C = free_correlator(lat, 0.0)
    E, dE = cr.bootstrap_energy(np.array([C] * 10), lat.delta, (0.2, 1.0), nboot=20)
    assert dE < 1e-12 and abs(E - cr.fit_energy(C, lat.delta, (0.2, 1.0))) < 1e-12


class DenseOracleContext:
    """Stands in for a Context on the CPU: load_field, solve_cg and apply_Mdag
    done with the oracle's dense M (only what correlator() calls)."""

    def __init__(self, lat):
        self.lat = lat
        self.phi = None

    def load_field(self, phi):
        self.phi = phi.numpy().copy()

    def solve_cg(self, phi, ms, b, tol):
        import torch
        D = fermion.dense_M(self.lat, self.phi, ms)
        return torch.tensor(np.linalg.solve(D @ D.conj().T, b.numpy())), {}

    def apply_Mdag(self, phi, ms, x):
        import torch
        return torch.tensor(fermion.apply_Mdag(self.lat, self.phi, ms, x.numpy()))


@pytest.mark.parametrize("k1,t0s", [(0.0, [0, 3]), (np.pi, [1, 5, 6]), (None, [2, 7])])
def test_correlator_assembly_on_a_random_field(k1, t0s):
    """correlator() against a plain loop over the dense propagator M^{-1} on a
    random field: the source sits on slice t0, every sink slice is projected on
    the orbital, the sign flips where t0 + tau wraps, and the sources are
    averaged."""
    torch = pytest.importorskip("torch")
    import workloads as W
    w = W.small(2, 1, 8, seed=81, U=4.0, beta=8.0)
    lat = Lattice.from_params(w.lat)
    G = np.linalg.inv(fermion.dense_M(lat, w.phi, 0.0))
    if k1 is None:  # any complex source vector on a slice (the band orbitals here are real)
        g = np.random.default_rng(7)
        o = g.normal(size=2 * lat.V) + 1j * g.normal(size=2 * lat.V)
    else:
        o = cr.band_orbital(lat.n, lat.m, k1)
    ref = np.zeros(lat.nt, complex)
    for t0 in t0s:
        col = G[:, cr.slice_indices(lat.n, lat.m, lat.nt, t0)] @ o
        for tau in range(lat.nt):
            t = (t0 + tau) % lat.nt
            sign = -1.0 if t0 + tau >= lat.nt else 1.0
            ref[tau] += sign * np.vdot(o, col[cr.slice_indices(lat.n, lat.m, lat.nt, t)])
    ref /= len(t0s)
    got = cr.correlator(DenseOracleContext(lat), w.lat, torch.tensor(w.phi), o, t0s)
    assert np.abs(got - ref).max() <= 1e-12 * np.abs(ref).max()
