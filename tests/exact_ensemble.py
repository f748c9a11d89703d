"""Exact expectation of phi.phi under the HMC weight exp(-phi^2/(2 delta U))
det(M M^dagger) (Section 2) on a tiny lattice, by importance sampling from the
Gaussian term and reweighting with the determinant from the oracle's dense M
(Eq. ferm_op). Used by the CPU and the GPU ensemble tests."""
import numpy as np

from oracle import fermion


def phi2_exact(lat, g, ns=200000):
    """(<phi.phi>, its importance-sampling error by the delta method)."""
    ph = g.normal(0.0, np.sqrt(lat.delta * lat.U), size=(ns, lat.N))
    M0 = fermion.dense_M(lat, np.zeros(lat.N), 0.0)
    tp, sign = lat.time_partner()
    rows = np.arange(lat.N)
    s, _, _, _ = lat.coords()
    Ms = np.repeat(M0[None], ns, axis=0)
    Ms[:, rows, tp] = sign * np.where(s == 0, np.exp(1j * ph), -np.exp(-1j * ph))
    # the phase entries written here are the oracle's own time hop
    hops = np.stack([fermion.time_hop(lat, p, 0.0) for p in ph[:2000]])
    assert np.allclose(Ms[:2000, rows, tp], hops)
    _, ld = np.linalg.slogdet(Ms)
    wts = np.exp(2 * ld - (2 * ld).max())
    obs = (ph * ph).sum(axis=1)
    exact = (wts * obs).sum() / wts.sum()
    wn = wts / wts.sum()
    return exact, np.sqrt(((wn * (obs - exact)) ** 2).sum())


def blocked(x, size=50):
    """Mean and standard error of x from blocks of `size` consecutive values."""
    x = np.asarray(x)
    b = x[: len(x) // size * size].reshape(-1, size).mean(axis=1)
    return b.mean(), b.std(ddof=1) / np.sqrt(len(b))
