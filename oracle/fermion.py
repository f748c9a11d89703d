"""The fermion operator M[phi; m_s] of Eq. ferm_op, its adjoint and M M^dagger.

Eq. ferm_op, per spatial site x and time slices t, t':
  M^AA_(x,t)(x,t') = -delta_tt' + (exp(+i phi_{x,t}) - delta m_s) delta_{t-1,t'}
  M^BB_(x,t)(x,t') = +delta_tt' - (exp(-i phi_{x,t}) - delta m_s) delta_{t+1,t'}
  M^AB = M^BA      = -delta kappa   for nearest neighbours at equal time.
Readings taken: the phase of a B row uses phi at the row's own time t (the
formula read literally); the time boundary is anti-periodic (lattice.py).

Everything here acts on complex128 vectors in the canonical layout of
lattice.py. The stencil functions use index tables; `dense_M` builds the matrix
entry by entry from the same equation, as an independent restatement.
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp

from .lattice import A, B, Lattice


def time_hop(lat: Lattice, phi: np.ndarray, ms: float) -> np.ndarray:
    """The time-hopping entry of M in every row (x, t), boundary sign included:
    A rows: +s (e^{+i phi_{x,t}} - delta m_s), B rows: -s (e^{-i phi_{x,t}} - delta m_s). Eq. ferm_op."""
    s, _, _, _ = lat.coords()
    _, sign = lat.time_partner()
    dm = lat.delta * ms
    hopA = np.exp(1j * phi) - dm
    hopB = -(np.exp(-1j * phi) - dm)
    return sign * np.where(s == A, hopA, hopB)


def diagonal(lat: Lattice) -> np.ndarray:
    """The time-diagonal entry: -1 on A rows, +1 on B rows (Eq. ferm_op)."""
    s, _, _, _ = lat.coords()
    return np.where(s == A, -1.0, 1.0)


def apply_M(lat: Lattice, phi: np.ndarray, ms: float, psi: np.ndarray) -> np.ndarray:
    """(M psi)(x,t) = d(x) psi(x,t) + hop(x,t) psi(time partner) - delta kappa sum_nb psi. Eq. ferm_op."""
    tp, _ = lat.time_partner()
    nb = lat.spatial_neighbours()
    hop = time_hop(lat, phi, ms)
    out = diagonal(lat) * psi + hop * np.take(psi, tp)
    out = out - lat.delta * lat.kappa * np.take(psi, nb).sum(axis=1)
    return out


def apply_Mdag(lat: Lattice, phi: np.ndarray, ms: float, psi: np.ndarray) -> np.ndarray:
    """(M^dagger psi)(y) = sum_x conj(M_xy) psi(x): the time entry of row x sits in
    column tp(x); its conjugate moves psi(x) to y = tp(x). The hopping part is
    real and symmetric, the diagonal real. Eq. ferm_op."""
    tp, _ = lat.time_partner()
    nb = lat.spatial_neighbours()
    hop = time_hop(lat, phi, ms)
    out = diagonal(lat) * psi
    timepart = np.zeros_like(psi)
    np.add.at(timepart, tp, np.conj(hop) * psi)
    out = out + timepart - lat.delta * lat.kappa * np.take(psi, nb).sum(axis=1)
    return out


def apply_MMdag(lat: Lattice, phi, ms, psi, sigma: float = 0.0):
    """A psi = M_{m_s} M_{m_s}^dagger psi + sigma psi (Eq. hamiltonian; the shifted
    form of the Hasenbusch splitting in Section 5.1)."""
    return apply_M(lat, phi, ms, apply_Mdag(lat, phi, ms, psi)) + sigma * psi


def dense_M(lat: Lattice, phi: np.ndarray, ms: float) -> np.ndarray:
    """M as an explicit N x N matrix, written entry by entry from Eq. ferm_op
    with loops over sites (tiny lattices only)."""
    n, m, nt = lat.n, lat.m, lat.nt
    dk = lat.delta * lat.kappa
    dm = lat.delta * ms
    Mx = np.zeros((lat.N, lat.N), dtype=np.complex128)
    idx = lat.index
    for j in range(m):
        for i in range(n):
            for t in range(nt):
                a = idx(A, t, i, j)
                b = idx(B, t, i, j)
                # AA block: -1 on the diagonal, (e^{i phi_{x,t}} - dm) to (x, t-1)
                Mx[a, a] += -1.0
                tm = t - 1
                sgn = 1.0
                if tm < 0:
                    tm += nt
                    sgn = -1.0
                Mx[a, idx(A, tm, i, j)] += sgn * (np.exp(1j * phi[a]) - dm)
                # BB block: +1 on the diagonal, -(e^{-i phi_{x,t}} - dm) to (x, t+1)
                Mx[b, b] += 1.0
                tq = t + 1
                sgn = 1.0
                if tq >= nt:
                    tq -= nt
                    sgn = -1.0
                Mx[b, idx(B, tq, i, j)] += -sgn * (np.exp(-1j * phi[b]) - dm)
                # AB / BA: -delta kappa per bond; each bond listed once from A
                for (bi, bj) in ((i, j), ((i - 1) % n, j), (i, (j - 1) % m)):
                    bb = idx(B, t, bi, bj)
                    Mx[a, bb] += -dk
                    Mx[bb, a] += -dk
    return Mx


def sparse_M(lat: Lattice, phi: np.ndarray, ms: float) -> sp.csc_matrix:
    """M as a scipy sparse matrix: per row the diagonal entry, the time-hopping
    entry at its time partner, and -delta kappa at each of the three hopping
    partners (duplicates summed, as for n or m below 3). Eq. ferm_op."""
    rows = np.arange(lat.N)
    tp, _ = lat.time_partner()
    nb = lat.spatial_neighbours()
    r = np.concatenate([rows, rows, np.repeat(rows, 3)])
    c = np.concatenate([rows, tp, nb.ravel()])
    v = np.concatenate([diagonal(lat).astype(np.complex128), time_hop(lat, phi, ms),
                        np.full(3 * lat.N, -lat.delta * lat.kappa, dtype=np.complex128)])
    return sp.csc_matrix((v, (r, c)), shape=(lat.N, lat.N))


def free_spectrum(lat: Lattice, ms: float, theta: float = 0.0) -> np.ndarray:
    """Closed-form eigenvalues of M M^dagger for the constant field phi = theta.

    With phi constant, M is diagonalised by plane waves e^{i(k.R + omega t)},
    omega = (2l+1) pi / nt (anti-periodic), k = (2 pi j1/n, 2 pi j2/m). Each
    (k, omega) block is [[a, -dk f], [-dk f*, -conj(a)]] with
    a = -1 + (e^{i theta} - delta m_s) e^{-i omega} and
    |f|^2 = 3 + 2 cos k1 + 2 cos k2 + 2 cos(k1 - k2), so M M^dagger is
    |a|^2 + (delta kappa)^2 |f|^2 times the 2x2 identity in every block.
    Returns the N eigenvalues, sorted. Eq. ferm_op."""
    nt = lat.nt
    omega = (2 * np.arange(nt) + 1) * np.pi / nt
    k1 = 2 * np.pi * np.arange(lat.n) / lat.n
    k2 = 2 * np.pi * np.arange(lat.m) / lat.m
    K1, K2 = np.meshgrid(k1, k2, indexing="ij")
    f2 = 3 + 2 * np.cos(K1) + 2 * np.cos(K2) + 2 * np.cos(K1 - K2)
    z = np.exp(1j * theta) - lat.delta * ms
    a2 = np.abs(-1.0 + z * np.exp(-1j * omega)) ** 2
    lam = a2[:, None] + (lat.delta * lat.kappa) ** 2 * f2.ravel()[None, :]
    return np.sort(np.concatenate([lam.ravel(), lam.ravel()]))
