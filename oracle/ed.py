"""Exact diagonalisation of the Hubbard model on a small honeycomb torus
(Section 8.1, the 4-site benchmark).

Hamiltonian (the model whose path integral Eq. hamiltonian represents, in
spin-1/2 language, at half filling):
    H = -kappa sum_{<x,y>, s} (c^dag_{x s} c_{y s} + h.c.) + (U/2) sum_x (n_x - 1)^2,
with the hopping matrix of lattice.py (bonds that coincide on a small torus
count with multiplicity). Reading of Section 8.1's "4-site model ... (i.e.
hexagonal lattice)": the 2x1 honeycomb torus, whose free single-particle
energies are kappa |f(k)| = 3 kappa at Gamma and kappa at M; this reading
reproduces the exact energies the paper prints (3.429 and 1.565 at U = 4).

E_k is the energy of adding one particle into the upper free band at momentum
k to the half-filled ground state: the lowest N+1 eigenstate with nonzero
overlap with c^dag_{k,+} |GS>, minus the ground-state energy. The Fock space
has 4^sites states, so this is for a handful of sites only.
"""
from __future__ import annotations

import numpy as np

from .lattice import Lattice


def hopping_matrix(lat: Lattice) -> np.ndarray:
    """Spatial hopping matrix K (sites ordered A(i,j) then B(i,j), cell index
    j*n + i), K_xy = number of bonds between x and y. Section 8.1's 4-site model, with the neighbour
    reading of lattice.py."""
    n, m = lat.n, lat.m
    V = n * m
    K = np.zeros((2 * V, 2 * V))
    for j in range(m):
        for i in range(n):
            a = j * n + i
            for (bi, bj) in ((i, j), ((i - 1) % n, j), (i, (j - 1) % m)):
                b = V + bj * n + bi
                K[a, b] += 1.0
                K[b, a] += 1.0
    return K


class Fock:
    """Fermionic Fock space of `nmodes` modes with Jordan-Wigner ordered
    creation operators as dense matrices (mode = 2*site + spin). Section 8.1 (exact diagonalisation)."""

    def __init__(self, nmodes: int):
        self.nmodes = nmodes
        dim = 1 << nmodes
        self.dim = dim
        self.cdag = []
        for mode in range(nmodes):
            M = np.zeros((dim, dim))
            for s in range(dim):
                if not (s >> mode) & 1:
                    sign = -1.0 if bin(s & ((1 << mode) - 1)).count("1") % 2 else 1.0
                    M[s | (1 << mode), s] = sign
            self.cdag.append(M)
        self.c = [M.T.copy() for M in self.cdag]
        self.number = np.array([bin(s).count("1") for s in range(dim)])


def hubbard_hamiltonian(lat: Lattice, fock: Fock) -> np.ndarray:
    """The Hubbard Hamiltonian of the module docstring on the Fock space (Section 8.1)."""
    K = hopping_matrix(lat)
    ns = K.shape[0]
    H = np.zeros((fock.dim, fock.dim))
    for x in range(ns):
        for y in range(ns):
            if K[x, y]:
                for s in range(2):
                    H -= lat.kappa * K[x, y] * fock.cdag[2 * x + s] @ fock.c[2 * y + s]
    one = np.eye(fock.dim)
    for x in range(ns):
        nx = fock.cdag[2 * x] @ fock.c[2 * x] + fock.cdag[2 * x + 1] @ fock.c[2 * x + 1]
        H += 0.5 * lat.U * (nx - one) @ (nx - one)
    return H


def upper_band_orbital(lat: Lattice, k1: float, k2: float = 0.0) -> np.ndarray:
    """Single-particle orbital of the upper free band (energy +kappa |f(k)|) at
    lattice momentum (k1, k2), as coefficients over the sites of hopping_matrix. Section 8.1."""
    n, m = lat.n, lat.m
    V = n * m
    a = np.zeros(2 * V, complex)
    b = np.zeros(2 * V, complex)
    for j in range(m):
        for i in range(n):
            ph = np.exp(1j * (k1 * i + k2 * j)) / np.sqrt(V)
            a[j * n + i] = ph
            b[V + j * n + i] = ph
    K = hopping_matrix(lat)
    Kk = np.array([[a.conj() @ K @ a, a.conj() @ K @ b], [b.conj() @ K @ a, b.conj() @ K @ b]])
    e, v = np.linalg.eigh(-lat.kappa * Kk)
    up = np.argmax(e)
    return v[0, up] * a + v[1, up] * b, float(e[up])


def quasiparticle_energy(lat: Lattice, k1: float, k2: float = 0.0, tol: float = 1e-10) -> float:
    """E(N+1, k) - E_0(N) for a particle added in the upper band at k. Section 8.1."""
    ns = 2 * lat.n * lat.m
    fock = Fock(2 * ns)
    H = hubbard_hamiltonian(lat, fock)
    half = [s for s in range(fock.dim) if fock.number[s] == ns]
    plus = [s for s in range(fock.dim) if fock.number[s] == ns + 1]
    e0, v0 = np.linalg.eigh(H[np.ix_(half, half)])
    gs = np.zeros(fock.dim, complex)
    gs[half] = v0[:, 0]
    orb, _ = upper_band_orbital(lat, k1, k2)
    op = sum(orb[x] * fock.cdag[2 * x] for x in range(ns))
    st = (op @ gs)[plus]
    e1, v1 = np.linalg.eigh(H[np.ix_(plus, plus)])
    w = np.abs(v1.conj().T @ st) ** 2
    return float(min(e1[i] for i in range(len(e1)) if w[i] > tol) - e0[0])
