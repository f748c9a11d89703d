"""Honeycomb torus geometry (Section 2 and Eq. ferm_op).

An n x m lattice of rhombic unit cells, each holding one A and one B site,
periodic along both oblique axes; 2*n*m spatial sites and nt time slices.

Reading of the neighbour convention (the paper defers it to a figure of another
reference): A(i, j) is bonded to B(i, j), B(i-1, j) and B(i, j-1), indices taken
mod n and mod m; B(i, j) is bonded to A(i, j), A(i+1, j) and A(i, j+1). For n or
m below 3 some of these bonds coincide and are counted with multiplicity, so
every site keeps exactly three bonds.

Canonical index of site (s, t, i, j):  ((s * nt + t) * m + j) * n + i.
"""
from __future__ import annotations

import numpy as np

A = 0
B = 1


class Lattice:
    """Section 2 and Eq. ferm_op, with the readings of the module docstring."""
    def __init__(self, n: int, m: int, nt: int, kappa: float, U: float, beta: float):
        if min(n, m, nt) < 1:
            raise ValueError("n, m, nt must be positive")
        self.n, self.m, self.nt = int(n), int(m), int(nt)
        self.kappa, self.U, self.beta = float(kappa), float(U), float(beta)
        # delta: the time step, beta / nt (text after Eq. hamiltonian).
        self.delta = self.beta / self.nt
        self.V = self.n * self.m
        self.N = 2 * self.V * self.nt

    @classmethod
    def from_params(cls, p) -> "Lattice":
        """Section 2."""
        return cls(p.n, p.m, p.nt, p.kappa, p.U, p.beta)

    def index(self, s, t, i, j):
        """The canonical layout of the module docstring."""
        return ((s * self.nt + t) * self.m + j) * self.n + i

    def coords(self):
        """Arrays (s, t, i, j) for every canonical index, in index order. The canonical layout of the module
        docstring."""
        s, t, j, i = np.meshgrid(np.arange(2), np.arange(self.nt), np.arange(self.m),
                                 np.arange(self.n), indexing="ij")
        return s.ravel(), t.ravel(), i.ravel(), j.ravel()

    def spatial_neighbours(self) -> np.ndarray:
        """(N, 3) array: the three hopping partners of every space-time site,
        at the same time slice, on the other sublattice. Eq. ferm_op, with the neighbour reading of the
        module docstring."""
        s, t, i, j = self.coords()
        n, m = self.n, self.m
        nb = np.empty((self.N, 3), dtype=np.int64)
        isA = s == A
        # A(i,j) -> B(i,j), B(i-1,j), B(i,j-1)
        nb[isA, 0] = self.index(B, t[isA], i[isA], j[isA])
        nb[isA, 1] = self.index(B, t[isA], (i[isA] - 1) % n, j[isA])
        nb[isA, 2] = self.index(B, t[isA], i[isA], (j[isA] - 1) % m)
        isB = ~isA
        # B(i,j) -> A(i,j), A(i+1,j), A(i,j+1)
        nb[isB, 0] = self.index(A, t[isB], i[isB], j[isB])
        nb[isB, 1] = self.index(A, t[isB], (i[isB] + 1) % n, j[isB])
        nb[isB, 2] = self.index(A, t[isB], i[isB], (j[isB] + 1) % m)
        return nb

    def time_partner(self):
        """The column of the time-hopping entry of M in every row, and its
        boundary sign. Eq. ferm_op: an A row (x, t) couples to (x, t-1), a B
        row (x, t) to (x, t+1). Reading of the time boundary (not stated in the
        paper, which defers to its references): anti-periodic, so the entry
        that wraps around the time circle carries a factor -1."""
        s, t, i, j = self.coords()
        nt = self.nt
        tp = np.where(s == A, (t - 1) % nt, (t + 1) % nt)
        wraps = np.where(s == A, t == 0, t == nt - 1)
        sign = np.where(wraps, -1.0, 1.0)
        return self.index(s, tp, i, j).astype(np.int64), sign
