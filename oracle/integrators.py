"""Molecular dynamics for HMC (Section 2's HMC outline, Section 4, Section 5.2).

State: the field phi and its momenta pi (both real, length N). The MD
equations (Eq. p_dot) are  dphi/dtau = pi,  dpi/dtau = -dS/dphi.  Two
elementary maps:
  Q(c):     phi <- phi + c pi                  (the paper's T_pi)
  P(k, c):  pi  <- pi  - c dS_k/dphi(phi)      (the paper's T_F for force k)

Integrators:
  leapfrog       -- Q(h/2) P(h) Q(h/2) (Section 4: c1 = c2 = 1/2, d1 = 1, d2 = 0)
  omelyan        -- P(zeta h) Q(h/2) P((1-2 zeta) h) Q(h/2) P(zeta h), force first as in
                    the multi-time-scale form of Section 5.2, zeta = 0.193
  force_gradient -- Eq. force_cal (fourth order, three forces per step)
  nested omelyan -- Section 5.2: level 0 is the outermost force, level n the
                    innermost; each level's step encloses `ratio` steps of the next.
                    For an odd ratio the inner sequence is split at the middle
                    force of one inner step (the half steps T^{1/2} of Section 5.2),
                    applied recursively.

Forces are cached per (level, phi version): a force is evaluated once for each
distinct phi it is asked at. Updates to pi are never merged, so the cache does
not change any result.
"""
from __future__ import annotations

from typing import Callable, List, Sequence

import numpy as np

from . import action
from .lattice import Lattice


class Phase:
    """(phi, pi) with a version counter for the force cache. Section 2 (the HMC outline)."""

    def __init__(self, phi: np.ndarray, pi: np.ndarray):
        self.phi = phi.astype(np.float64).copy()
        self.pi = pi.astype(np.float64).copy()
        self.version = 0
        self._cache = {}
        self.nforce = 0

    def Q(self, c: float):
        self.phi = self.phi + c * self.pi
        self.version += 1

    def P(self, grad: Callable, level: int, c: float):
        key = (level, self.version)
        if key not in self._cache:
            self._cache = {k: v for k, v in self._cache.items() if k[1] == self.version}
            self._cache[key] = grad(level, self.phi)
            self.nforce += 1
        self.pi = self.pi - c * self._cache[key]


def leapfrog(st: Phase, grad: Callable, nsteps: int, tau: float = 1.0):
    """Section 4 (c1 = c2 = 1/2, d1 = 1, d2 = 0)."""
    h = tau / nsteps
    for _ in range(nsteps):
        st.Q(0.5 * h)
        st.P(grad, 0, h)
        st.Q(0.5 * h)


def omelyan(st: Phase, grad: Callable, nsteps: int, tau: float = 1.0, zeta: float = 0.193):
    """Section 4.1, force first as in Section 5.2."""
    nested_omelyan(st, grad, [nsteps], tau, zeta)


def force_gradient(st: Phase, grad: Callable, nsteps: int, tau: float = 1.0):
    """Eq. force_cal, one level. The middle kick uses the force at
    phi_tilde = phi_1 - (h^2/24) dS/dphi(phi_1)."""
    h = tau / nsteps
    for _ in range(nsteps):
        st.P(grad, 0, h / 6.0)
        st.Q(0.5 * h)
        g1 = grad(0, st.phi)
        st.nforce += 1
        phit = st.phi - (h * h / 24.0) * g1
        st.pi = st.pi - (2.0 / 3.0) * h * grad(0, phit)
        st.nforce += 1
        st.Q(0.5 * h)
        st.P(grad, 0, h / 6.0)


def level_steps(nmd: int, N: Sequence[int]) -> List[int]:
    """Steps per trajectory on each level (Section 5.2): the chi_k force (k < n)
    is applied nmd / N_k times, the innermost phi + chi_n force nmd times.
    N_0 must divide nmd and N_{k+1} must divide N_k."""
    n = len(N)
    if n and nmd % N[0]:
        raise ValueError("N_0 must divide N_MD")
    for k in range(n - 1):
        if N[k] % N[k + 1]:
            raise ValueError("N_{k+1} must divide N_k")
    return [nmd // Nk for Nk in N] + [nmd]


def nested_omelyan(st: Phase, grad: Callable, steps: Sequence[int], tau: float = 1.0,
                   zeta: float = 0.193):
    """Multi-time-scale Omelyan integrator. steps[k] = steps of level k per trajectory. Section 5.2."""
    L = len(steps)
    ratio = [steps[0]] + [steps[k] // steps[k - 1] for k in range(1, L)]
    for k in range(1, L):
        if steps[k] % steps[k - 1]:
            raise ValueError("each level's step count must divide the next")

    def inner_first(k, h):
        if k == L - 1:
            st.Q(0.5 * h)
            return
        r = ratio[k + 1]
        hh = h / r
        for _ in range(r // 2):
            step(k + 1, hh)
        if r % 2:
            half_first(k + 1, hh)

    def inner_second(k, h):
        if k == L - 1:
            st.Q(0.5 * h)
            return
        r = ratio[k + 1]
        hh = h / r
        if r % 2:
            half_second(k + 1, hh)
        for _ in range(r // 2):
            step(k + 1, hh)

    def step(k, h):
        st.P(grad, k, zeta * h)
        inner_first(k, h)
        st.P(grad, k, (1.0 - 2.0 * zeta) * h)
        inner_second(k, h)
        st.P(grad, k, zeta * h)

    def half_first(k, h):
        st.P(grad, k, zeta * h)
        inner_first(k, h)
        st.P(grad, k, 0.5 * (1.0 - 2.0 * zeta) * h)

    def half_second(k, h):
        st.P(grad, k, 0.5 * (1.0 - 2.0 * zeta) * h)
        inner_second(k, h)
        st.P(grad, k, zeta * h)

    h0 = tau / steps[0]
    for _ in range(steps[0]):
        step(0, h0)


class HasenbuschForces:
    """Level forces for n staggered masses: level k < n is the chi_k term,
    level n the Gaussian term plus the chi_n term (Section 5.2)."""

    def __init__(self, lat: Lattice, masses: Sequence[float], chis, solve):
        self.lat, self.masses, self.chis, self.solve = lat, list(masses), chis, solve

    def __call__(self, level: int, phi: np.ndarray) -> np.ndarray:
        n = len(self.masses)
        g = action.term_grad(self.lat, phi, self.masses, self.chis, level, self.solve)
        if level == n:
            g = g + action.grad_gaussian(self.lat, phi)
        return g

    def merged(self, level: int, phi: np.ndarray) -> np.ndarray:
        """All levels summed (for single-time-scale integrators)."""
        return sum(self(k, phi) for k in range(len(self.masses) + 1))


def hamiltonian(lat: Lattice, phi, pi, masses, chis, solve) -> float:
    """Eq. hamiltonian with the Hasenbusch sum in place of the single term."""
    return action.total_action(lat, phi, masses, chis, solve) + 0.5 * float(pi @ pi)


def trajectory(lat: Lattice, phi0, pi0, rhos, masses: Sequence[float], nmd: int,
               N: Sequence[int], solve, zeta: float = 0.193, tau: float = 1.0,
               integrator: str = "nested_omelyan"):
    """One MD trajectory (Section 2's HMC outline): pseudofermions from rho,
    H0, nested Omelyan integration, H1. H0 uses S_i(start) = rho_i^dagger rho_i,
    which holds exactly by construction of chi_i. Returns (phi1, pi1, H0, H1, nforce)."""
    masses = list(masses)
    chis = action.make_chi(lat, phi0, masses, rhos, solve)
    H0 = (action.gaussian_action(lat, phi0)
          + sum(float(np.real(np.vdot(r, r))) for r in rhos) + 0.5 * float(pi0 @ pi0))
    forces = HasenbuschForces(lat, masses, chis, solve)
    st = Phase(phi0, pi0)
    if integrator == "nested_omelyan":
        nested_omelyan(st, forces, level_steps(nmd, N), tau, zeta)
    elif integrator == "omelyan":
        omelyan(st, lambda k, p: forces.merged(k, p), nmd, tau, zeta)
    elif integrator == "leapfrog":
        leapfrog(st, lambda k, p: forces.merged(k, p), nmd, tau)
    elif integrator == "force_gradient":
        force_gradient(st, lambda k, p: forces.merged(k, p), nmd, tau)
    else:
        raise ValueError(integrator)
    H1 = hamiltonian(lat, st.phi, st.pi, masses, chis, solve)
    return st.phi, st.pi, H0, H1, st.nforce
