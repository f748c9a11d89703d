"""Fermion determinant, pseudofermion action and force, and the Hasenbusch
splitting (Section 2 Eq. hamiltonian; Section 5 Eqs. p_dot, eta_xi, the n-mass
splitting, f_chi_i and def_xi_i).

Sign convention: the functions named `grad_*` return dS/dphi, the derivative of
the action; the MD force of Eq. p_dot is its negative, F = -dS/dphi.

The derivative of M with respect to phi_{x,t} has a single nonzero entry, in
row (x,t) at the time-hopping column (lattice.time_partner). From Eq. ferm_op:
  A row: d/dphi [ s (e^{+i phi} - delta m_s)] = +i s e^{+i phi_{x,t}}
  B row: d/dphi [-s (e^{-i phi} - delta m_s)] = +i s e^{-i phi_{x,t}}
and it does not depend on m_s (the remark above Eq. p_dot's Hasenbusch form).
"""
from __future__ import annotations

from dataclasses import dataclass
from typing import Callable, List, Optional, Sequence

import numpy as np

from . import fermion, solvers
from .lattice import A, Lattice


def dM_dphi(lat: Lattice, phi: np.ndarray) -> np.ndarray:
    """The one nonzero entry of dM/dphi_{x,t}, per row (x,t). Eq. ferm_op; the derivative entering Eqs. p_dot
    and f_chi_i."""
    s, _, _, _ = lat.coords()
    _, sign = lat.time_partner()
    return sign * np.where(s == A, 1j * np.exp(1j * phi), 1j * np.exp(-1j * phi))


def logdet_MMdag(lat: Lattice, phi: np.ndarray, ms: float = 0.0) -> float:
    """log det(M M^dagger) = 2 log|det M|, by dense LU (numpy slogdet). The fermion weight det(M M^dagger) of
    Eq. hamiltonian."""
    _, ld = np.linalg.slogdet(fermion.dense_M(lat, phi, ms))
    return 2.0 * float(ld)


def grad_logdet_MMdag(lat: Lattice, phi: np.ndarray, ms: float = 0.0) -> np.ndarray:
    """d/dphi_{x,t} log det(M M^dagger) = 2 Re tr(M^{-1} dM/dphi_{x,t})
    = 2 Re( (M^{-1})_{tp(x,t), (x,t)} * dM_{(x,t), tp(x,t)} ). Derivative of the fermion weight of Eq.
    hamiltonian."""
    Minv = np.linalg.inv(fermion.dense_M(lat, phi, ms))
    tp, _ = lat.time_partner()
    rows = np.arange(lat.N)
    return 2.0 * np.real(Minv[tp, rows] * dM_dphi(lat, phi))


def gaussian_action(lat: Lattice, phi: np.ndarray) -> float:
    """(1/2) phi^T phi / (delta U), the first term of Eq. hamiltonian."""
    return 0.5 * float(phi @ phi) / (lat.delta * lat.U)


def grad_gaussian(lat: Lattice, phi: np.ndarray) -> np.ndarray:
    """Its derivative phi / (delta U); Eq. p_dot carries -phi/(delta U) in F.
    Reading: the form -delta phi^T V^{-1} written for F_phi in the Hasenbusch
    equations is taken to mean this same term."""
    return phi / (lat.delta * lat.U)


def force_kernel(lat: Lattice, phi: np.ndarray, eta: np.ndarray, w: np.ndarray) -> np.ndarray:
    """dS/dphi_{x,t} = -2 Re( eta^*_{x,t} dM_{(x,t),tp} w_{tp} ) for an action whose
    variation is dS = -2 Re(eta^dagger dM w) (Eq. p_dot with w = xi, Eq. f_chi_i
    with w = xi - chi)."""
    tp, _ = lat.time_partner()
    return -2.0 * np.real(np.conj(eta) * dM_dphi(lat, phi) * np.take(w, tp))


class SolveA:
    """x = (M_ms M_ms^dagger)^{-1} b by one of the oracle's solvers:
    "dense" (LU of the explicit M M^dagger), "splu" (sparse LU of M, then
    x = M^{-dagger} (M^{-1} b)) or "cg"."""

    def __init__(self, lat: Lattice, method: str = "dense", tol: float = 1e-13):
        self.lat, self.method, self.tol = lat, method, tol

    def __call__(self, phi, ms, b):
        lat = self.lat
        if self.method == "dense":
            Mx = fermion.dense_M(lat, phi, ms)
            return solvers.dense_solve(Mx @ Mx.conj().T, b)
        if self.method == "splu":
            import scipy.sparse.linalg as spla
            lu = spla.splu(fermion.sparse_M(lat, phi, ms))
            return lu.solve(lu.solve(b.astype(np.complex128)), trans="H")
        if self.method == "cg":
            res = solvers.cg(lambda v: fermion.apply_MMdag(lat, phi, ms, v), b, tol=self.tol)
            if not res.converged:
                raise RuntimeError("oracle CG did not converge")
            return res.x
        raise ValueError(self.method)


def pf_action(lat: Lattice, phi, ms, chi, solve: SolveA) -> float:
    """S = chi^dagger (M M^dagger)^{-1} chi (Eq. hamiltonian)."""
    eta = solve(phi, ms, chi)
    return float(np.real(np.vdot(chi, eta)))


def grad_pf_action(lat: Lattice, phi, ms, chi, solve: SolveA) -> np.ndarray:
    """dS/dphi for S = chi^dagger (M M^dagger)^{-1} chi at fixed chi:
    eta = (M M^dagger)^{-1} chi, xi = M^dagger eta (Eq. eta_xi), dS = -2 Re(eta^dagger dM xi)."""
    eta = solve(phi, ms, chi)
    xi = fermion.apply_Mdag(lat, phi, ms, eta)
    return force_kernel(lat, phi, eta, xi)


# ----- Hasenbusch splitting with staggered masses (Section 5.1) ---------------
#
# Masses mu_0 < ... < mu_{n-1}; M_{mu_{-1}} = M (m_s = 0). Terms i = 0..n:
#   S_n = chi_n^dagger (M_{mu_{n-1}} M_{mu_{n-1}}^dagger)^{-1} chi_n
#   S_i = |M_{mu_{i-1}}^{-1} M_{mu_i} chi_i|^2
#       = (M_{mu_i} chi_i)^dagger (M_{mu_{i-1}} M_{mu_{i-1}}^dagger)^{-1} (M_{mu_i} chi_i), i < n.

def lower_mass(masses: Sequence[float], i: int) -> float:
    """mu_{i-1}, with mu_{-1} = 0 (the unshifted operator). Section 5.1."""
    return 0.0 if i == 0 else float(masses[i - 1])


def make_chi(lat: Lattice, phi, masses: Sequence[float], rhos: Sequence[np.ndarray],
             solve: SolveA) -> List[np.ndarray]:
    """Pseudofermions from heat-bath vectors rho_i:
    chi_n = M_{mu_{n-1}} rho_n;  chi_i = M_{mu_i}^dagger (M_{mu_i} M_{mu_i}^dagger)^{-1} M_{mu_{i-1}}
    rho_i. Section 5.1."""
    n = len(masses)
    if len(rhos) != n + 1:
        raise ValueError("need n+1 heat-bath vectors for n masses")
    chis = []
    for i in range(n):
        u = fermion.apply_M(lat, phi, lower_mass(masses, i), rhos[i])
        y = solve(phi, masses[i], u)
        chis.append(fermion.apply_Mdag(lat, phi, masses[i], y))
    top = float(masses[n - 1]) if n > 0 else 0.0
    chis.append(fermion.apply_M(lat, phi, top, rhos[n]))
    return chis


def term_action(lat: Lattice, phi, masses, chis, i: int, solve: SolveA) -> float:
    """S_i of the Hasenbusch splitting with staggered masses (Section 5.1)."""
    n = len(masses)
    lo = lower_mass(masses, i)
    if i == n:
        src = chis[n]
    else:
        src = fermion.apply_M(lat, phi, masses[i], chis[i])
    eta = solve(phi, lo, src)
    return float(np.real(np.vdot(src, eta)))


def term_grad(lat: Lattice, phi, masses, chis, i: int, solve: SolveA) -> np.ndarray:
    """dS_i/dphi. Eq. f_chi_i with eta_i = (M_{i-1} M_{i-1}^dagger)^{-1} M_{mu_i} chi_i,
    xi_i = M_{i-1}^dagger eta_i, and w = xi_i - chi_i; for the top term w = xi_n."""
    n = len(masses)
    lo = lower_mass(masses, i)
    if i == n:
        eta = solve(phi, lo, chis[n])
        xi = fermion.apply_Mdag(lat, phi, lo, eta)
        return force_kernel(lat, phi, eta, xi)
    src = fermion.apply_M(lat, phi, masses[i], chis[i])
    eta = solve(phi, lo, src)
    xi = fermion.apply_Mdag(lat, phi, lo, eta)
    return force_kernel(lat, phi, eta, xi - chis[i])


def total_action(lat: Lattice, phi, masses, chis, solve: SolveA) -> float:
    """S(phi) = (1/2) phi^2/(delta U) + sum_i S_i. Eq. hamiltonian with the splitting of Section 5.1."""
    return gaussian_action(lat, phi) + sum(
        term_action(lat, phi, masses, chis, i, solve) for i in range(len(masses) + 1))


def total_grad(lat: Lattice, phi, masses, chis, solve: SolveA) -> np.ndarray:
    """dS/dphi of total_action: the Gaussian term plus every term (Eqs. p_dot, f_chi_i, def_xi_i)."""
    g = grad_gaussian(lat, phi)
    for i in range(len(masses) + 1):
        g = g + term_grad(lat, phi, masses, chis, i, solve)
    return g
