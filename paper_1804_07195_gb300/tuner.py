"""Automatic choice of Hasenbusch masses and time scales (Section 7.2).

The procedure of Section 7.2, steps 2 to 4, on top of libhmc:
  * measure the time of one inversion of M_ms M_ms^dagger for several staggered
    masses and fit  t(m_s) = t0 (lambda_max + m_s) / (lambda_min + m_s)
    (Eq. solver_time_eqn), which yields the spectral bounds;
  * place n masses geometrically between them,
    mu_i = lambda_min (lambda_max / lambda_min)^((i+1)/(n+1))  (Eq. mu_i_eqn);
  * measure the forces of the Hasenbusch terms for the mass pairs the paper
    lists and fit  |F_chi1| = a |mu1 - mu0| / ((b + mu0)(b + mu1))^c
    (Eq. small_force_eqn) and  |F_phi+chi_n| = F0 - a~ m_s / (b~ (b~ + m_s))^c~
    (Eq. large_force_eqn);
  * time-scale ratios N_i' = sqrt(F_phi+chi_n(mu_{n-1}) / F_chi_i(mu_{i-1}, mu_i))
    (Eq. approx_N_i_eqn), and for two masses N_0 = N_1 = floor(sqrt(N_0' N_1'))
    (Eq. used_N_eqn).
The fits are plain host code (scipy); the measurements call the library.
"""
from __future__ import annotations

import math
import time
from dataclasses import dataclass, field
from typing import Callable, Dict, List, Sequence, Tuple

import numpy as np

# Step 2 of Section 7.2: the mass pairs (m_0, m_1) measured with N_0 = N_1 = 1.
SECTION_7_2_MASS_PAIRS = ((0.05, 0.2), (0.1, 0.3), (0.2, 1.5), (0.4, 0.8), (1.2, 2.0))


def solver_time_model(ms, t0, lam_max, lam_min):
    """Eq. solver_time_eqn."""
    ms = np.asarray(ms, dtype=float)
    return t0 * (lam_max + ms) / (lam_min + ms)


def fit_solver_time(ms: Sequence[float], times: Sequence[float]) -> Tuple[float, float, float]:
    """Least-squares fit of Eq. solver_time_eqn; returns (t0, lambda_max, lambda_min)
    with 0 < lambda_min < lambda_max. Relative residuals are minimised, since
    the times span orders of magnitude."""
    from scipy.optimize import least_squares
    ms = np.asarray(ms, dtype=float)
    times = np.asarray(times, dtype=float)
    if ms.size < 3:
        raise ValueError("need at least three (m_s, time) points")
    # start from the two extreme points, with lambda_min small
    x0 = np.array([np.log(times.min()), np.log(4.0), np.log(0.05)])

    def res(p):
        t0, lmax, lmin = np.exp(p)
        return solver_time_model(ms, t0, lmax, lmin) / times - 1.0

    sol = least_squares(res, x0, method="lm", xtol=1e-14, ftol=1e-14, gtol=1e-14, max_nfev=20000)
    t0, lmax, lmin = np.exp(sol.x)
    if lmin > lmax:
        lmin, lmax = lmax, lmin
    return float(t0), float(lmax), float(lmin)


def hasenbusch_masses(lam_min: float, lam_max: float, n: int) -> List[float]:
    """Eq. mu_i_eqn: n masses placed geometrically in [lambda_min, lambda_max]."""
    if not (0 < lam_min < lam_max) or n < 1:
        raise ValueError("need 0 < lambda_min < lambda_max and n >= 1")
    return [lam_min * (lam_max / lam_min) ** ((i + 1) / (n + 1)) for i in range(n)]


def small_force_model(mu0, mu1, a, b, c):
    """Eq. small_force_eqn."""
    mu0 = np.asarray(mu0, dtype=float)
    mu1 = np.asarray(mu1, dtype=float)
    return a * np.abs(mu1 - mu0) / ((b + mu0) * (b + mu1)) ** c


def fit_small_force(mu0, mu1, F) -> Tuple[float, float, float]:
    from scipy.optimize import least_squares
    mu0, mu1, F = (np.asarray(v, dtype=float) for v in (mu0, mu1, F))

    def res(p):
        a, b, c = p
        return small_force_model(mu0, mu1, a, b, c) / F - 1.0

    sol = least_squares(res, np.array([0.4, 0.1, 0.4]), bounds=([1e-12, 1e-9, 0.0], [np.inf, 10.0, 5.0]),
                        xtol=1e-14, ftol=1e-14, gtol=1e-14, max_nfev=20000)
    return tuple(float(v) for v in sol.x)


def large_force_model(ms, F0, a, b, c):
    """Eq. large_force_eqn."""
    ms = np.asarray(ms, dtype=float)
    return F0 - a * ms / (b * (b + ms)) ** c


def fit_large_force(ms, F) -> Tuple[float, float, float, float]:
    from scipy.optimize import least_squares
    ms, F = np.asarray(ms, dtype=float), np.asarray(F, dtype=float)

    def res(p):
        return large_force_model(ms, *p) / F - 1.0

    x0 = np.array([F.max() * 1.05, 0.1, 0.1, 0.8])
    sol = least_squares(res, x0, bounds=([0.0, 0.0, 1e-9, 0.0], [np.inf, np.inf, 10.0, 5.0]),
                        xtol=1e-14, ftol=1e-14, gtol=1e-14, max_nfev=20000)
    return tuple(float(v) for v in sol.x)


def time_scale_ratios(F_top: float, F_terms: Sequence[float]) -> List[float]:
    """Eq. approx_N_i_eqn: N_i' = sqrt(F_phi+chi_n / F_chi_i)."""
    return [math.sqrt(F_top / f) for f in F_terms]


def two_mass_ratios(masses: Sequence[float], small: Sequence[float], large: Sequence[float]) -> List[float]:
    """N_0', N_1' for two masses from the fitted force models: the chi_0 term
    couples mu_0 to the unshifted operator (mu_{-1} = 0), the chi_1 term mu_0 to
    mu_1, and the top term phi + chi_2 depends on mu_1."""
    F_terms = [float(small_force_model(0.0, masses[0], *small)),
               float(small_force_model(masses[0], masses[1], *small))]
    F_top = float(large_force_model(masses[1], *large))
    return time_scale_ratios(F_top, F_terms)


def two_mass_time_scales(Np: Sequence[float]) -> Tuple[int, int]:
    """Eq. used_N_eqn: N_0 = N_1 = floor(sqrt(N_0' N_1')) (at least 1)."""
    n = max(1, int(math.floor(math.sqrt(Np[0] * Np[1]))))
    return n, n


def nmd_for_time_scales(nmd_target: int, N: Sequence[int]) -> int:
    """The smallest N_MD >= nmd_target that the coarsest ratio divides."""
    k = max(int(N[0]), 1)
    return int(math.ceil(nmd_target / k) * k)


@dataclass
class TuneResult:
    lam_min: float
    lam_max: float
    t0: float
    masses: List[float]
    small_force: Tuple[float, float, float]
    large_force: Tuple[float, float, float, float]
    N_prime: List[float]
    N: Tuple[int, int]
    measurements: Dict[str, list] = field(default_factory=dict)


def force_norm(g) -> float:
    """Size of one force term: the root mean square over sites."""
    import torch
    return float(torch.linalg.vector_norm(g).item() / math.sqrt(g.numel()))


def pair_forces(ctx, phi, rho, m0: float, m1: float, opts):
    """The two forces Section 7.2 measures for the mass pair (m0, m1) of a
    two-mass Hasenbusch action, as CUDA tensors: dS_1/dphi of the chi_1 term
    (Eq. f_chi_i; its size enters Eq. small_force_eqn) and dS/dphi of the
    Gaussian plus top term phi + chi_2 (Eq. large_force_eqn). The
    pseudofermions come from the heat-bath vectors rho at the field phi."""
    from . import _abi
    chis, _ = ctx.make_chi(phi, [m0, m1], rho, opts=opts)
    F1, _ = ctx.force(phi, [m0, m1], chis, term=1, flags=_abi.HMC_FERMION, opts=opts)
    F2, _ = ctx.force(phi, [m0, m1], chis, term=2, flags=_abi.HMC_FERMION | _abi.HMC_GAUSSIAN, opts=opts)
    return F1, F2


def measure_and_tune(ctx, phi, rho, solve_masses: Sequence[float] = (0.05, 0.1, 0.2, 0.4, 0.8, 1.5, 3.0),
                     pairs: Sequence[Tuple[float, float]] = SECTION_7_2_MASS_PAIRS, tol: float = 1e-10,
                     repeats: int = 2) -> TuneResult:
    """Steps 2-4 of Section 7.2 on the field phi (a CUDA tensor) with heat-bath
    vectors rho (three complex128 CUDA tensors): time the mixed-precision
    inversion of M_ms M_ms^dagger for each staggered mass, measure the three
    forces of the two-mass Hasenbusch action for each mass pair, fit, and
    return two masses and their time scales."""
    import torch
    from . import SolverOpts, _abi
    opts = SolverOpts(method=_abi.HMC_SOLVER_FGMRES_MIXED, tol=tol)
    b = rho[0]
    ctx.load_field(phi)
    times = []
    for ms in solve_masses:
        best = math.inf
        for _ in range(repeats):
            torch.cuda.synchronize()
            t = time.perf_counter()
            ctx.solve_fgmres(None, ms, b, tol=tol)
            torch.cuda.synchronize()
            best = min(best, time.perf_counter() - t)
        times.append(best)
    t0, lmax, lmin = fit_solver_time(solve_masses, times)
    small_mu0, small_mu1, small_F, top_ms, top_F = [], [], [], [], []
    for (m0, m1) in pairs:
        F1, F2 = pair_forces(ctx, phi, rho, m0, m1, opts)
        small_mu0.append(m0)
        small_mu1.append(m1)
        small_F.append(force_norm(F1))
        top_ms.append(m1)
        top_F.append(force_norm(F2))
    a, bb, c = fit_small_force(small_mu0, small_mu1, small_F)
    large = fit_large_force(top_ms, top_F)
    masses = hasenbusch_masses(lmin, lmax, 2)
    Np = two_mass_ratios(masses, (a, bb, c), large)
    return TuneResult(lmin, lmax, t0, masses, (a, bb, c), large, Np, two_mass_time_scales(Np),
                      {"solve_masses": list(solve_masses), "times": times, "pairs": [list(p) for p in pairs],
                       "F_chi1": small_F, "F_top": top_F})
