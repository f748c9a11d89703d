"""Host logic of the Hasenbusch-parameter tuner (Section 7.2): the fits of
Eqs. solver_time_eqn, small_force_eqn and large_force_eqn recover known
parameters, the masses follow Eq. mu_i_eqn, and with the paper's printed fit
values the two time-scale ratios come out nearly equal, as Section 7.2 states
for c ~ 0.4. CPU only."""
import math

import numpy as np
import pytest

from paper_1804_07195_gb300 import tuner


def test_solver_time_fit_recovers_parameters(paper):
    lam = paper["solver_time_fit"]
    ms = np.array([0.02, 0.05, 0.1, 0.2, 0.5, 1.0, 2.0, 3.0])
    t = tuner.solver_time_model(ms, 0.3, lam["lambda_max"], lam["lambda_min"])
    t0, lmax, lmin = tuner.fit_solver_time(ms, t)
    assert abs(t0 - 0.3) < 1e-6 and abs(lmax - 4.1) < 1e-5 and abs(lmin - 0.054) < 1e-7


def test_masses_are_geometric_between_the_bounds():
    mu = tuner.hasenbusch_masses(0.054, 4.1, 2)
    assert math.isclose(mu[0], 0.054 ** (2 / 3) * 4.1 ** (1 / 3), rel_tol=1e-13)
    assert math.isclose(mu[1], 0.054 ** (1 / 3) * 4.1 ** (2 / 3), rel_tol=1e-13)
    mu = tuner.hasenbusch_masses(0.1, 10.0, 4)
    ratios = np.array(mu[1:]) / np.array(mu[:-1])
    assert np.allclose(ratios, ratios[0]) and math.isclose(ratios[0], 100 ** 0.2)
    assert 0.1 < mu[0] and mu[-1] < 10.0
    with pytest.raises(ValueError):
        tuner.hasenbusch_masses(1.0, 0.5, 2)


def test_small_force_fit_and_symmetry(paper):
    p = paper["small_force_fit"]
    mu0 = np.array([0.05, 0.1, 0.2, 0.4, 1.2, 0.3, 0.7])
    mu1 = np.array([0.2, 0.3, 1.5, 0.8, 2.0, 0.35, 0.75])
    F = tuner.small_force_model(mu0, mu1, p["a"], p["b"], p["c"])
    a, b, c = tuner.fit_small_force(mu0, mu1, F)
    assert abs(a - p["a"]) < 1e-6 and abs(b - p["b"]) < 1e-6 and abs(c - p["c"]) < 1e-6
    # symmetric in the two masses, proportional to |mu1 - mu0| for small differences
    assert math.isclose(tuner.small_force_model(0.3, 0.9, a, b, c), tuner.small_force_model(0.9, 0.3, a, b, c))
    f1 = tuner.small_force_model(0.5, 0.5 + 1e-4, a, b, c)
    f2 = tuner.small_force_model(0.5, 0.5 + 2e-4, a, b, c)
    assert abs(f2 / f1 - 2.0) < 1e-3


def test_large_force_fit(paper):
    p = paper["large_force_fit"]
    ms = np.array([0.05, 0.1, 0.2, 0.4, 0.8, 1.5, 2.0, 3.0])
    F = tuner.large_force_model(ms, 10.0, 0.9, p["b"], p["c"])
    F0, a, b, c = tuner.fit_large_force(ms, F)
    assert np.allclose(tuner.large_force_model(ms, F0, a, b, c), F, rtol=1e-8)


def test_two_masses_give_nearly_equal_time_scales(paper):
    """Section 7.2: for two masses N_0' ~ N_1' when c ~ 0.4. With the printed fit
    values (lambda bounds of Section 6.1, small-force fit of Section 6.2) the
    ratio of the two small forces is close to one, so sqrt of it is too."""
    lam = paper["solver_time_fit"]
    s = paper["small_force_fit"]
    mu = tuner.hasenbusch_masses(lam["lambda_min"], lam["lambda_max"], 2)
    Np = tuner.two_mass_ratios(mu, (s["a"], s["b"], s["c"]), (10.0, 0.9, 0.0992, 0.789))
    assert abs(Np[0] / Np[1] - 1.0) < 0.15
    N0, N1 = tuner.two_mass_time_scales(Np)
    assert N0 == N1 == max(1, math.floor(math.sqrt(Np[0] * Np[1])))
    assert tuner.nmd_for_time_scales(29, (N0, N1)) % N0 == 0


class _Clock:
    def __init__(self):
        self.t = 0.0

    def now(self):
        return self.t


class _ModelContext:
    """Stands in for a Context in measure_and_tune: a solve at staggered mass
    m_s advances the clock by Eq. solver_time_eqn, and the chi_1 and top-term
    forces are constant vectors whose root mean square follows Eqs.
    small_force_eqn and large_force_eqn."""

    def __init__(self, torch, clock, N, t_par, small, large):
        self.torch, self.clock, self.N = torch, clock, N
        self.t_par, self.small, self.large = t_par, small, large
        self.solves = []

    def load_field(self, phi):
        pass

    def solve_fgmres(self, phi, ms, b, tol):
        self.solves.append(ms)
        self.clock.t += float(tuner.solver_time_model(ms, *self.t_par))
        return None, {}

    def make_chi(self, phi, masses, rho, opts=None):
        return list(masses), {}

    def force(self, phi, masses, chis, term, flags, opts=None):
        m0, m1 = masses
        v = tuner.small_force_model(m0, m1, *self.small) if term == 1 else tuner.large_force_model(m1, *self.large)
        return self.torch.full((self.N,), float(v), dtype=self.torch.float64), {}


def test_measure_and_tune_recovers_the_models(paper, monkeypatch):
    """Steps 2-4 of Section 7.2 end to end on model data: the fitted spectral
    bounds and force models reproduce the ones the data came from, the masses
    follow Eq. mu_i_eqn and the time scales Eqs. approx_N_i_eqn and used_N_eqn."""
    torch = pytest.importorskip("torch")
    clock = _Clock()
    monkeypatch.setattr(tuner.time, "perf_counter", clock.now)
    monkeypatch.setattr(torch.cuda, "synchronize", lambda: None)
    lam = paper["solver_time_fit"]
    sf = paper["small_force_fit"]
    lf = paper["large_force_fit"]
    t_par = (0.01, lam["lambda_max"], lam["lambda_min"])
    small = (sf["a"], sf["b"], sf["c"])
    large = (3.0, 0.1, lf["b"], lf["c"])
    N = 64
    ctx = _ModelContext(torch, clock, N, t_par, small, large)
    res = tuner.measure_and_tune(ctx, torch.zeros(N, dtype=torch.float64),
                                 [torch.zeros(N, dtype=torch.complex128)] * 3, repeats=2)
    assert ctx.solves == [m for m in (0.05, 0.1, 0.2, 0.4, 0.8, 1.5, 3.0) for _ in range(2)]
    assert math.isclose(res.lam_min, lam["lambda_min"], rel_tol=1e-6)
    assert math.isclose(res.lam_max, lam["lambda_max"], rel_tol=1e-6)
    assert np.allclose(res.small_force, small, rtol=1e-5)
    mu = tuner.hasenbusch_masses(lam["lambda_min"], lam["lambda_max"], 2)
    assert np.allclose(res.masses, mu, rtol=1e-6)
    top = [m1 for _, m1 in tuner.SECTION_7_2_MASS_PAIRS] + [mu[1]]
    assert np.allclose(tuner.large_force_model(top, *res.large_force), tuner.large_force_model(top, *large),
                       rtol=1e-6)
    assert res.N == tuner.two_mass_time_scales(tuner.two_mass_ratios(mu, small, large))
