"""Host logic of the N_MD auto-tuner (Algorithm B.1), pinned to mathematics:
the skew-normal CDF against its closed forms and a direct quadrature of its
density, the model inversion against the normal quantile, and the whole loop
against a simulated HMC whose acceptance has a closed form.

For a Gaussian energy violation dH ~ N(mu, 2 mu) (the form that
<exp(-dH)> = 1 forces on a Gaussian), the mean acceptance probability is
<min(1, exp(-dH))> = erfc(sqrt(mu) / 2); with a second-order integrator
mu = C / N_MD^4, so the N_MD that gives acceptance p is
(C / (4 erfcinv(p)^2))^(1/4)."""
import math
from statistics import NormalDist

import numpy as np
import pytest

from paper_1804_07195_gb300 import nmd_tuner as nt

PHI = NormalDist().cdf


@pytest.mark.parametrize("x", [-2.5, -0.7, 0.0, 0.3, 1.9])
def test_skewnorm_cdf_closed_forms(x):
    # alpha = 0 is the normal distribution, alpha = 1 gives Phi(x)^2
    assert abs(float(nt.skewnorm_cdf(x, 0.0)) - PHI(x)) < 1e-14
    assert abs(float(nt.skewnorm_cdf(x, 1.0)) - PHI(x) ** 2) < 1e-14
    # alpha -> infinity: the half-normal, 2 Phi(x) - 1 on x > 0 and 0 below
    lim = 2 * PHI(x) - 1 if x > 0 else 0.0
    if x != 0.0:
        assert abs(float(nt.skewnorm_cdf(x, 1e6)) - lim) < 1e-9
    # reflection: F(x; -alpha) = 1 - F(-x; alpha)
    assert abs(float(nt.skewnorm_cdf(x, -3.0)) - (1 - float(nt.skewnorm_cdf(-x, 3.0)))) < 1e-14


@pytest.mark.parametrize("alpha", [-4.0, 0.5, 3.0])
def test_skewnorm_cdf_against_quadrature_of_the_density(alpha):
    from scipy.integrate import quad
    pdf = lambda t: 2.0 * math.exp(-0.5 * t * t) / math.sqrt(2 * math.pi) * PHI(alpha * t)
    for x in (-1.5, 0.2, 1.1):
        val, _ = quad(pdf, -40.0, x, epsabs=1e-14, epsrel=1e-13)
        assert abs(float(nt.skewnorm_cdf(x, alpha)) - val) < 1e-10


def test_confidence_interval():
    m, lo, hi = nt.confidence_interval([0.5, 0.7, 0.6, 0.9])
    s = math.sqrt(((0.5 - 0.675) ** 2 + (0.7 - 0.675) ** 2 + (0.6 - 0.675) ** 2 + (0.9 - 0.675) ** 2) / 3)
    assert math.isclose(m, 0.675)
    assert math.isclose(lo, 0.675 - 1.96 * s / 2) and math.isclose(hi, 0.675 + 1.96 * s / 2)
    # clipped to [0, 1]
    m, lo, hi = nt.confidence_interval([1.0, 1.0, 0.2])
    assert hi == 1.0 and lo > 0.0
    assert nt.confidence_interval([0.3]) == (0.3, 0.0, 1.0)


def test_predict_inverts_the_normal_model():
    b1, b0 = 0.05, -2.0
    for p in (0.3, 0.66, 0.9):
        n_exact = (NormalDist().inv_cdf(p) - b0) / b1
        assert nt.predict_nmd((b1, b0, 0.0), p) == math.ceil(n_exact)
        assert nt.predict_nmd((b1, b0, 0.0), p, multiple=6) == 6 * math.ceil(n_exact / 6)


def test_fit_recovers_the_model_from_exact_points():
    truth = (0.04, -1.5, 2.0)
    N = np.array([10.0, 25.0, 40.0, 60.0, 90.0])
    P = nt.acceptance_model(N, *truth)
    b1, b0, al = nt.fit_acceptance(N, P, anchors=False)
    assert np.max(np.abs(nt.acceptance_model(N, b1, b0, al) - P)) < 1e-6
    assert abs(nt.predict_nmd((b1, b0, al)) - nt.predict_nmd(truth)) <= 1


def gaussian_hmc(C, seed):
    g = np.random.default_rng(seed)

    def simulate(nmd):
        mu = C / float(nmd) ** 4
        dH = g.normal(mu, math.sqrt(2 * mu))
        return math.exp(min(0.0, -dH))
    return simulate


def n_star(C, p=nt.TARGET_ACCEPTANCE):
    from scipy.special import erfcinv
    return (C / (4 * erfcinv(p) ** 2)) ** 0.25


def test_gaussian_hmc_acceptance_closed_form():
    # the simulator itself: mean acceptance erfc(sqrt(mu)/2)
    C = 2.0e5
    sim = gaussian_hmc(C, 1)
    for nmd in (15, 25):
        acc = np.mean([sim(nmd) for _ in range(40000)])
        assert abs(acc - math.erfc(math.sqrt(C / nmd ** 4) / 2)) < 0.01


@pytest.mark.parametrize("C,nmd0,seed", [(2.0e5, 500, 3), (3.0e7, 500, 4), (5.0e4, 8, 5)])
def test_tuner_finds_the_target_acceptance(C, nmd0, seed):
    res = nt.tune_nmd(gaussian_hmc(C, seed), nmd0=nmd0)
    target = n_star(C)
    assert res.total_trajectories <= 500
    assert res.reason in ("repeated N_MD", "target inside interval", "trajectory limit")
    p_final = math.erfc(math.sqrt(C / res.nmd ** 4) / 2)
    assert abs(p_final - nt.TARGET_ACCEPTANCE) < 0.12, (res.nmd, target, p_final)
    # every phase ran more than five trajectories or hit the limit
    assert all(h.trajectories > 5 or res.reason == "trajectory limit" for h in res.history)


def test_tuner_stops_at_the_trajectory_limit():
    calls = []

    def sim(nmd):
        calls.append(nmd)
        return 0.0 if len(calls) % 2 else 1.0   # wide interval: phase 1 never settles

    res = nt.tune_nmd(sim, nmd0=20, max_total=40)
    assert res.reason == "trajectory limit" and res.total_trajectories == 40 == len(calls)


def test_tuner_respects_time_scale_multiple():
    res = nt.tune_nmd(gaussian_hmc(2.0e5, 7), nmd0=500, multiple=4)
    assert all(h.nmd % 4 == 0 for h in res.history) and res.nmd % 4 == 0


@pytest.mark.parametrize("C,seed,split", [(2.0e5, 3, 1), (3.0e7, 4, 2)])
def test_resumed_experiment_ends_as_the_unsplit_one(tmp_path, C, seed, split):
    """Algorithm B.1 resumed from a saved experiment: stopping after `split`
    phases (trajectory limit at that phase's end), saving the measurements,
    loading them and resuming with the same trajectory stream reproduces the
    unsplit run: the same N_MD, stopping rule, trajectory count and phases."""
    full = nt.tune_nmd(gaussian_hmc(C, seed), nmd0=500)
    assert len(full.history) > split
    sim = gaussian_hmc(C, seed)
    first = nt.tune_nmd(sim, nmd0=500, max_total=sum(h.trajectories for h in full.history[:split]))
    assert first.reason == "trajectory limit" and len(first.history) == split
    path = str(tmp_path / "nmd.json")
    nt.save_history(first.history, path)
    resumed = nt.tune_nmd(sim, nmd0=500, resume=nt.load_history(path))
    assert (resumed.nmd, resumed.reason, resumed.total_trajectories) == \
        (full.nmd, full.reason, full.total_trajectories)
    assert [(h.nmd, h.trajectories, h.mean) for h in resumed.history] == \
        [(h.nmd, h.trajectories, h.mean) for h in full.history]


def test_resume_applies_the_stopping_rules_first():
    """A resumed experiment that already meets a stopping rule runs no
    trajectory."""
    def never(nmd):
        raise AssertionError("no trajectory expected")

    hit = [nt.NmdMeasurement(40, 0.66, 0.6, 0.72, 10)] * 3
    res = nt.tune_nmd(never, resume=hit)
    assert res.reason in ("target inside interval", "repeated N_MD") and res.total_trajectories == 30
    spent = [nt.NmdMeasurement(20, 0.1, 0.0, 0.3, 250), nt.NmdMeasurement(60, 0.9, 0.8, 1.0, 250)]
    res = nt.tune_nmd(never, resume=spent)
    assert res.reason == "trajectory limit" and res.total_trajectories == 500
    assert 20 < res.nmd < 60
