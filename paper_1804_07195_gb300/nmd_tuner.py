"""Automatic choice of the number of MD steps N_MD (Section 7.1, Algorithm B.1).

The tuner alternates two phases until one of its stopping rules holds:
  1. run trajectories at the current N_MD until the confidence interval of the
     mean acceptance is narrow (width <= 0.25 after more than five
     trajectories), the interval taken from the normal approximation of the
     sample mean and clipped to [0, 1];
  2. fit the model p_acc(N_MD) = CDF_skew-normal(beta_1 N_MD + beta_0; alpha)
     to every (N_MD, mean acceptance) pair measured so far, plus two artificial
     anchor points that fix the ends of the S-shaped curve, and take the next
     N_MD where the model reaches the target acceptance (0.66).
It stops after 500 trajectories in all, when the proposed N_MD has already
been measured three times, or when the target fell inside the measured
confidence interval three times.
An experiment can be saved (`save_history`) and resumed from its
measurements (`tune_nmd(..., resume=load_history(path))`), the algorithm's
"initialise or resume" step.

The skew-normal CDF (Azzalini's distribution) is Phi(x) - 2 T(x, alpha) with
T Owen's T function. This module is host logic only: `simulate(nmd)` runs one
trajectory (on the device, through `Chain.trajectory`) and returns that
trajectory's acceptance probability min(1, exp(-dH)).
"""
from __future__ import annotations

import json
import math
from dataclasses import asdict, dataclass, field
from typing import Callable, List, Optional, Sequence, Tuple

import numpy as np

TARGET_ACCEPTANCE = 0.66


def skewnorm_cdf(x, alpha):
    """CDF of the standard skew-normal distribution with shape alpha."""
    from scipy.special import ndtr, owens_t
    x = np.asarray(x, dtype=float)
    return ndtr(x) - 2.0 * owens_t(x, alpha)


def acceptance_model(nmd, beta1: float, beta0: float, alpha: float):
    """The model of the second phase: p_acc as a function of N_MD."""
    return skewnorm_cdf(beta1 * np.asarray(nmd, dtype=float) + beta0, alpha)


def confidence_interval(samples: Sequence[float], z: float = 1.96) -> Tuple[float, float, float]:
    """(mean, lower, upper): mean +- z s / sqrt(n), clipped to [0, 1]. With
    fewer than two samples the interval is all of [0, 1]."""
    a = np.asarray(samples, dtype=float)
    if a.size == 0:
        return 0.0, 0.0, 1.0
    mean = float(a.mean())
    if a.size < 2:
        return mean, 0.0, 1.0
    half = z * float(a.std(ddof=1)) / math.sqrt(a.size)
    return mean, max(0.0, mean - half), min(1.0, mean + half)


def anchor_points(nmds: Sequence[float], far: float = 10.0) -> List[Tuple[float, float]]:
    """The two artificial points: no acceptance at N_MD = 0, full acceptance
    far beyond the largest N_MD measured."""
    return [(0.0, 0.0), (far * max(max(nmds), 1.0), 1.0)]


def fit_acceptance(nmds: Sequence[float], paccs: Sequence[float],
                   anchors: bool = True) -> Tuple[float, float, float]:
    """Least-squares fit of (beta_1, beta_0, alpha) to the measured pairs (and
    the anchors). beta_1 is kept positive so that acceptance grows with N_MD;
    the best of a few starting points is kept."""
    from scipy.optimize import least_squares
    pts = list(zip(map(float, nmds), map(float, paccs)))
    if anchors:
        pts += anchor_points(nmds)
    N = np.array([p[0] for p in pts])
    P = np.array([p[1] for p in pts])
    scale = max(float(np.max(np.asarray(nmds, dtype=float))), 1.0)
    u = N / scale  # fit in N / scale so that the parameters are of order one

    def res(q):
        return skewnorm_cdf(q[0] * u + q[1], q[2]) - P

    best = None
    for s in ((4.0, -2.0, 0.0), (8.0, -3.0, 2.0), (2.0, -1.0, -2.0), (16.0, -6.0, 4.0)):
        sol = least_squares(res, np.array(s), bounds=([1e-9, -np.inf, -50.0], [np.inf, np.inf, 50.0]),
                            xtol=1e-12, ftol=1e-12, gtol=1e-12, max_nfev=5000)
        if best is None or sol.cost < best.cost:
            best = sol
    b1, b0, al = best.x
    return float(b1 / scale), float(b0), float(al)


def predict_nmd(params: Tuple[float, float, float], target: float = TARGET_ACCEPTANCE,
                multiple: int = 1, n_max: int = 1 << 20) -> int:
    """The smallest N_MD (a multiple of `multiple`) at which the model reaches
    the target acceptance."""
    b1, b0, al = params
    lo, hi = 0.0, 1.0
    f = lambda n: float(acceptance_model(n, b1, b0, al)) - target
    while f(hi) < 0.0 and hi < n_max:
        lo, hi = hi, hi * 2.0
    if f(hi) < 0.0:
        return int(math.ceil(n_max / multiple) * multiple)
    for _ in range(200):  # bisection on the monotone model
        mid = 0.5 * (lo + hi)
        if f(mid) < 0.0:
            lo = mid
        else:
            hi = mid
    return max(multiple, int(math.ceil(hi / multiple) * multiple))


@dataclass
class NmdMeasurement:
    nmd: int
    mean: float
    lower: float
    upper: float
    trajectories: int


@dataclass
class NmdTuneResult:
    nmd: int
    reason: str
    total_trajectories: int
    history: List[NmdMeasurement] = field(default_factory=list)
    params: Optional[Tuple[float, float, float]] = None


def save_history(history: Sequence[NmdMeasurement], path: str) -> None:
    """Write the measurements of an experiment (one entry per N_MD phase) as
    JSON, for a later run to resume from."""
    with open(path, "w") as f:
        json.dump({"history": [asdict(h) for h in history]}, f)


def load_history(path: str) -> List[NmdMeasurement]:
    with open(path) as f:
        return [NmdMeasurement(**h) for h in json.load(f)["history"]]


def tune_nmd(simulate: Callable[[int], float], nmd0: int = 500, target: float = TARGET_ACCEPTANCE,
             ci_width: float = 0.25, min_trajectories: int = 5, max_total: int = 500,
             repeat_stop: int = 3, hit_stop: int = 3, multiple: int = 1, z: float = 1.96,
             resume: Optional[Sequence[NmdMeasurement]] = None) -> NmdTuneResult:
    """Algorithm B.1. `simulate(nmd)` runs one trajectory with N_MD = nmd and
    returns its acceptance probability; `multiple` rounds every proposed N_MD
    up to a multiple of the coarsest time-scale ratio.

    `resume`: the measurements of a previous experiment (the algorithm's
    "initialise or resume" step). They count as if just made: the model is fitted
    to them, the stopping rules see them, and their trajectories count toward
    `max_total`; the run then continues at the N_MD the model proposes, so an
    experiment split at a phase boundary ends as the unsplit one would."""
    nmd = int(math.ceil(nmd0 / multiple) * multiple)
    history: List[NmdMeasurement] = list(resume or [])
    nmd_list: List[int] = [h.nmd for h in history]
    p_list: List[float] = [h.mean for h in history]
    total = sum(h.trajectories for h in history)
    hits = sum(1 for h in history if h.lower <= target <= h.upper)
    params = None
    if history:
        params = fit_acceptance(nmd_list, p_list)
        nmd = predict_nmd(params, target, multiple)
        if total >= max_total:
            return NmdTuneResult(nmd, "trajectory limit", total, history, params)
        if nmd_list.count(nmd) >= repeat_stop:
            return NmdTuneResult(nmd, "repeated N_MD", total, history, params)
        if hits >= hit_stop:
            return NmdTuneResult(nmd, "target inside interval", total, history, params)
    while True:
        # phase 1: measure the acceptance at nmd until its interval is narrow
        samples: List[float] = []
        while True:
            samples.append(float(simulate(nmd)))
            total += 1
            mean, lo, hi = confidence_interval(samples, z)
            if (hi - lo <= ci_width and len(samples) > min_trajectories) or total >= max_total:
                break
        history.append(NmdMeasurement(nmd, mean, lo, hi, len(samples)))
        nmd_list.append(nmd)
        p_list.append(mean)
        if lo <= target <= hi:
            hits += 1
        # phase 2: model and next N_MD
        params = fit_acceptance(nmd_list, p_list)
        nmd = predict_nmd(params, target, multiple)
        if total >= max_total:
            return NmdTuneResult(nmd, "trajectory limit", total, history, params)
        if nmd_list.count(nmd) >= repeat_stop:
            return NmdTuneResult(nmd, "repeated N_MD", total, history, params)
        if hits >= hit_stop:
            return NmdTuneResult(nmd, "target inside interval", total, history, params)
