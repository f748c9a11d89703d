"""A Markov chain of HMC trajectories (the HMC outline of Section 2) on top of
hmc_md_trajectory: heat-bath momenta pi ~ exp(-pi^2/2) and vectors
rho ~ exp(-rho^dagger rho) drawn on the host from a seeded generator, one
trajectory on the device, and the Metropolis step min(1, exp(-dH)).
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field
from typing import Callable, List, Optional, Sequence

import numpy as np


@dataclass
class ChainResult:
    phi: object
    accepted: int
    trajectories: int
    dH: List[float] = field(default_factory=list)
    measurements: list = field(default_factory=list)

    @property
    def acceptance(self) -> float:
        return self.accepted / max(self.trajectories, 1)


class Chain:
    """One Markov chain: the current field and the generator of its momenta,
    heat-bath vectors and Metropolis draws (in that order per trajectory)."""

    def __init__(self, ctx, phi, masses: Sequence[float], md_opts, action_opts, seed):
        self.ctx = ctx
        self.phi = phi.clone()
        self.masses = list(masses)
        self.md_opts = md_opts
        self.action_opts = action_opts
        self.g = np.random.Generator(np.random.PCG64(np.random.SeedSequence(seed)))

    def trajectory(self, integ):
        """One trajectory with integrator `integ` and the accept/reject step;
        returns (dH, accepted)."""
        import torch
        N = self.ctx.N
        dev = self.phi.device
        g = self.g
        pi = torch.tensor(g.normal(size=N), device=dev)
        rho = [torch.tensor((g.normal(0.0, math.sqrt(0.5), N) + 1j * g.normal(0.0, math.sqrt(0.5), N)),
                            device=dev) for _ in range(len(self.masses) + 1)]
        trial = self.phi.clone()
        H0, H1, _ = self.ctx.md_trajectory(trial, pi, self.masses, rho, integ, self.md_opts, self.action_opts)
        dH = H1 - H0
        accepted = g.uniform() < math.exp(min(0.0, -dH))
        if accepted:
            self.phi = trial
        return dH, accepted


def acceptance_probability(dH: float) -> float:
    """min(1, exp(-dH)), the probability with which a trajectory is accepted."""
    return math.exp(min(0.0, -dH))


def run_chain(ctx, phi, n_traj: int, masses: Sequence[float], integ, md_opts, action_opts, seed,
              therm: int = 0, measure: Optional[Callable] = None, measure_every: int = 1) -> ChainResult:
    """Run therm + n_traj trajectories from phi (a float64 CUDA tensor, not
    modified); `measure(phi)` is called on the current field after each of the
    last n_traj trajectories (every `measure_every`)."""
    chain = Chain(ctx, phi, masses, md_opts, action_opts, seed)
    res = ChainResult(chain.phi, 0, 0)
    for it in range(therm + n_traj):
        dH, accepted = chain.trajectory(integ)
        if it >= therm:
            res.accepted += int(accepted)
            res.trajectories += 1
            res.dH.append(dH)
            if measure is not None and (it - therm) % measure_every == 0:
                res.measurements.append(measure(chain.phi))
    res.phi = chain.phi
    return res
