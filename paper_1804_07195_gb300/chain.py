"""A Markov chain of HMC trajectories (the HMC outline of Section 2) on top of
hmc_md_trajectory: heat-bath momenta pi ~ exp(-pi^2/2) and vectors
rho ~ exp(-rho^dagger rho) drawn on the host from a seeded generator, one
trajectory on the device, and the Metropolis step min(1, exp(-dH)).
"""
from __future__ import annotations

import json
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
    heat-bath vectors and Metropolis draws (in that order per trajectory).

    `log`: a file that receives one JSON line per trajectory (its number, H0,
    H1, dH, the Metropolis decision and the solver statistics the library
    reports). `save` writes a checkpoint (field, generator state, counters);
    `Chain.load` resumes from it, and the resumed chain continues exactly as the
    uninterrupted one would."""

    def __init__(self, ctx, phi, masses: Sequence[float], md_opts, action_opts, seed,
                 log: Optional[str] = None):
        self.ctx = ctx
        self.phi = phi.clone()
        self.masses = list(masses)
        self.md_opts = md_opts
        self.action_opts = action_opts
        self.g = np.random.Generator(np.random.PCG64(np.random.SeedSequence(seed)))
        self.log = log
        self.trajectories = 0
        self.accepted = 0

    def save(self, path: str) -> None:
        """Checkpoint: the current field, the generator state, the masses and
        the trajectory and acceptance counters (numpy .npz)."""
        np.savez(path, phi=self.phi.detach().cpu().numpy(), masses=np.array(self.masses, dtype=np.float64),
                 rng_state=np.array(json.dumps(self.g.bit_generator.state)),
                 counters=np.array([self.trajectories, self.accepted], dtype=np.int64))

    @classmethod
    def load(cls, ctx, path: str, md_opts, action_opts, device="cuda", log: Optional[str] = None) -> "Chain":
        """Resume a chain from a checkpoint written by `save`."""
        import torch
        with np.load(path) as z:
            phi = torch.tensor(z["phi"], device=device)
            ch = cls(ctx, phi, [float(v) for v in z["masses"]], md_opts, action_opts, seed=0, log=log)
            ch.g.bit_generator.state = json.loads(str(z["rng_state"]))
            ch.trajectories, ch.accepted = (int(v) for v in z["counters"])
        return ch

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
        H0, H1, info = self.ctx.md_trajectory(trial, pi, self.masses, rho, integ, self.md_opts, self.action_opts)
        dH = H1 - H0
        accepted = g.uniform() < math.exp(min(0.0, -dH))
        if accepted:
            self.phi = trial
        self.trajectories += 1
        self.accepted += int(accepted)
        if self.log is not None:
            with open(self.log, "a") as f:
                f.write(json.dumps({"trajectory": self.trajectories, "H0": H0, "H1": H1, "dH": dH,
                                    "accepted": bool(accepted), "solver": dict(info or {})}) + "\n")
        return dH, accepted


def acceptance_probability(dH: float) -> float:
    """min(1, exp(-dH)), the probability with which a trajectory is accepted."""
    return math.exp(min(0.0, -dH))


def run_chain(ctx, phi, n_traj: int, masses: Sequence[float], integ, md_opts, action_opts, seed,
              therm: int = 0, measure: Optional[Callable] = None, measure_every: int = 1,
              log: Optional[str] = None) -> ChainResult:
    """Run therm + n_traj trajectories from phi (a float64 CUDA tensor, not
    modified); `measure(phi)` is called on the current field after each of the
    last n_traj trajectories (every `measure_every`); `log` as for Chain."""
    chain = Chain(ctx, phi, masses, md_opts, action_opts, seed, log=log)
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
