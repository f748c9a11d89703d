"""Seeded synthetic inputs shared by the oracle, the tests and the benchmark.

This module holds no arithmetic of the method: it only draws random numbers
(numpy PCG64 streams seeded through SeedSequence) and describes lattice sizes
and physical parameters. Both the CPU oracle and the CUDA path receive the
very same arrays from here.

Layout of every space-time array (the canonical layout used throughout):
    idx = ((s * nt + t) * m + j) * n + i,   s in {A=0, B=1}, cell (i, j), time t.

Distributions (Section 2, Eq. (hamiltonian) and the HMC outline):
    phi ~ N(0, delta*U) per site (the Gaussian weight of phi in H),
    pi  ~ N(0, 1)          (weight exp(-pi^2/2)),
    rho, b complex with Re, Im ~ N(0, 1/2) each (weight exp(-rho^dagger rho)).
"""
from __future__ import annotations

from dataclasses import dataclass, field
from typing import List, Optional, Sequence

import numpy as np


@dataclass(frozen=True)
class LatticeParams:
    """An n x m honeycomb torus with nt time slices and couplings kappa, U, beta."""
    n: int
    m: int
    nt: int
    kappa: float = 1.0
    U: float = 2.0
    beta: float = 4.0

    @property
    def delta(self) -> float:
        return self.beta / self.nt

    @property
    def nsites(self) -> int:
        """Number of complex entries of a fermion vector, 2*n*m*nt."""
        return 2 * self.n * self.m * self.nt


def rng(seed) -> np.random.Generator:
    if isinstance(seed, np.random.SeedSequence):
        return np.random.Generator(np.random.PCG64(seed))
    return np.random.Generator(np.random.PCG64(np.random.SeedSequence(seed)))


def draw_phi(g: np.random.Generator, lat: LatticeParams) -> np.ndarray:
    return g.normal(0.0, np.sqrt(lat.delta * lat.U), lat.nsites)


def draw_complex(g: np.random.Generator, nsites: int) -> np.ndarray:
    re = g.normal(0.0, np.sqrt(0.5), nsites)
    im = g.normal(0.0, np.sqrt(0.5), nsites)
    return re + 1j * im


def draw_pi(g: np.random.Generator, nsites: int) -> np.ndarray:
    return g.normal(0.0, 1.0, nsites)


@dataclass
class Workload:
    """One seeded problem instance: field phi, a right-hand side b, momenta pi
    and heat-bath vectors rho (one per pseudofermion term)."""
    name: str
    lat: LatticeParams
    phi: np.ndarray
    b: np.ndarray
    pi: np.ndarray
    rho: List[np.ndarray]
    masses: List[float] = field(default_factory=list)


def make_workload(name: str, lat: LatticeParams, seed, masses: Sequence[float] = (),
                  nrho: Optional[int] = None) -> Workload:
    """Draw phi, b, pi, rho_0..rho_{nrho-1} in that fixed order from one stream."""
    g = rng(seed)
    phi = draw_phi(g, lat)
    b = draw_complex(g, lat.nsites)
    pi = draw_pi(g, lat.nsites)
    if nrho is None:
        nrho = len(masses) + 1
    rho = [draw_complex(g, lat.nsites) for _ in range(nrho)]
    return Workload(name, lat, phi, b, pi, rho, list(masses))


# The workloads: plain FP64 method on 6x6 (nt 16); Hasenbusch force on 12x12
# (nt 32); mixed-precision solve on 36x36 (nt 64); a batch of 48 uneven
# lattices; one trajectory on the 102x102, nt=64 graphene sheet.
L6 = LatticeParams(6, 6, 16, kappa=1.0, U=2.0, beta=4.0)
L12 = LatticeParams(12, 12, 32, kappa=1.0, U=3.0, beta=6.0)
L36 = LatticeParams(36, 36, 64, kappa=1.0, U=3.5, beta=8.0)
L102 = LatticeParams(102, 102, 64, kappa=1.0, U=3.8, beta=12.0)

L12_MASSES = (0.3, 1.0)
BATCH_MASSES = (0.1, 0.5, 2.0)
L102_MASSES = (0.1, 0.5, 2.0)
L102_NMD = 30
L102_NI = (6, 2, 2)
OMELYAN_ZETA = 0.193

SEEDS = {"L6x6x16": 1001, "L12x12x32": 1002, "L36x36x64": 1003, "batch48": 1004, "L102x102x64": 1005}


def workload(name: str) -> Workload:
    """One of the named workloads: "L6x6x16", "L12x12x32" (two Hasenbusch
    masses), "L36x36x64", "L102x102x64" (three masses)."""
    if name == "L6x6x16":
        return make_workload(name, L6, SEEDS[name], ())
    if name == "L12x12x32":
        return make_workload(name, L12, SEEDS[name], L12_MASSES)
    if name == "L36x36x64":
        return make_workload(name, L36, SEEDS[name], ())
    if name == "L102x102x64":
        return make_workload(name, L102, SEEDS[name], L102_MASSES)
    raise KeyError(name)


BATCH_L = (6, 12, 18, 24, 36)
BATCH_NT = (16, 32, 48)


def batch_instances(count: int = 48) -> List[Workload]:
    """The batched workload: `count` independent instances, lattice size L and
    nt drawn per instance, U=3, beta=6, each carrying one b per shift mass."""
    out = []
    for k, child in enumerate(np.random.SeedSequence(SEEDS["batch48"]).spawn(count)):
        g = rng(child)
        L = int(g.choice(BATCH_L))
        nt = int(g.choice(BATCH_NT))
        lat = LatticeParams(L, L, nt, kappa=1.0, U=3.0, beta=6.0)
        phi = draw_phi(g, lat)
        bs = [draw_complex(g, lat.nsites) for _ in BATCH_MASSES]
        out.append(Workload(f"batch[{k}]", lat, phi, bs[0], np.zeros(0), bs, list(BATCH_MASSES)))
    return out


# the batched instances advanced as Markov chains: nested Omelyan, N_MD and
# time-scale ratios for the three masses
BATCH_NMD = 8
BATCH_NI = (2, 1, 1)


def batch_chains(instances: List[Workload]) -> List[tuple]:
    """Momenta and heat-bath vectors for running the batched instances as
    Markov chains: per instance (its lattice and phi), pi ~ N(0,1) and one
    complex Gaussian rho per Hasenbusch term (masses + 1), drawn from a stream
    of their own. Returns [(pi, [rho_0, ..., rho_n]), ...]."""
    out = []
    children = np.random.SeedSequence(SEEDS["batch48"] + 100).spawn(len(instances))
    for w, child in zip(instances, children):
        g = rng(child)
        pi = draw_pi(g, w.lat.nsites)
        rho = [draw_complex(g, w.lat.nsites) for _ in range(len(w.masses) + 1)]
        out.append((pi, rho))
    return out


def small(n, m, nt, seed, kappa=1.0, U=2.0, beta=4.0, masses=()) -> Workload:
    """A small lattice for tests (ragged sizes, n or m down to 1)."""
    lat = LatticeParams(n, m, nt, kappa, U, beta)
    return make_workload(f"L{n}x{m}x{nt}", lat, seed, masses)
