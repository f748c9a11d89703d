"""Independent Markov chains on lattices of uneven sizes advanced in lockstep
(hmc_md_trajectory_batched: every solve of one point of the schedule, one per
chain, as one batched solve). Each chain's trajectory is checked against the
oracle's trajectory on the same seeded inputs (Sections 2, 4, 5.1, 5.2):
|dH_GPU - dH_oracle| <= 1e-8, the final fields within 1e-9 (phi) and 1e-8
(pi), H0 to 1e-9 relative; the mixed-precision batched solves against the
FP64 ones; and the chains against one-at-a-time hmc_md_trajectory."""
import numpy as np
import pytest

import workloads as W
from oracle import action as oa
from oracle import integrators as oi
from oracle.lattice import Lattice as OLat

from gpu_util import dev, host, need_gpu, torch

pytestmark = pytest.mark.gpu

# uneven lattices, n or m of 1 to 3 included (every wrap), odd nt
SHAPES = [(3, 3, 8), (2, 1, 6), (4, 3, 6), (1, 2, 5)]


def opts(method, tol):
    import paper_1804_07195_gb300 as hmc
    return hmc.SolverOpts(method=method, tol=tol, maxit=200000)


def chains_for(masses, seed0=500):
    ws = [W.small(*sh, seed=seed0 + k, masses=masses, U=2.0, beta=4.0) for k, sh in enumerate(SHAPES)]
    for w in ws:
        w.phi0 = w.phi * 0.5
    return ws


def run_batched(ws, masses, integ, md, act):
    import paper_1804_07195_gb300 as hmc
    from paper_1804_07195_gb300 import build
    build.build()
    chains = []
    for w in ws:
        p = w.lat
        chains.append({"lattice": hmc.Lattice(p.n, p.m, p.nt, p.kappa, p.U, p.beta), "phi": dev(w.phi0),
                       "pi": dev(w.pi), "rho": [dev(r) for r in w.rho]})
    p = ws[0].lat
    with hmc.Context(hmc.Lattice(p.n, p.m, p.nt, p.kappa, p.U, p.beta)) as ctx:
        H0, H1, infos = ctx.md_trajectory_batched(chains, list(masses), integ, md, act)
    return chains, H0, H1, infos


@pytest.mark.parametrize("masses,nmd,N,kind", [((0.3, 1.0), 6, (3, 1), 0), ((0.5,), 4, (), 1),
                                               ((0.5,), 3, (), 2)])
def test_batched_chains_match_the_oracle(masses, nmd, N, kind):
    need_gpu()
    import paper_1804_07195_gb300 as hmc
    ws = chains_for(masses)
    integ_name = {0: "nested_omelyan", 1: "leapfrog", 2: "force_gradient"}[kind]
    chains, H0, H1, infos = run_batched(ws, masses, hmc.Integrator(kind, nmd, N), opts(0, 1e-13), opts(0, 1e-13))
    for k, w in enumerate(ws):
        ol = OLat.from_params(w.lat)
        p1, pi1, h0, h1, _ = oi.trajectory(ol, w.phi0, w.pi, w.rho, list(masses), nmd, N, oa.SolveA(ol, "dense"),
                                           integrator=integ_name)
        assert abs(H0[k] - h0) <= 1e-9 * abs(h0), (k, H0[k], h0)
        assert abs((H1[k] - H0[k]) - (h1 - h0)) <= 1e-8, (k, H1[k] - H0[k], h1 - h0)
        assert np.abs(host(chains[k]["phi"]) - p1).max() <= 1e-9, k
        assert np.abs(host(chains[k]["pi"]) - pi1).max() <= 1e-8, k
        assert infos[k]["applies64"] > 0


def test_batched_chains_equal_single_trajectories_and_mixed_solves():
    """The same chains one at a time through hmc_md_trajectory (FP64 CG at
    1e-13) agree with the batched run; with mixed-precision batched solves at
    1e-12 the energy changes stay within 1e-7 of the FP64 ones."""
    need_gpu()
    import paper_1804_07195_gb300 as hmc
    masses = (0.3, 1.0)
    integ = hmc.Integrator(0, 6, (3, 1))
    ws = chains_for(masses, seed0=600)
    chains, H0, H1, _ = run_batched(ws, masses, integ, opts(0, 1e-13), opts(0, 1e-13))
    for k, w in enumerate(ws):
        p = w.lat
        with hmc.Context(hmc.Lattice(p.n, p.m, p.nt, p.kappa, p.U, p.beta)) as ctx:
            phi, pi = dev(w.phi0), dev(w.pi)
            g0, g1, _ = ctx.md_trajectory(phi, pi, list(masses), [dev(r) for r in w.rho], integ, opts(0, 1e-13),
                                          opts(0, 1e-13))
        assert abs((g1 - g0) - (H1[k] - H0[k])) <= 1e-9
        assert np.abs(host(phi) - host(chains[k]["phi"])).max() <= 1e-10
    chains_m, H0m, H1m, infos = run_batched(ws, masses, integ, opts(1, 1e-12), opts(1, 1e-12))
    for k in range(len(ws)):
        assert abs((H1m[k] - H0m[k]) - (H1[k] - H0[k])) <= 1e-7
        assert infos[k]["applies32"] > 0


def test_batched_trajectory_rejects_bad_chains():
    need_gpu()
    import paper_1804_07195_gb300 as hmc
    ws = chains_for((0.3,), seed0=700)
    with pytest.raises(hmc.HMCError):
        run_batched(ws, (0.3,), hmc.Integrator(0, 5, (2,)), opts(0, 1e-10), opts(0, 1e-10))  # 2 does not divide 5


def test_batched_trajectory_reports_which_chain_is_invalid():
    """A mass with 1 - delta mu = 0 on one chain's lattice (nt = 4, beta = 4,
    mu = 1: the time hop vanishes) is rejected, and the message names the chain."""
    need_gpu()
    import paper_1804_07195_gb300 as hmc
    ws = chains_for((1.0,), seed0=710)
    ws[1] = W.small(2, 1, 4, seed=711, masses=(1.0,), U=2.0, beta=4.0)
    ws[1].phi0 = ws[1].phi * 0.5
    with pytest.raises(hmc.HMCError) as e:
        run_batched(ws, (1.0,), hmc.Integrator(0, 4, (2,)), opts(0, 1e-10), opts(0, 1e-10))
    assert e.value.status == -1 and "chain 1" in str(e.value)
