"""The Hasenbusch tuner of Section 7.2 run end to end on the GPU (12x12,
nt=32): solve times for several staggered masses fit Eq. solver_time_eqn with
0 < lambda_min < lambda_max, the two masses sit geometrically between them,
the measured small forces grow with |mu_1 - mu_0|, and the time scales are
positive integers."""
import math

import numpy as np
import pytest

import workloads as W

from gpu_util import ctx_for, dev, need_gpu

pytestmark = pytest.mark.gpu


def test_tuner_end_to_end():
    need_gpu()
    from paper_1804_07195_gb300 import tuner
    w = W.workload("L12x12x32")
    with ctx_for(w.lat) as ctx:
        res = tuner.measure_and_tune(ctx, dev(w.phi), [dev(r) for r in w.rho], repeats=2)
    assert 0 < res.lam_min < res.lam_max
    mu = res.masses
    assert res.lam_min < mu[0] < mu[1] < res.lam_max
    assert math.isclose(mu[1] / mu[0], mu[0] / res.lam_min, rel_tol=1e-9)
    # the pair (0.2, 1.5) is far apart, (0.1, 0.3) close: its force is smaller
    F = dict(zip(map(tuple, res.measurements["pairs"]), res.measurements["F_chi1"]))
    assert F[(0.2, 1.5)] > F[(0.1, 0.3)]
    assert all(np.isfinite(res.small_force)) and all(np.isfinite(res.large_force))
    assert res.N[0] == res.N[1] >= 1


@pytest.mark.parametrize("pair", [(0.1, 0.3), (0.2, 1.5)])
def test_tuner_forces_match_the_oracle(pair):
    """The force vectors behind the tuner's F_chi1 and F_top (tuner.pair_forces,
    the function measure_and_tune calls) at 12x12, nt=32 against the oracle:
    pseudofermions from oracle.action.make_chi, then oracle.action.term_grad of
    the chi_1 term and of the top term plus the Gaussian gradient, all with
    sparse-LU solves; element by element within 1e-7 of the largest entry
    (library solves at 1e-12, FP64-outer mixed FGMRES as in the tuner)."""
    need_gpu()
    import paper_1804_07195_gb300 as hmc
    from paper_1804_07195_gb300 import tuner
    from oracle import action as oa
    from oracle.lattice import Lattice as OLat
    from gpu_util import host, rel_max
    w = W.workload("L12x12x32")
    ol = OLat.from_params(w.lat)
    m0, m1 = pair
    solve = oa.SolveA(ol, "splu")
    chis = oa.make_chi(ol, w.phi, [m0, m1], w.rho, solve)
    F1_ref = oa.term_grad(ol, w.phi, [m0, m1], chis, 1, solve)
    F2_ref = oa.term_grad(ol, w.phi, [m0, m1], chis, 2, solve) + oa.grad_gaussian(ol, w.phi)
    opts = hmc.SolverOpts(method=hmc._abi.HMC_SOLVER_FGMRES_MIXED, tol=1e-12)
    with ctx_for(w.lat) as ctx:
        F1, F2 = tuner.pair_forces(ctx, dev(w.phi), [dev(r) for r in w.rho], m0, m1, opts)
        F1, F2 = host(F1), host(F2)
    assert rel_max(F1, F1_ref) <= 1e-7
    assert rel_max(F2, F2_ref) <= 1e-7
    # and the sizes the tuner fits (root mean square over sites)
    for got, ref in ((F1, F1_ref), (F2, F2_ref)):
        assert abs(np.sqrt(np.mean(got ** 2)) - np.sqrt(np.mean(ref ** 2))) <= 1e-7 * np.sqrt(np.mean(ref ** 2))


def test_nmd_tuner_on_the_four_site_model(paper):
    """Algorithm B.1 driving real trajectories (4-site model, nt = 64, where
    the Omelyan integrator is unstable at N_MD = 8 and stable at 16): the tuned
    N_MD gives a mean acceptance probability near the 0.66 target."""
    need_gpu()
    import paper_1804_07195_gb300 as hmc
    from paper_1804_07195_gb300 import chain, nmd_tuner
    from gpu_util import torch
    lat = hmc.Lattice(2, 1, 64, 1.0, paper["ed_U_over_kappa"], paper["ed_beta_kappa"])
    opts = hmc.SolverOpts(method=hmc._abi.HMC_SOLVER_CG64, tol=1e-12)

    def integ(n):
        return hmc.Integrator(hmc._abi.HMC_INTEG_NESTED_OMELYAN, n, ())

    with hmc.Context(lat) as ctx:
        ch = chain.Chain(ctx, torch.zeros(lat.nsites, dtype=torch.float64, device="cuda"), [], opts, opts,
                         seed=661)
        for _ in range(30):
            ch.trajectory(integ(24))
        res = nmd_tuner.tune_nmd(lambda n: chain.acceptance_probability(ch.trajectory(integ(n))[0]),
                                 nmd0=40, max_total=250)
        acc = [chain.acceptance_probability(ch.trajectory(integ(res.nmd))[0]) for _ in range(100)]
    assert res.total_trajectories <= 250
    assert 8 < res.nmd < 40, res
    assert 0.4 < float(np.mean(acc)) < 0.92, (res.nmd, np.mean(acc), res.history)
