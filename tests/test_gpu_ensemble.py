"""The GPU Markov chain samples the HMC weight of Section 2 exactly: on a tiny
lattice (1x1 torus, nt = 4, 8 phi variables) a chain of GPU trajectories with
one Hasenbusch mass (nested Omelyan, Section 5.2) gives <exp(-dH)> = 1 and
reproduces <phi.phi> of exp(-phi^2/(2 delta U)) det(M M^dagger), the latter
computed exactly by reweighting Gaussian samples with the oracle's dense
determinant. The chain uses the mixed-precision solver (FP32 CG inside FP64
FGMRES, Algorithm A.1), the production path; the FP64 path is held to the
oracle trajectory by trajectory elsewhere."""
import numpy as np
import pytest

from exact_ensemble import blocked, phi2_exact
from gpu_util import need_gpu, torch
from oracle.lattice import Lattice as OLat

pytestmark = [pytest.mark.gpu, pytest.mark.slow]


def test_gpu_chain_samples_the_exact_distribution():
    need_gpu()
    import paper_1804_07195_gb300 as hmc
    from paper_1804_07195_gb300 import chain
    lat = hmc.Lattice(1, 1, 4, 1.0, 2.0, 2.0)
    opts = hmc.SolverOpts(method=hmc._abi.HMC_SOLVER_FGMRES_MIXED, tol=1e-12)
    integ = hmc.Integrator(hmc._abi.HMC_INTEG_NESTED_OMELYAN, 4, (2,))
    with hmc.Context(lat) as ctx:
        ch = chain.Chain(ctx, torch.zeros(lat.nsites, dtype=torch.float64, device="cuda"), [0.5], opts, opts,
                         seed=4041)
        meas, expdh = [], []
        for it in range(2100):
            dH, _ = ch.trajectory(integ)
            if it >= 100:
                p = ch.phi.cpu().numpy()
                meas.append(float(p @ p))
                expdh.append(float(np.exp(-dH)))
    hmc_v, hmc_err = blocked(meas)
    eb, eb_err = blocked(expdh)
    assert abs(eb - 1.0) < 5 * eb_err + 1e-3, (eb, eb_err)
    exact, ex_err = phi2_exact(OLat(1, 1, 4, 1.0, 2.0, 2.0), np.random.default_rng(99))
    assert abs(hmc_v - exact) < 4 * np.hypot(hmc_err, ex_err), (hmc_v, hmc_err, exact, ex_err)
