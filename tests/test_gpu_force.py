"""Parity of the CUDA force and actions (Eqs. p_dot, f_chi_i, def_xi_i; the
Hasenbusch splitting of Section 5.1) with the oracle, and of the autograd
wrapper with finite differences of the GPU action."""
import numpy as np
import pytest

import workloads as W
from oracle import action as oa
from oracle.lattice import Lattice as OLat

from gpu_util import ctx_for, dev, host, need_gpu, rel_max, torch

pytestmark = pytest.mark.gpu


def tight(method=0):
    import paper_1804_07195_gb300 as hmc
    return hmc.SolverOpts(method=method, tol=1e-13, maxit=200000)


@pytest.mark.parametrize("ms", [0.0, 0.5])
def test_single_term_force_matches_dense_oracle(ms):
    need_gpu()
    w = W.workload("L6x6x16")
    ol = OLat.from_params(w.lat)
    ref = oa.grad_pf_action(ol, w.phi, ms, w.b, oa.SolveA(ol, "dense"))
    with ctx_for(w.lat) as ctx:
        # one term (nmass = 0) at mass ms is the chi_n term with mu_{n-1} = ms: use one mass
        # equal to ms with an all-zero lower term switched off via term selection
        if ms == 0.0:
            g, _ = ctx.force(dev(w.phi), [], [dev(w.b)], flags=2, opts=tight())
        else:
            g, _ = ctx.force(dev(w.phi), [ms], [dev(w.b), dev(w.b)], term=1, flags=2, opts=tight())
    assert rel_max(host(g), ref) <= 1e-9


@pytest.mark.parametrize("method", [0, 1])
def test_hasenbusch_chi_action_and_force_12x12(method):
    """12x12, nt=32 with masses (0.3, 1.0): chi creation, S_i and dS/dphi from
    the GPU against the oracle with sparse-LU solves; rel. error <= 1e-7."""
    need_gpu()
    w = W.workload("L12x12x32")
    ol = OLat.from_params(w.lat)
    masses = list(w.masses)
    solve = oa.SolveA(ol, "splu")
    chis_ref = oa.make_chi(ol, w.phi, masses, w.rho, solve)
    phi1 = w.phi + 0.05 * np.random.default_rng(5).normal(size=ol.N)
    with ctx_for(w.lat) as ctx:
        chis, _ = ctx.make_chi(dev(w.phi), masses, [dev(r) for r in w.rho], opts=tight(method))
        for c, cr in zip(chis, chis_ref):
            assert np.linalg.norm(host(c) - cr) <= 1e-9 * np.linalg.norm(cr)
        # at the start field S_i = rho_i^dagger rho_i
        for i in range(3):
            S, _ = ctx.action(dev(w.phi), masses, chis, term=i, flags=2, opts=tight(method))
            rr = float(np.vdot(w.rho[i], w.rho[i]).real)
            assert abs(S - rr) <= 1e-9 * rr
        g, _ = ctx.force(dev(phi1), masses, chis, opts=tight(method))
        S, _ = ctx.action(dev(phi1), masses, chis, opts=tight(method))
    g_ref = oa.total_grad(ol, phi1, masses, chis_ref, solve)
    S_ref = oa.total_action(ol, phi1, masses, chis_ref, solve)
    assert rel_max(host(g), g_ref) <= 1e-7
    assert abs(S - S_ref) <= 1e-10 * abs(S_ref)


def test_autograd_force_vs_finite_differences_12x12():
    """PseudofermionAction: backward equals central finite differences of the
    forward (h = 1e-6) along random directions, rel. error <= 1e-7."""
    need_gpu()
    import paper_1804_07195_gb300 as hmc
    w = W.workload("L12x12x32")
    masses = list(w.masses)
    with ctx_for(w.lat) as ctx:
        phi = dev(w.phi)
        chis, _ = ctx.make_chi(phi, masses, [dev(r) for r in w.rho], opts=tight())
        phi1 = (phi + 0.05 * torch.randn(phi.shape, dtype=torch.float64, device="cuda",
                                         generator=torch.Generator("cuda").manual_seed(1)))
        p = phi1.clone().requires_grad_(True)
        S = hmc.PseudofermionAction.apply(p, ctx, masses, chis, tight(), True)
        S.backward()
        g = p.grad.detach()
        rng = np.random.default_rng(11)
        S0 = S.item()
        eps = np.finfo(np.float64).eps
        for _ in range(3):
            d = rng.normal(size=w.lat.nsites)
            d /= np.linalg.norm(d)
            dd = dev(d)
            an = float((g * dd).sum())
            for h in (1e-6, 1e-4):
                Sp = hmc.PseudofermionAction.apply(phi1 + h * dd, ctx, masses, chis, tight(), True).item()
                Sm = hmc.PseudofermionAction.apply(phi1 - h * dd, ctx, masses, chis, tight(), True).item()
                fd = (Sp - Sm) / (2 * h)
                # central differences carry a rounding error of about eps |S| / h
                # (1.5e-6 here at h = 1e-6, with |S| ~ 3e4) on top of the 1e-7 target
                assert abs(fd - an) <= 1e-7 * max(abs(an), 1.0) + 4 * eps * abs(S0) / h, (h, fd, an)


def test_gaussian_term_only():
    need_gpu()
    w = W.workload("L6x6x16")
    ol = OLat.from_params(w.lat)
    with ctx_for(w.lat) as ctx:
        g, _ = ctx.force(dev(w.phi), [], [], flags=1)
        S, _ = ctx.action(dev(w.phi), [], [], flags=1)
    assert rel_max(host(g), oa.grad_gaussian(ol, w.phi)) <= 1e-15
    assert abs(S - oa.gaussian_action(ol, w.phi)) <= 1e-12 * S


@pytest.mark.slow
def test_force_at_full_size_is_the_action_derivative():
    """102x102x64 with the three Hasenbusch masses, mixed-precision solves at
    1e-13: the force dS/dphi (all terms) agrees with central differences of
    the action along random unit directions, within the rounding of the
    differences plus 1e-6 relative. The rounding allowance is 40 eps |S| / h:
    each action is a sum of 1.3M terms reduced in a tree of depth about 20.
    A property that holds at any size; the oracle cannot form this lattice's
    solves."""
    need_gpu()
    import paper_1804_07195_gb300 as hmc
    w = W.workload("L102x102x64")
    masses = list(w.masses)
    opts = hmc.SolverOpts(method=hmc._abi.HMC_SOLVER_FGMRES_MIXED, tol=1e-13, maxit=200000)
    eps = np.finfo(np.float64).eps
    with ctx_for(w.lat) as ctx:
        phi = dev(w.phi)
        chis, _ = ctx.make_chi(phi, masses, [dev(r) for r in w.rho], opts=opts)
        F, _ = ctx.force(phi, masses, chis, opts=opts)
        S0, _ = ctx.action(phi, masses, chis, opts=opts)
        rng = np.random.default_rng(5)
        for _ in range(2):
            d = rng.normal(size=w.lat.nsites)
            d /= np.linalg.norm(d)
            dd = dev(d)
            an = float((F * dd).sum())
            h = 1e-3
            Sp, _ = ctx.action(phi + h * dd, masses, chis, opts=opts)
            Sm, _ = ctx.action(phi - h * dd, masses, chis, opts=opts)
            fd = (Sp - Sm) / (2 * h)
            assert abs(fd - an) <= 1e-6 * abs(an) + 40 * eps * abs(S0) / h, (fd, an, S0)


@pytest.mark.parametrize("method", [0, 1])
def test_full_size_force_against_closed_form_solves(method):
    """102x102x64 with the three Hasenbusch masses and a constant field
    phi = 0.3, where every solve has the exact free-field form: the oracle's own
    pseudofermions, action and force (Sections 5.1, Eqs. f_chi_i, def_xi_i),
    computed with those exact solves, against the library's, with solves at
    1e-13 (FP64 CG and mixed FGMRES). The heat-bath vectors are random, so the
    force varies from site to site. Each solution is within kappa * 1e-13
    (kappa about 2300 here) of the exact one in norm; the pseudofermions and
    the force, linear and bilinear in the solutions, get a few times that, and
    1e-8 leaves a margin above it. The actions, a sum of 1.3M terms, agree to
    1e-11 relative."""
    need_gpu()
    import paper_1804_07195_gb300 as hmc
    from oracle import free_field
    w = W.workload("L102x102x64")
    ol = OLat.from_params(w.lat)
    theta = 0.3
    masses = list(w.masses)
    phi = np.full(ol.N, theta)

    def exact_solve(p, ms, b):
        assert np.all(p == theta)
        return free_field.solve_A(ol, ms, 0.0, b, theta)

    kappa = max(free_field.condition_number(ol, mu, 0.0, theta) for mu in [0.0] + masses)
    assert kappa < 3000
    chis = oa.make_chi(ol, phi, masses, list(w.rho), exact_solve)
    F_ref = oa.total_grad(ol, phi, masses, chis, exact_solve)
    S_ref = oa.total_action(ol, phi, masses, chis, exact_solve)
    opts = hmc.SolverOpts(method=method, tol=1e-13, maxit=200000)
    with ctx_for(w.lat) as ctx:
        phid = dev(phi)
        gchis, _ = ctx.make_chi(phid, masses, [dev(r) for r in w.rho], opts=opts)
        F, _ = ctx.force(phid, masses, [dev(c) for c in chis], opts=opts)
        S, _ = ctx.action(phid, masses, [dev(c) for c in chis], opts=opts)
    for g, c in zip(gchis, chis):
        assert np.linalg.norm(host(g) - c) <= 1e-8 * np.linalg.norm(c)
    F = host(F)
    assert np.linalg.norm(F - F_ref) <= 1e-8 * np.linalg.norm(F_ref)
    assert rel_max(F, F_ref) <= 1e-8
    assert abs(S - S_ref) <= 1e-11 * abs(S_ref), (S, S_ref)
