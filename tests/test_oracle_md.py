"""Pins of the oracle's integrators and HMC (Sections 2, 4 and 5.2): the error
norms the paper prints, order of accuracy, reversibility, area preservation,
and the equilibrium distribution of a tiny lattice. CPU only."""
import numpy as np
import pytest
import scipy.linalg as sla

import workloads as W
from oracle import action, integrators
from oracle.lattice import Lattice

from exact_ensemble import blocked, phi2_exact


def harmonic_map(step_fn, h):
    """One-step map of the integrator on H = (phi^2 + pi^2)/2 as a 2x2 matrix
    acting on (phi, pi)."""
    cols = []
    for v in ((1.0, 0.0), (0.0, 1.0)):
        st = integrators.Phase(np.array([v[0]]), np.array([v[1]]))
        step_fn(st, lambda k, p: p.copy(), h)
        cols.append([st.phi[0], st.pi[0]])
    return np.array(cols).T


def third_order_norm(step_fn):
    """|C| of Section 4.1 from the local error S(h) - exp((a+b)h) = C h^3 + O(h^4),
    Richardson-extrapolated; the force-first scheme's C is alpha [b,[b,a]] +
    beta [a,[b,a]] with [b,[b,a]] = [[0,0],[-2,0]] and [a,[b,a]] = [[0,-2],[0,0]]."""
    gen = np.array([[0.0, 1.0], [-1.0, 0.0]])
    D = lambda h: harmonic_map(step_fn, h) - sla.expm(gen * h)
    h = 2e-2
    C = (16 * D(h / 2) - D(h)) / h ** 3
    alpha, beta = -C[1, 0] / 2, -C[0, 1] / 2
    return np.hypot(alpha, beta)


def test_omelyan_and_leapfrog_error_norms(paper):
    z = paper["omelyan_zeta"]
    c_om = third_order_norm(lambda st, g, h: integrators.omelyan(st, g, 1, h, z))
    c_lf = third_order_norm(lambda st, g, h: integrators.omelyan(st, g, 1, h, 0.0))
    assert abs(c_om - paper["omelyan_C_norm"]) < 0.001      # printed as ~0.009
    assert abs(c_lf - paper["leapfrog_C_norm"]) < 0.005     # printed as ~0.09
    assert abs(c_om / c_lf * 4 - paper["omelyan_leapfrog_error_ratio"]) < 0.05


def small_system(shape=(2, 1, 4), seed=3, masses=(0.5,), U=2.0, beta=4.0):
    w = W.small(*shape, seed=seed, masses=masses, U=U, beta=beta)
    lat = Lattice.from_params(w.lat)
    solve = action.SolveA(lat, "dense")
    return w, lat, solve


@pytest.mark.parametrize("integ,order", [("leapfrog", 2), ("omelyan", 2), ("force_gradient", 4)])
def test_order_of_accuracy(integ, order):
    w, lat, solve = small_system(shape=(3, 2, 4))
    dH = []
    for nmd in (8, 16, 32):
        _, _, H0, H1, _ = integrators.trajectory(lat, w.phi * 0.5, w.pi, w.rho, w.masses,
                                                 nmd, (1,), solve, integrator=integ)
        dH.append(abs(H1 - H0))
    r1, r2 = dH[0] / dH[1], dH[1] / dH[2]
    expect = 2 ** order
    assert 0.6 * expect < r2 < 1.5 * expect, (dH, r1, r2)


def test_nested_reversibility_with_odd_ratios():
    masses = (0.3, 1.0)
    w, lat, solve = small_system(shape=(3, 2, 4), masses=masses)
    chis = action.make_chi(lat, w.phi, masses, w.rho, solve)
    forces = integrators.HasenbuschForces(lat, masses, chis, solve)
    steps = integrators.level_steps(6, (3, 1))   # ratios 2 (odd: 3 -> 1) ...
    assert steps == [2, 6, 6]
    st = integrators.Phase(w.phi, w.pi)
    integrators.nested_omelyan(st, forces, steps)
    st.pi = -st.pi
    integrators.nested_omelyan(st, forces, steps)
    assert np.abs(st.phi - w.phi).max() < 1e-11
    assert np.abs(-st.pi - w.pi).max() < 1e-11


def test_half_step_split_weights_and_force_counts():
    """Odd ratios split inner steps in two halves (Section 5.2). Whatever the
    split, every level's kicks add up to the trajectory length, and a level with
    s steps evaluates its force at 2 s + 1 distinct fields (the end kick of one
    step and the first of the next, and the two halves of a split middle kick,
    see the same phi)."""
    weight, evals = {}, {}

    def grad(level, phi):
        evals[level] = evals.get(level, 0) + 1
        return phi

    class Weighing(integrators.Phase):
        def P(self, g, level, c):
            weight[level] = weight.get(level, 0.0) + c
            super().P(g, level, c)

    st = Weighing(np.ones(1), np.zeros(1))
    steps = [5, 15, 15, 30]
    integrators.nested_omelyan(st, grad, steps)
    assert all(abs(weight[k] - 1.0) < 1e-14 for k in range(4))
    assert evals == {k: 2 * s + 1 for k, s in enumerate(steps)}


def test_area_preservation():
    """det of the Jacobian of one trajectory map (phi, pi) -> (phi', pi') is 1."""
    masses = (0.4,)
    w, lat, solve = small_system(shape=(1, 1, 4), masses=masses)
    chis = action.make_chi(lat, w.phi, masses, w.rho, solve)
    forces = integrators.HasenbuschForces(lat, masses, chis, solve)
    N = lat.N

    def flow(z):
        st = integrators.Phase(z[:N], z[N:])
        integrators.nested_omelyan(st, forces, integrators.level_steps(4, (2,)))
        return np.concatenate([st.phi, st.pi])

    z0 = np.concatenate([w.phi, w.pi])
    h = 1e-6
    J = np.empty((2 * N, 2 * N))
    for k in range(2 * N):
        e = np.zeros(2 * N)
        e[k] = h
        J[:, k] = (flow(z0 + e) - flow(z0 - e)) / (2 * h)
    assert abs(np.linalg.det(J) - 1.0) < 1e-6


def test_level_steps_validation():
    assert integrators.level_steps(30, (6, 2, 2)) == [5, 15, 15, 30]
    with pytest.raises(ValueError):
        integrators.level_steps(30, (4,))
    with pytest.raises(ValueError):
        integrators.level_steps(30, (6, 4))


@pytest.mark.slow
def test_hmc_samples_the_exact_distribution():
    """Tiny lattice (1x1 torus, nt=4, 8 phi variables): an HMC chain with one
    Hasenbusch mass must give <exp(-dH)> = 1 and reproduce <phi.phi> of the exact
    weight exp(-phi^2/(2 delta U)) det(M M^dagger), computed here by importance
    sampling from the Gaussian."""
    lat = Lattice(1, 1, 4, 1.0, 2.0, 2.0)
    masses = (0.5,)
    solve = action.SolveA(lat, "dense")
    g = np.random.default_rng(123)
    phi = np.zeros(lat.N)
    meas, expdh = [], []
    for it in range(2600):
        pi = g.normal(size=lat.N)
        rhos = [(g.normal(size=lat.N) + 1j * g.normal(size=lat.N)) * np.sqrt(0.5) for _ in range(2)]
        p1, _, H0, H1, _ = integrators.trajectory(lat, phi, pi, rhos, masses, 4, (2,), solve)
        dH = H1 - H0
        if g.uniform() < np.exp(-dH):
            phi = p1
        if it >= 100:
            meas.append(phi @ phi)
            expdh.append(np.exp(-dH))
    hmc, hmc_err = blocked(meas)
    eb, eb_err = blocked(expdh)
    assert abs(eb - 1.0) < 5 * eb_err + 1e-3
    exact, ex_err = phi2_exact(lat, g)
    assert abs(hmc - exact) < 4 * np.hypot(hmc_err, ex_err), (hmc, hmc_err, exact, ex_err)


@pytest.mark.slow
@pytest.mark.parametrize("shape,seed", [((2, 1, 8), 9), ((3, 3, 4), 10)])
def test_mean_exp_minus_dH_is_one(shape, seed):
    """<exp(-dH)> = 1 over an equilibrium chain (reversible, area-preserving
    MD; Section 2) on the 2x1 and 3x3 tori with one Hasenbusch mass. The step
    size (N_MD = 4, <dH> about 0.08) keeps exp(-dH) well behaved: near the
    integrator's stability limit its distribution is so heavy-tailed that the
    sample mean converges far more slowly than its standard error suggests."""
    lat = Lattice(*shape, 1.0, 2.0, 2.0)
    solve = action.SolveA(lat, "dense")
    g = np.random.default_rng(seed)
    phi = np.zeros(lat.N)
    ex = []
    for it in range(2100):
        pi = g.normal(size=lat.N)
        rhos = [(g.normal(size=lat.N) + 1j * g.normal(size=lat.N)) * np.sqrt(0.5) for _ in range(2)]
        p1, _, H0, H1, _ = integrators.trajectory(lat, phi, pi, rhos, (0.5,), 4, (2,), solve)
        dH = H1 - H0
        if g.uniform() < np.exp(-dH):
            phi = p1
        if it >= 100:
            ex.append(np.exp(-dH))
    mean, err = blocked(ex, 100)
    assert abs(mean - 1.0) < 4 * err + 1e-3, (mean, err)
