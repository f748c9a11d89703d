"""The seeded input recipe: lattice sizes and couplings of each workload, the
fixed draw order from one PCG64 stream, the stated distributions (phi ~
N(0, delta U), pi ~ N(0, 1), b and rho complex with E|.|^2 = 1), and the
batch of 48 uneven lattices. CPU only."""
import numpy as np

import workloads as W


def test_workload_parameters():
    expect = {"L6x6x16": ((6, 6, 16), 2.0, 4.0, ()), "L12x12x32": ((12, 12, 32), 3.0, 6.0, (0.3, 1.0)),
              "L36x36x64": ((36, 36, 64), 3.5, 8.0, ()),
              "L102x102x64": ((102, 102, 64), 3.8, 12.0, (0.1, 0.5, 2.0))}
    for name, (shape, U, beta, masses) in expect.items():
        w = W.workload(name)
        p = w.lat
        assert (p.n, p.m, p.nt) == shape and p.kappa == 1.0 and p.U == U and p.beta == beta
        assert tuple(w.masses) == masses and len(w.rho) == len(masses) + 1
        assert w.phi.shape == w.pi.shape == (p.nsites,) and w.b.shape == (p.nsites,)
    assert W.workload("L102x102x64").lat.nsites == 1331712
    assert (W.L102_NMD, W.L102_NI) == (30, (6, 2, 2))


def test_draw_order_and_reproducibility():
    """phi, b, pi, rho_0..rho_n in that order from the stream seeded by the
    workload's seed; the same seed gives the same arrays."""
    w = W.workload("L12x12x32")
    p = w.lat
    g = np.random.Generator(np.random.PCG64(np.random.SeedSequence(W.SEEDS["L12x12x32"])))
    phi = g.normal(0.0, np.sqrt(p.delta * p.U), p.nsites)
    b = g.normal(0.0, np.sqrt(0.5), p.nsites) + 1j * g.normal(0.0, np.sqrt(0.5), p.nsites)
    pi = g.normal(0.0, 1.0, p.nsites)
    assert np.array_equal(w.phi, phi) and np.array_equal(w.b, b) and np.array_equal(w.pi, pi)
    r0 = g.normal(0.0, np.sqrt(0.5), p.nsites) + 1j * g.normal(0.0, np.sqrt(0.5), p.nsites)
    assert np.array_equal(w.rho[0], r0)
    w2 = W.workload("L12x12x32")
    assert all(np.array_equal(a, c) for a, c in zip(w.rho, w2.rho))


def test_distributions_at_full_size():
    w = W.workload("L102x102x64")
    p = w.lat
    N = p.nsites
    tol = 5 / np.sqrt(N)
    assert abs(w.phi.var() / (p.delta * p.U) - 1) < 2 * tol and abs(w.phi.mean()) < tol
    assert abs(w.pi.var() - 1) < 2 * tol
    for v in [w.b] + w.rho:
        assert abs(np.mean(np.abs(v) ** 2) - 1) < 2 * tol
        assert abs(v.real.var() - 0.5) < tol and abs(v.imag.var() - 0.5) < tol


def test_batch_of_48_uneven_lattices():
    inst = W.batch_instances()
    assert len(inst) == 48
    shapes = {(w.lat.n, w.lat.nt) for w in inst}
    assert len(shapes) > 5  # uneven
    for w in inst:
        assert w.lat.n == w.lat.m and w.lat.n in W.BATCH_L and w.lat.nt in W.BATCH_NT
        assert (w.lat.U, w.lat.beta) == (3.0, 6.0) and tuple(w.masses) == W.BATCH_MASSES
        assert len(w.rho) == 3 and all(r.shape == (w.lat.nsites,) for r in w.rho)
    sizes = [w.lat.nsites for w in inst]
    assert (min(sizes), max(sizes)) == (1152, 124416)
    assert sum(w.lat.nsites * len(w.rho) for w in inst) == 5474304  # 144 systems
    again = W.batch_instances()
    assert all(np.array_equal(a.phi, c.phi) for a, c in zip(inst, again))
