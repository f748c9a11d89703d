"""Failure detection, with every fault made on the host: a NaN planted in the
field or the right-hand side, an iteration limit that is too small, invalid
arguments and descriptors. Each must come back as a status, never as a fault,
a hang or an abort, and the context must stay usable afterwards."""
import numpy as np
import pytest

import workloads as W

from gpu_util import ctx_for, dev, host, need_gpu, torch

pytestmark = pytest.mark.gpu


def test_nan_in_field_is_reported_and_context_survives():
    need_gpu()
    import paper_1804_07195_gb300 as hmc
    w = W.workload("L6x6x16")
    bad = w.phi.copy()
    bad[17] = np.nan
    with ctx_for(w.lat) as ctx:
        for solve in (lambda p: ctx.solve_cg(p, 0.0, dev(w.b), tol=1e-10),
                      lambda p: ctx.solve_fgmres(p, 0.0, dev(w.b), tol=1e-10)):
            with pytest.raises(hmc.HMCError) as e:
                solve(dev(bad))
            assert e.value.status == -4  # HMC_ERR_NAN
        # the same context still solves a good system
        x, info = ctx.solve_cg(dev(w.phi), 0.0, dev(w.b), tol=1e-10)
        assert info["true_rel_res"] <= 1e-10


def test_nan_in_rhs_is_reported():
    need_gpu()
    import paper_1804_07195_gb300 as hmc
    w = W.workload("L6x6x16")
    b = w.b.copy()
    b[3] = complex(np.nan, 0.0)
    with ctx_for(w.lat) as ctx:
        with pytest.raises(hmc.HMCError) as e:
            ctx.solve_fgmres(dev(w.phi), 0.0, dev(b), tol=1e-10)
        assert e.value.status == -4


def test_spcg_iteration_limit():
    need_gpu()
    import paper_1804_07195_gb300 as hmc
    w = W.workload("L6x6x16")
    with ctx_for(w.lat) as ctx:
        with pytest.raises(hmc.HMCError) as e:
            ctx.solve_spcg(dev(w.phi), 0.0, dev(w.b.astype(np.complex64)), tol=1e-7, maxit=3)
        assert e.value.status == -3
        _, info = ctx.solve_spcg(dev(w.phi), 0.0, dev(w.b.astype(np.complex64)), tol=1e-7, maxit=3,
                                 allow_fail=True)
        assert info["iters"] == 3


def test_invalid_arguments():
    need_gpu()
    import paper_1804_07195_gb300 as hmc
    w = W.small(3, 3, 4, seed=2)
    with ctx_for(w.lat) as ctx:
        phi, b = dev(w.phi), dev(w.b)
        with pytest.raises(hmc.HMCError):
            ctx.solve_cg(phi, 0.0, b, tol=-1.0)
        with pytest.raises(hmc.HMCError):
            ctx.solve_cg(phi, 0.0, b, maxit=0)
        with pytest.raises(hmc.HMCError):
            ctx.solve_fgmres(phi, 0.0, b, restart=0)
        with pytest.raises(hmc.HMCError):
            ctx.solve_fgmres(phi, 0.0, b, inner_prec=16)
        with pytest.raises(hmc.HMCError):
            ctx.force(phi, [0.1] * 9, [b] * 10)  # more masses than supported
        with pytest.raises(hmc.HMCError):
            ctx.md_trajectory(phi.clone(), dev(w.pi), [0.2], [b, b], hmc.Integrator(0, 5, (2,)),
                              hmc.SolverOpts(), hmc.SolverOpts())  # N_0 does not divide N_MD
        with pytest.raises(ValueError):
            ctx.apply_M(phi, 0.0, b[:-1])  # wrong length is caught in the binding


def test_partially_overlapping_vectors_are_rejected():
    """in/out (and b/x) ranges that share some entries, not only identical
    pointers, are rejected with HMC_ERR_INVALID before any launch; disjoint
    parts of one buffer are accepted."""
    need_gpu()
    import paper_1804_07195_gb300 as hmc
    w = W.small(3, 3, 4, seed=3)
    N = w.lat.nsites
    with ctx_for(w.lat) as ctx:
        phi = dev(w.phi)
        for dt in (torch.complex128, torch.complex64):
            buf = torch.zeros(2 * N, dtype=dt, device="cuda")
            buf[:N] = dev(w.b).to(dt)
            for shift in (1, N // 2, N - 1):
                for fn in (ctx.apply_M, ctx.apply_Mdag, ctx.apply_MMdag):
                    with pytest.raises(hmc.HMCError) as e:
                        fn(phi, 0.0, buf[:N], out=buf[shift:shift + N])
                    assert e.value.status == -1
            ctx.apply_MMdag(phi, 0.0, buf[:N], out=buf[N:])  # disjoint: fine
        buf = torch.zeros(2 * N, dtype=torch.complex128, device="cuda")
        buf[:N] = dev(w.b)
        with pytest.raises(hmc.HMCError) as e:
            ctx.solve_cg(phi, 0.0, buf[:N], x=buf[3:3 + N])
        assert e.value.status == -1
        torch.cuda.synchronize()


def test_bad_batched_descriptor():
    need_gpu()
    import paper_1804_07195_gb300 as hmc
    w = W.small(3, 3, 4, seed=2)
    lat = hmc.Lattice(3, 3, 4, 1.0, 2.0, 4.0)
    good = {"lattice": lat, "phi": dev(w.phi), "ms": 0.0, "b": dev(w.b),
            "x": torch.zeros(lat.nsites, dtype=torch.complex128, device="cuda")}
    with ctx_for(w.lat) as ctx:
        bad = dict(good, sigma=-1.0)
        with pytest.raises(hmc.HMCError):
            ctx.solve_batched([good, bad])
        bad = dict(good, tol=0.0)
        with pytest.raises(hmc.HMCError):
            ctx.solve_batched([bad])
        infos = ctx.solve_batched([good])
        assert infos[0]["true_rel_res"] <= 1e-10


def test_bounded_grid_barrier_wait_times_out_and_context_survives():
    """The persistent FP32 CG kernel's grid barriers wait a bounded number of SM
    cycles: with the test hook making every barrier wait for one arrival that
    never comes, the solve returns HMC_ERR_TIMEOUT after about a millisecond,
    and the same context then solves normally, agreeing with the two-kernel
    CG (both meet the tolerance up to FP32 rounding drift)."""
    need_gpu()
    import time
    import paper_1804_07195_gb300 as hmc
    w = W.workload("L6x6x16")
    b32 = dev(w.b.astype(np.complex64))
    with ctx_for(w.lat) as ref:
        ref.set_cg_variant(1)
        x_ref, _ = ref.solve_spcg(dev(w.phi), 0.3, b32, tol=1e-6)
    with ctx_for(w.lat) as ctx:
        ctx.set_cg_variant(4)
        ctx.set_wait_test(1, 2_000_000)
        t = time.perf_counter()
        with pytest.raises(hmc.HMCError) as e:
            ctx.solve_spcg(dev(w.phi), 0.3, b32, tol=1e-6)
        assert e.value.status == hmc._abi.HMC_ERR_TIMEOUT
        assert time.perf_counter() - t < 30.0
        ctx.set_wait_test(0, 0)
        x, info = ctx.solve_spcg(dev(w.phi), 0.3, b32, tol=1e-6)
        assert info["status"] == 0
        assert ctx.profile_read()["cg_persist_f32"]["launches"] == 2
    from oracle import fermion as of
    from oracle.lattice import Lattice as OLat
    ol = OLat.from_params(w.lat)
    b = w.b.astype(np.complex64).astype(np.complex128)
    for xs in (host(x_ref), host(x)):
        r = b - of.apply_MMdag(ol, w.phi, 0.3, xs.astype(np.complex128))
        assert np.linalg.norm(r) <= 1e-4 * np.linalg.norm(b)


def test_guard_bands_stay_intact_and_a_write_past_a_buffer_is_reported():
    """Every device buffer of a context carries guard bands; after operator
    applications in both designs, CG, mixed FGMRES and fCG solves, forces, a
    trajectory and a batched solve, no band has changed. A byte written just
    past the end of the phase table (the test hook, a plain memset inside the
    allocation) is reported."""
    need_gpu()
    import paper_1804_07195_gb300 as hmc
    w = W.small(12, 12, 16, seed=41, masses=(0.3, 1.0), U=3.0, beta=6.0)
    with ctx_for(w.lat) as ctx:
        phi, b = dev(w.phi), dev(w.b)
        for v in (1, 2):
            ctx.set_apply_variant(v)
            ctx.apply_MMdag(phi, 0.1, b)
            ctx.apply_MMdag(phi, 0.1, b.to(torch.complex64))
        ctx.apply_M(phi, 0.1, b)
        ctx.apply_Mdag(phi, 0.1, b.to(torch.complex64))
        ctx.solve_cg(phi, 0.0, b)
        ctx.solve_fgmres(phi, 0.2, b)
        ctx.solve_fcg(phi, 0.2, b)
        opts = hmc.SolverOpts(tol=1e-10)
        chis, _ = ctx.make_chi(phi, [0.3, 1.0], [dev(r) for r in w.rho], opts=opts)
        ctx.force(phi, [0.3, 1.0], chis, opts=opts)
        ctx.md_trajectory(phi.clone(), dev(w.pi), [0.3, 1.0], [dev(r) for r in w.rho], hmc.Integrator(0, 4, (2, 1)),
                          opts, opts)
        lat = hmc.Lattice(w.lat.n, w.lat.m, w.lat.nt, w.lat.kappa, w.lat.U, w.lat.beta)
        ctx.solve_batched([{"lattice": lat, "phi": phi, "ms": 0.1, "b": b, "x": torch.zeros_like(b)}], mixed=True)
        assert ctx.check_guards() == 0
        assert ctx.lib.hmc_guard_test_write(ctx.h) == 0
        assert ctx.check_guards() == 1
        assert b"workspace slot 0 (after its end)" in ctx.lib.hmc_last_error(ctx.h)
