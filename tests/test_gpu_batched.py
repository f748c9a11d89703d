"""Batched solves of independent systems on uneven lattices (one launch per
kernel over all systems, CUDA-graph replay, convergence masks): every system's
true residual, evaluated by the oracle's operator on its own lattice, meets its
tolerance, in the FP64 and in the mixed-precision mode."""
import numpy as np
import pytest

import workloads as W
from oracle import fermion as of
from oracle import solvers as osv
from oracle.lattice import Lattice as OLat

from gpu_util import ctx_for, dev, host, need_gpu, torch

pytestmark = pytest.mark.gpu


def run_batch(instances, mixed, tol=1e-10):
    import paper_1804_07195_gb300 as hmc
    systems = []
    for w, ms, sigma, b in instances:
        p = w.lat
        systems.append({"lattice": hmc.Lattice(p.n, p.m, p.nt, p.kappa, p.U, p.beta), "phi": dev(w.phi),
                        "ms": ms, "sigma": sigma, "b": dev(b), "x": torch.zeros(p.nsites, dtype=torch.complex128, device="cuda"),
                        "tol": tol, "maxit": 100000})
    with ctx_for(instances[0][0].lat) as ctx:
        infos = ctx.solve_batched(systems, mixed=mixed)
    return [host(s["x"]) for s in systems], infos


def check(instances, xs, infos, tol):
    for (w, ms, sigma, b), x, info in zip(instances, xs, infos):
        ol = OLat.from_params(w.lat)
        rel = osv.true_rel_residual(lambda v: of.apply_MMdag(ol, w.phi, ms, v, sigma), x, b)
        assert rel <= tol * 1.0001, (w.name, ms, sigma, rel, info)
        assert abs(info["true_rel_res"] - rel) <= 1e-3 * tol + 1e-14


def run_batch_variant(instances, mixed, variant, tol=1e-10):
    import paper_1804_07195_gb300 as hmc
    systems = []
    for w, ms, sigma, b in instances:
        p = w.lat
        systems.append({"lattice": hmc.Lattice(p.n, p.m, p.nt, p.kappa, p.U, p.beta), "phi": dev(w.phi),
                        "ms": ms, "sigma": sigma, "b": dev(b), "x": torch.zeros(p.nsites, dtype=torch.complex128, device="cuda"),
                        "tol": tol, "maxit": 100000})
    with ctx_for(instances[0][0].lat) as ctx:
        ctx.set_batched_variant(variant)
        infos = ctx.solve_batched(systems, mixed=mixed)
        used = ctx.batched_variant()
    return [host(s["x"]) for s in systems], infos, used


@pytest.mark.parametrize("variant", [1, 2])
def test_fp32_batched_designs(variant):
    """The two designs of the batched FP32 CG (graph loop of per-iteration
    kernels; one persistent cooperative launch with grid barriers) under FP64
    defect correction: every system's true residual against the oracle."""
    need_gpu()
    shapes = [(1, 1, 2), (3, 3, 8), (6, 6, 16), (2, 5, 4), (12, 12, 16), (4, 3, 10), (18, 18, 32)]
    inst = []
    for k, sh in enumerate(shapes):
        w = W.small(*sh, seed=320 + k, U=3.0, beta=6.0)
        inst.append((w, [0.0, 0.1, 0.5, 2.0][k % 4], [0.0, 0.0, 0.04][k % 3], w.b))
    xs, infos, used = run_batch_variant(inst, 1, variant)
    assert used == variant
    check(inst, xs, infos, 1e-10)


def test_persistent_batched_wait_times_out_and_context_survives():
    """The persistent batched kernel's grid barriers wait a bounded number of
    SM cycles: with the test hook making every barrier wait for one arrival
    that never comes, the solve returns HMC_ERR_TIMEOUT, and after the hook is
    cleared the same context solves correctly."""
    need_gpu()
    import paper_1804_07195_gb300 as hmc
    w = W.small(6, 6, 16, seed=330, U=3.0, beta=6.0)
    p = w.lat
    lat = hmc.Lattice(p.n, p.m, p.nt, p.kappa, p.U, p.beta)
    mk = lambda: [{"lattice": lat, "phi": dev(w.phi), "ms": 0.1, "b": dev(w.b),
                   "x": torch.zeros(p.nsites, dtype=torch.complex128, device="cuda")}]
    with ctx_for(p) as ctx:
        ctx.set_batched_variant(2)
        ctx.set_wait_test(1, 2_000_000)
        with pytest.raises(hmc.HMCError) as e:
            ctx.solve_batched(mk(), mixed=True)
        assert e.value.status == -5
        ctx.set_wait_test(0, 0)
        sy = mk()
        infos = ctx.solve_batched(sy, mixed=True)
    check([(w, 0.1, 0.0, w.b)], [host(sy[0]["x"])], infos, 1e-10)


@pytest.mark.parametrize("mixed", [0, 1])
def test_uneven_small_batch(mixed):
    need_gpu()
    shapes = [(1, 1, 2), (3, 3, 8), (6, 6, 16), (2, 5, 4), (12, 12, 16), (4, 3, 10)]
    inst = []
    for k, sh in enumerate(shapes):
        w = W.small(*sh, seed=300 + k, U=3.0, beta=6.0)
        inst.append((w, [0.0, 0.1, 0.5, 2.0][k % 4], [0.0, 0.0, 0.04][k % 3], w.b))
    xs, infos = run_batch(inst, mixed)
    check(inst, xs, infos, 1e-10)
    if mixed:
        assert all(i["iters_outer"] >= 1 and i["applies32"] > 0 for i in infos)


def test_batched_matches_single_solves():
    """The FP64 batched mode runs the same CG as hmc_solve_cg on each system."""
    need_gpu()
    inst = []
    for k, sh in enumerate([(3, 3, 8), (6, 6, 16)]):
        w = W.small(*sh, seed=400 + k, U=3.0, beta=6.0)
        inst.append((w, 0.1 * k, 0.0, w.b))
    xs, infos = run_batch(inst, 0)
    for (w, ms, sigma, b), x, info in zip(inst, xs, infos):
        with ctx_for(w.lat) as ctx:
            xr, ir = ctx.solve_cg(dev(w.phi), ms, dev(b), tol=1e-10)
        assert abs(info["iters"] - ir["iters"]) <= 1
        assert np.linalg.norm(x - host(xr)) <= 1e-8 * np.linalg.norm(x)


@pytest.mark.parametrize("mixed", [1, 0])
def test_batch_of_48_lattices(mixed):
    """48 instances, L in {6..36}, nt in {16,32,48}, 3 shifts each: 144 systems."""
    need_gpu()
    inst = []
    for w in W.batch_instances():
        for ms, b in zip(w.masses, w.rho):
            inst.append((w, ms, 0.0, b))
    xs, infos = run_batch(inst, mixed)
    # every one of the 144 systems: its true residual evaluated with the
    # oracle's operator on its own lattice, and the library's report of it
    assert len(inst) == 144
    check(inst, xs, infos, 1e-10)
