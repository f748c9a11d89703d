"""The resident-tile FP32 CG (variant 7: one cooperative launch per solve, p
and u = M^dagger p of every block's tile in shared memory, the neighbouring
tiles' edge rows and slices exchanged through memory between grid barriers)
against the oracle's textbook CG (Section 3), with one cell per thread (odd
n) and two (even n): the same CG step, so x after k
iterations matches the oracle's FP64 CG after k iterations to FP32
rounding, on lattices with n or m of 1 to 3 (every wrap: a tile's padding
row or slice is its own cells), odd nt (uneven tiles), sigma != 0, and the
102x102x64 benchmark lattice (136 tiles of 102 x 6 x 8 cells); a wrong
padding cell, sign or parity of the exchanged edges moves x_2 far outside
that bound. Also: a converged solve stops where the oracle's CG stops, and a
barrier wait that runs out returns HMC_ERR_TIMEOUT with the context usable."""
import numpy as np
import pytest

import workloads as W
from oracle import fermion as of
from oracle import solvers as osv
from oracle.lattice import Lattice as OLat

from gpu_util import ctx_for, dev, host, need_gpu, rel_max, torch

pytestmark = pytest.mark.gpu

SHAPES = [(1, 1, 4), (2, 1, 4), (1, 3, 5), (3, 3, 8), (2, 5, 3), (6, 6, 16), (7, 5, 9), (12, 12, 32),
          (35, 12, 21)]


@pytest.mark.parametrize("shape", SHAPES)
@pytest.mark.parametrize("ms,sigma", [(0.3, 0.0), (0.1, 0.2)])
def test_resident_iterates_equal_cg(shape, ms, sigma):
    need_gpu()
    w = W.small(*shape, seed=1600 + sum(shape))
    ol = OLat.from_params(w.lat)
    A = lambda v: of.apply_MMdag(ol, w.phi, ms, v, sigma)
    b32 = w.b.astype(np.complex64)
    kmax = max(1, min(5, w.lat.nsites // 4))
    with ctx_for(w.lat) as ctx:
        ctx.set_cg_variant(7)
        for k in sorted({1, 2, kmax}):
            x, info = ctx.solve_spcg(dev(w.phi), ms, dev(b32), sigma=sigma, tol=1e-30, maxit=k, allow_fail=True)
            assert info["iters"] == k, (shape, k, info)
            ref = osv.cg(A, b32.astype(np.complex128), tol=1e-30, maxit=k)
            assert rel_max(host(x).astype(np.complex128), ref.x) <= 2e-5 * k, (shape, k)
        st = ctx.profile_read()["cg_resident_f32"]
        assert st["launches"] >= 2
        # two cells per thread (16-byte pairs) where n is even
        assert st["design"] == (4 if shape[0] % 2 == 0 else 0)
        # the roofline's algorithmic bytes: 96 B per site for exactly the
        # iterations that ran, whatever the launches
        assert st["bytes"] == 96.0 * w.lat.nsites * sum(sorted({1, 2, kmax}))


def test_resident_iterates_at_full_size():
    """102x102x64: x after 3 iterations against the oracle's CG (the oracle's
    operator on 1.3M sites takes a few seconds per application)."""
    need_gpu()
    w = W.workload("L102x102x64")
    ol = OLat.from_params(w.lat)
    b32 = w.b.astype(np.complex64)
    with ctx_for(w.lat) as ctx:
        ctx.set_cg_variant(7)
        x, info = ctx.solve_spcg(dev(w.phi), 0.1, dev(b32), tol=1e-30, maxit=3, allow_fail=True)
        st = ctx.profile_read()["cg_resident_f32"]
        assert st["launches"] >= 1 and st["bytes"] == 96.0 * w.lat.nsites * 3
    ref = osv.cg(lambda v: of.apply_MMdag(ol, w.phi, 0.1, v), b32.astype(np.complex128), tol=1e-30, maxit=3)
    assert info["iters"] == 3
    assert rel_max(host(x).astype(np.complex128), ref.x) <= 1e-4


def test_resident_stops_where_cg_stops():
    need_gpu()
    w = W.workload("L36x36x64")
    ol = OLat.from_params(w.lat)
    A = lambda v: of.apply_MMdag(ol, w.phi, 0.4, v, 0.05)
    b32 = w.b.astype(np.complex64).astype(np.complex128)
    ref = osv.cg(A, b32, tol=1e-5, maxit=5000)
    with ctx_for(w.lat) as ctx:
        ctx.set_cg_variant(7)
        x, info = ctx.solve_spcg(dev(w.phi), 0.4, dev(w.b.astype(np.complex64)), sigma=0.05, tol=1e-5, maxit=5000)
        assert ctx.profile_read()["cg_resident_f32"]["launches"] >= 1
    assert abs(info["iters"] - ref.iters) <= 1
    r = b32 - A(host(x).astype(np.complex128))
    assert np.linalg.norm(r) / np.linalg.norm(b32) <= 5e-5


def test_resident_barrier_wait_times_out_and_context_survives():
    need_gpu()
    import time
    import paper_1804_07195_gb300 as hmc
    w = W.workload("L6x6x16")
    b32 = dev(w.b.astype(np.complex64))
    with ctx_for(w.lat) as ctx:
        ctx.set_cg_variant(7)
        ctx.set_wait_test(1, 2_000_000)
        t = time.perf_counter()
        with pytest.raises(hmc.HMCError) as e:
            ctx.solve_spcg(dev(w.phi), 0.3, b32, tol=1e-6)
        assert e.value.status == hmc._abi.HMC_ERR_TIMEOUT
        assert time.perf_counter() - t < 30.0
        ctx.set_wait_test(0, 0)
        x, info = ctx.solve_spcg(dev(w.phi), 0.3, b32, tol=1e-6)
        assert info["status"] == 0
    ol = OLat.from_params(w.lat)
    b = w.b.astype(np.complex64).astype(np.complex128)
    r = b - of.apply_MMdag(ol, w.phi, 0.3, host(x).astype(np.complex128))
    assert np.linalg.norm(r) <= 1e-4 * np.linalg.norm(b)


def test_resident_falls_back_where_its_tiles_do_not_fit():
    """n = 2101 (odd, more cells per row than a block has threads): variant 7
    runs the grid-stride pair instead, and the solve still meets the oracle's
    CG iterates."""
    need_gpu()
    w = W.small(2101, 1, 4, seed=1620)
    ol = OLat.from_params(w.lat)
    b32 = w.b.astype(np.complex64)
    with ctx_for(w.lat) as ctx:
        ctx.set_cg_variant(7)
        x, info = ctx.solve_spcg(dev(w.phi), 0.3, dev(b32), tol=1e-30, maxit=3, allow_fail=True)
        assert ctx.profile_read()["cg_resident_f32"]["launches"] == 0
    ref = osv.cg(lambda v: of.apply_MMdag(ol, w.phi, 0.3, v), b32.astype(np.complex128), tol=1e-30, maxit=3)
    assert info["iters"] == 3
    assert rel_max(host(x).astype(np.complex128), ref.x) <= 1e-4


def test_resident_with_an_unaligned_solution_vector():
    """A caller's x that is 8- but not 16-byte aligned: the same iterates as an
    aligned x (the two-cell kernel needs 16-byte vectors; the library solves
    in a workspace vector or takes the one-cell kernel)."""
    need_gpu()
    import ctypes as C
    from paper_1804_07195_gb300 import _abi
    w = W.small(12, 12, 32, seed=1630, U=3.0, beta=6.0)
    N = w.lat.nsites
    b32 = dev(w.b.astype(np.complex64))
    with ctx_for(w.lat) as ctx:
        ctx.set_cg_variant(7)
        xa, ia = ctx.solve_spcg(dev(w.phi), 0.1, b32, tol=1e-5, maxit=5000)
        buf = torch.zeros(N + 1, dtype=torch.complex64, device="cuda")
        info = _abi.hmc_solve_info()
        st = ctx.lib.hmc_solve_spcg(ctx.h, C.c_void_p(dev(w.phi).data_ptr()), 0.1, 0.0, C.c_void_p(b32.data_ptr()),
                                    C.c_void_p(buf[1:].data_ptr()), 1e-5, 5000, C.byref(info))
        torch.cuda.synchronize()
        assert st == 0 and ctx.profile_read()["cg_resident_f32"]["launches"] >= 2
    assert abs(info.iters - ia["iters"]) <= 1
    assert rel_max(host(buf[1:]).astype(np.complex128), host(xa).astype(np.complex128)) <= 1e-5
