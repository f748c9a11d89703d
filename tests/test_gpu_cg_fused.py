"""The single-reduction FP32 CG (variant 6: one fused kernel and one grid-wide
reduction per iteration) against the oracle's textbook CG (Section 3): in
exact arithmetic the single-reduction recurrences (Chronopoulos and Gear)
produce the same iterates x_k as CG, so x after k iterations must match the
oracle's FP64 CG after k iterations to FP32 rounding; on lattices with n or
m of 1 to 3 (every wrap), odd nt, sigma != 0 and pinned tiles that leave
ragged tails in i, j and t; a wrong sign, index or term in any recurrence
(alpha, beta, s, w, p, x, r) moves x_2 far outside that bound. Solves to the
FP32 floor and mixed FGMRES on top are in test_gpu_solvers.py."""
import numpy as np
import pytest

import workloads as W
from oracle import fermion as of
from oracle import solvers as osv
from oracle.lattice import Lattice as OLat

from gpu_util import ctx_for, dev, host, need_gpu, rel_max, torch

pytestmark = pytest.mark.gpu

SHAPES = [(1, 1, 4), (2, 1, 4), (1, 3, 5), (3, 3, 8), (2, 5, 3), (6, 6, 16), (7, 5, 9), (12, 12, 32)]
# (Ti, Tj, Tt, depth): default-like, ragged in every direction, the smallest
# tile, the deep ring
TILES = [None, (30, 8, 16, 2), (5, 3, 7, 2), (1, 1, 1, 6), (14, 6, 5, 6), (4, 4, 2, 2)]


def k_iterates(ctx, w, ms, sigma, k):
    b32 = dev(w.b.astype(np.complex64))
    x, info = ctx.solve_spcg(dev(w.phi), ms, b32, sigma=sigma, tol=1e-30, maxit=k, allow_fail=True)
    return host(x).astype(np.complex128), info


@pytest.mark.parametrize("shape", SHAPES)
@pytest.mark.parametrize("ms,sigma", [(0.3, 0.0), (0.1, 0.2)])
def test_single_reduction_iterates_equal_cg(shape, ms, sigma):
    need_gpu()
    w = W.small(*shape, seed=1500 + sum(shape))
    ol = OLat.from_params(w.lat)
    A = lambda v: of.apply_MMdag(ol, w.phi, ms, v, sigma)
    b32 = w.b.astype(np.complex64).astype(np.complex128)
    kmax = max(1, min(5, w.lat.nsites // 4))
    for tile in TILES:
        with ctx_for(w.lat) as ctx:
            ctx.set_cg_variant(6)
            if tile is not None:
                ctx.set_cg_fused_tile(*tile)
            for k in sorted({1, 2, kmax}):
                x, info = k_iterates(ctx, w, ms, sigma, k)
                assert ctx.cg_fused_tile()[4] == 1
                assert info["iters"] == k, (shape, tile, k, info)
                ref = osv.cg(A, b32, tol=1e-30, maxit=k)
                assert ref.iters == k
                assert rel_max(x, ref.x) <= 2e-5 * k, (shape, tile, k)


def test_single_reduction_stops_where_cg_stops():
    """Converged solves: the recursive residual test ends the solve at the
    same iteration as the oracle's CG (up to one step of FP32 rounding), and
    the solution's true residual meets the tolerance plus the rounding drift."""
    need_gpu()
    w = W.workload("L36x36x64")
    ol = OLat.from_params(w.lat)
    A = lambda v: of.apply_MMdag(ol, w.phi, 0.4, v, 0.05)
    b32 = w.b.astype(np.complex64).astype(np.complex128)
    ref = osv.cg(A, b32, tol=1e-5, maxit=5000)
    with ctx_for(w.lat) as ctx:
        ctx.set_cg_variant(6)
        x, info = ctx.solve_spcg(dev(w.phi), 0.4, dev(w.b.astype(np.complex64)), sigma=0.05, tol=1e-5, maxit=5000)
        prof = ctx.profile_read()
    assert abs(info["iters"] - ref.iters) <= 1
    r = b32 - A(host(x).astype(np.complex128))
    assert np.linalg.norm(r) / np.linalg.norm(b32) <= 5e-5
    assert prof["cg1_fused_f32"]["launches"] >= info["iters"]


def test_single_reduction_zero_rhs_and_iteration_limit():
    """b = 0 returns x = 0 without an iteration; maxit = 0 is rejected."""
    need_gpu()
    import paper_1804_07195_gb300 as hmc
    w = W.small(6, 6, 16, seed=1520)
    with ctx_for(w.lat) as ctx:
        ctx.set_cg_variant(6)
        z = torch.zeros(w.lat.nsites, dtype=torch.complex64, device="cuda")
        x, info = ctx.solve_spcg(dev(w.phi), 0.2, z, tol=1e-6, maxit=100)
        assert info["iters"] == 0 and float(x.abs().max()) == 0.0
        with pytest.raises(hmc.HMCError):
            ctx.solve_spcg(dev(w.phi), 0.2, dev(w.b.astype(np.complex64)), tol=1e-6, maxit=0)


def test_single_reduction_tile_limits():
    need_gpu()
    import paper_1804_07195_gb300 as hmc
    w = W.small(36, 36, 16, seed=1530)
    with ctx_for(w.lat) as ctx:
        with pytest.raises(hmc.HMCError):
            ctx.set_cg_fused_tile(30, 30, 8)  # 32 x 32 threads > 512
        with pytest.raises(hmc.HMCError):
            ctx.set_cg_fused_tile(14, 6, 8, 3)  # depth 2 or 6
        with pytest.raises(hmc.HMCError):
            ctx.set_cg_fused_tile(0, 6, 8)
        ctx.set_cg_fused_tile(14, 6, 8, 2)
        assert ctx.cg_fused_tile()[:4] == (14, 6, 8, 2)
        ctx.set_cg_fused_tile(0, 0, 0)
