"""The fused M M^dagger kernel (u = M^dagger p kept in shared memory) against
the oracle's M M^dagger + sigma (Eq. ferm_op, Eq. hamiltonian): element by
element within 1e-12 of the largest entry in FP64 and 1e-5 in FP32, on
lattices with n or m of 1 to 3 (every wrap, coinciding bonds), odd and small
nt, and on pinned tiles that leave ragged tails in i, j and t (down to a
1 x 1 cell tile of one time slice); against the two-pass design at full size;
and the choice the library makes between the two."""
import numpy as np
import pytest

import workloads as W
from oracle import fermion as of
from oracle.lattice import Lattice as OLat

from gpu_util import ctx_for, dev, host, need_gpu, rel_max, torch

pytestmark = pytest.mark.gpu

SHAPES = [(1, 1, 2), (2, 1, 4), (1, 3, 5), (3, 3, 8), (2, 5, 3), (6, 6, 16), (7, 5, 9), (12, 12, 32),
          (36, 36, 64)]
# (Ti, Tj, Tt, depth): default-like, ragged in every direction, the smallest tile, each depth
TILES = [(30, 8, 16, 2), (5, 3, 7, 2), (1, 1, 1, 6), (62, 6, 64, 2), (30, 6, 5, 6), (4, 4, 2, 2)]
# FP64 takes depth 2 only
TILES64 = [t for t in TILES if t[3] == 2]


def fused_ctx(w, prec, tile=None):
    ctx = ctx_for(w.lat)
    ctx.set_apply_variant(2)
    if tile is not None:
        ctx.set_fused_tile(prec, *tile)
    return ctx


@pytest.mark.parametrize("shape", SHAPES)
@pytest.mark.parametrize("ms,sigma", [(0.0, 0.0), (0.3, 0.25)])
def test_fused_fp64_matches_oracle(shape, ms, sigma):
    need_gpu()
    w = W.small(*shape, seed=1200 + sum(shape))
    ol = OLat.from_params(w.lat)
    ref = of.apply_MMdag(ol, w.phi, ms, w.b, sigma)
    for tile in [None] + [t + (0,) for t in TILES64]:
        with fused_ctx(w, 64, tile) as ctx:
            got = host(ctx.apply_MMdag(dev(w.phi), ms, dev(w.b), sigma))
            assert ctx.apply_variant(64) == 2
        assert rel_max(got, ref) <= 1e-12, (shape, tile)


# FP32 tiles of the kernel with two cells per thread (Ti even): a wide tile,
# ragged ones, the smallest (one pair, one row, one slice) and a tall one
PAIR_TILES = [(60, 4, 16, 2), (4, 3, 5, 6), (2, 1, 1, 2), (28, 14, 64, 2), (10, 2, 3, 6), (28, 6, 5, 6)]


@pytest.mark.parametrize("shape", SHAPES)
def test_fused_fp32_matches_oracle(shape):
    need_gpu()
    import paper_1804_07195_gb300 as hmc
    w = W.small(*shape, seed=1300 + sum(shape))
    ol = OLat.from_params(w.lat)
    ref = of.apply_MMdag(ol, w.phi, 0.2, w.b, 0.04)
    x32 = dev(w.b).to(torch.complex64)
    tiles = [None] + [t + (0,) for t in TILES]
    if shape[0] % 2 == 0:
        tiles += [t + (1,) for t in PAIR_TILES]
    for tile in tiles:
        with fused_ctx(w, 32, tile) as ctx:
            got = host(ctx.apply_MMdag(dev(w.phi), 0.2, x32, 0.04))
        assert rel_max(got.astype(np.complex128), ref) <= 1e-5, (shape, tile)
    if shape[0] % 2 == 1:
        with ctx_for(w.lat) as ctx:
            with pytest.raises(hmc.HMCError):
                ctx.set_fused_tile(32, 2, 2, 2, 2, 1)  # odd n: no cell pairs


def test_fused_pairs_fall_back_on_unaligned_vectors():
    """Vectors that are 8- but not 16-byte aligned run the one-cell kernel
    even when the two-cell kernel is pinned; the result is the same."""
    need_gpu()
    w = W.small(12, 12, 32, seed=1310)
    N = w.lat.nsites
    ol = OLat.from_params(w.lat)
    ref = of.apply_MMdag(ol, w.phi, 0.1, w.b, 0.0)
    buf = torch.zeros(N + 2, dtype=torch.complex64, device="cuda")
    buf[1:N + 1] = dev(w.b).to(torch.complex64)
    out = torch.zeros(N + 2, dtype=torch.complex64, device="cuda")
    with fused_ctx(w, 32, (8, 4, 8, 2, 1)) as ctx:
        ctx.apply_MMdag(dev(w.phi), 0.1, buf[1:N + 1], out=out[1:N + 1])
        assert ctx.fused_tile(32)[4] == 1
    assert rel_max(host(out[1:N + 1]).astype(np.complex128), ref) <= 1e-5


@pytest.mark.parametrize("prec", [32, 64])
def test_fused_equals_two_pass_at_full_size(prec):
    """102x102x64 (the benchmark lattice) and a 306x306x64 lattice larger than
    L2: the fused kernel performs the two-pass design's operations in the same
    order, so the results agree to the last bits; rows sampled against the
    oracle (the full oracle apply at 12M sites is too slow for a test)."""
    need_gpu()
    import paper_1804_07195_gb300 as hmc
    for (n, m, nt) in ((102, 102, 64), (306, 306, 64)):
        lat = hmc.Lattice(n, m, nt, 1.0, 3.8, 12.0)
        g = np.random.default_rng(n)
        phi = torch.tensor(g.normal(0.0, np.sqrt(lat.delta * 3.8), lat.nsites), device="cuda")
        ct = torch.complex64 if prec == 32 else torch.complex128
        x = (torch.randn(lat.nsites, dtype=torch.complex128, device="cuda",
                         generator=torch.Generator("cuda").manual_seed(n))).to(ct)
        with hmc.Context(lat) as ctx:
            ctx.set_apply_variant(1)
            a = host(ctx.apply_MMdag(phi, 0.1, x, 0.01))
            ctx.set_apply_variant(2)
            b = host(ctx.apply_MMdag(phi, 0.1, x, 0.01))
        tol = 1e-6 if prec == 32 else 1e-14
        assert rel_max(b, a) <= tol
        if n == 102:
            # every 997th row against the oracle's operator, evaluated on the full lattice
            ol = OLat.from_params(W.LatticeParams(n, m, nt, 1.0, 3.8, 12.0))
            ref = of.apply_MMdag(ol, host(phi), 0.1, host(x).astype(np.complex128), 0.01)
            rows = np.arange(0, lat.nsites, 997)
            assert rel_max(b[rows].astype(np.complex128), ref[rows]) <= (1e-5 if prec == 32 else 1e-12)


def test_apply_variant_is_chosen_and_kept():
    need_gpu()
    w = W.small(12, 12, 32, seed=1400)
    with ctx_for(w.lat) as ctx:
        assert ctx.apply_variant(32) == 0 and ctx.apply_variant(64) == 0
        y1 = host(ctx.apply_MMdag(dev(w.phi), 0.0, dev(w.b)))
        v = ctx.apply_variant(64)
        assert v in (1, 2)
        y2 = host(ctx.apply_MMdag(dev(w.phi), 0.0, dev(w.b)))
        assert ctx.apply_variant(64) == v
        assert rel_max(y2, y1) <= 1e-14


def test_fused_tile_limits():
    need_gpu()
    import paper_1804_07195_gb300 as hmc
    w = W.small(36, 36, 16, seed=1401)
    with ctx_for(w.lat) as ctx:
        with pytest.raises(hmc.HMCError):
            ctx.set_fused_tile(32, 62, 30, 8)   # 64 x 32 threads > 1024
        with pytest.raises(hmc.HMCError):
            ctx.set_fused_tile(64, 0, 8, 8)
        with pytest.raises(hmc.HMCError):
            ctx.set_fused_tile(64, 30, 8, 8, 6)  # FP64: depth 2 only
        ctx.set_fused_tile(32, 30, 30, 16)      # 32 x 32 = 1024 threads: fits
