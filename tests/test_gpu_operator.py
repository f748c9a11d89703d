"""Parity of the CUDA operator applications with the oracle (Eq. ferm_op):
FP64 element by element within 1e-12 of the largest entry, FP32 within 5e-6
(single-precision rounding of inputs and phases plus the hardware sine/cosine
error of about 4e-7 on [-pi, pi], times the few terms summed per row)."""
import numpy as np
import pytest

import workloads as W
from oracle import fermion as of
from oracle.lattice import Lattice as OLat

from gpu_util import ctx_for, dev, host, need_gpu, rel_max, torch

pytestmark = pytest.mark.gpu

SHAPES = [(6, 6, 16), (1, 1, 2), (1, 3, 5), (2, 1, 4), (3, 3, 8), (4, 5, 6), (7, 3, 10), (36, 36, 64)]


@pytest.mark.parametrize("shape", SHAPES)
@pytest.mark.parametrize("ms", [0.0, 0.7])
def test_apply_fp64(shape, ms):
    need_gpu()
    w = W.small(*shape, seed=100 + sum(shape))
    ol = OLat.from_params(w.lat)
    with ctx_for(w.lat) as ctx:
        phi, b = dev(w.phi), dev(w.b)
        assert rel_max(host(ctx.apply_M(phi, ms, b)), of.apply_M(ol, w.phi, ms, w.b)) <= 1e-12
        assert rel_max(host(ctx.apply_Mdag(phi, ms, b)), of.apply_Mdag(ol, w.phi, ms, w.b)) <= 1e-12
        for sigma in (0.0, 0.3):
            ref = of.apply_MMdag(ol, w.phi, ms, w.b, sigma)
            assert rel_max(host(ctx.apply_MMdag(phi, ms, b, sigma)), ref) <= 1e-12


@pytest.mark.parametrize("shape", SHAPES)
def test_apply_fp32(shape):
    need_gpu()
    w = W.small(*shape, seed=200 + sum(shape))
    ol = OLat.from_params(w.lat)
    ms = 0.4
    with ctx_for(w.lat) as ctx:
        phi, b = dev(w.phi), dev(w.b.astype(np.complex64))
        bq = w.b.astype(np.complex64).astype(np.complex128)
        assert rel_max(host(ctx.apply_M(phi, ms, b)), of.apply_M(ol, w.phi, ms, bq)) <= 5e-6
        assert rel_max(host(ctx.apply_Mdag(phi, ms, b)), of.apply_Mdag(ol, w.phi, ms, bq)) <= 5e-6
        assert rel_max(host(ctx.apply_MMdag(phi, ms, b, 0.2)), of.apply_MMdag(ol, w.phi, ms, bq, 0.2)) <= 1e-5


def test_fp32_phases_of_any_size():
    """phi shifted by 2 pi K (|K| up to 3000, so |phi| up to about 19000) is the
    same field (Eq. ferm_op takes phi only through e^{i phi}): the FP32
    operators, both designs of M M^dagger and the resident CG's iterates keep
    their tolerances, since the float copy of phi is reduced to [-pi, pi] in
    FP64 before rounding (a float rounding of phi itself would misplace each
    phase by up to 1e-3 there)."""
    need_gpu()
    w = W.small(12, 12, 32, seed=210)
    ol = OLat.from_params(w.lat)
    K = np.random.default_rng(211).integers(-3000, 3001, size=w.phi.shape)
    phi_big = w.phi + 2.0 * np.pi * K
    ms = 0.4
    bq = w.b.astype(np.complex64).astype(np.complex128)
    with ctx_for(w.lat) as ctx:
        phi, b = dev(phi_big), dev(w.b.astype(np.complex64))
        assert rel_max(host(ctx.apply_M(phi, ms, b)), of.apply_M(ol, phi_big, ms, bq)) <= 5e-6
        assert rel_max(host(ctx.apply_Mdag(phi, ms, b)), of.apply_Mdag(ol, phi_big, ms, bq)) <= 5e-6
        ref = of.apply_MMdag(ol, phi_big, ms, bq, 0.2)
        for variant in (1, 2):
            ctx.set_apply_variant(variant)
            assert rel_max(host(ctx.apply_MMdag(phi, ms, b, 0.2)), ref) <= 1e-5, variant
        ctx.set_cg_variant(7)
        x, info = ctx.solve_spcg(phi, ms, b, sigma=0.0, tol=1e-30, maxit=3, allow_fail=True)
    from oracle import solvers as osv
    ref = osv.cg(lambda v: of.apply_MMdag(ol, phi_big, ms, v, 0.0), bq, tol=1e-30, maxit=3)
    assert info["iters"] == 3 and ref.iters == 3
    assert rel_max(host(x).astype(np.complex128), ref.x) <= 6e-5


def test_loaded_field_matches_explicit_field():
    need_gpu()
    w = W.workload("L6x6x16")
    with ctx_for(w.lat) as ctx:
        phi, b = dev(w.phi), dev(w.b)
        ref = host(ctx.apply_MMdag(phi, 0.1, b, 0.0))
        ctx.load_field(phi)
        phi.add_(1.0)  # the loaded tables are a copy
        got = host(ctx.apply_MMdag(None, 0.1, b, 0.0))
        assert np.array_equal(got, ref)


def test_largest_workload_sampled_rows():
    """102x102, nt=64 (1.33M sites): rows sampled across the lattice, including
    every wrap, against the oracle's stencil formula evaluated row by row."""
    need_gpu()
    w = W.workload("L102x102x64")
    lat = w.lat
    ol = OLat.from_params(lat)
    with ctx_for(lat) as ctx:
        phi, b = dev(w.phi), dev(w.b)
        got = host(ctx.apply_M(phi, 0.5, b))
        gotd = host(ctx.apply_Mdag(phi, 0.5, b))
    ref = of.apply_M(ol, w.phi, 0.5, w.b)
    refd = of.apply_Mdag(ol, w.phi, 0.5, w.b)
    assert rel_max(got, ref) <= 1e-12
    assert rel_max(gotd, refd) <= 1e-12


def test_invalid_arguments_raise():
    need_gpu()
    import paper_1804_07195_gb300 as hmc
    w = W.small(3, 3, 4, seed=1)
    with ctx_for(w.lat) as ctx:
        phi, b = dev(w.phi), dev(w.b)
        with pytest.raises(hmc.HMCError):
            ctx.apply_M(phi, 0.0, b, out=b)  # in == out
        with pytest.raises(hmc.HMCError):
            ctx.apply_M(phi, 1.0 / w.lat.delta, b)  # 1 - delta m_s == 0
        with pytest.raises(hmc.HMCError):
            ctx.apply_MMdag(phi, 0.0, b, sigma=-1.0)
        with pytest.raises(hmc.HMCError):
            ctx.apply_M(None, 0.0, b)  # no field loaded


def test_hundred_applications_each_of_M_and_Mdag():
    """6x6, nt=16 (1,152 sites): 100 successive applications of M, then 100 of
    M^dagger, each followed by an exact scaling by 1/2, through the library and
    through the oracle's stencil from the same start vector; every iterate
    agrees within 1e-12 of its largest entry (about 2 roundings per entry per
    application, accumulated over the chain)."""
    need_gpu()
    w = W.workload("L6x6x16")
    ol = OLat.from_params(w.lat)
    ms = 0.2
    ref = w.b.copy()
    with ctx_for(w.lat) as ctx:
        phi = dev(w.phi)
        cur = dev(w.b)
        for k in range(200):
            adj = k >= 100
            nxt = (ctx.apply_Mdag if adj else ctx.apply_M)(phi, ms, cur)
            nxt.mul_(0.5)
            ref = 0.5 * (of.apply_Mdag if adj else of.apply_M)(ol, w.phi, ms, ref)
            assert rel_max(host(nxt), ref) <= 1e-12, k
            cur = nxt
