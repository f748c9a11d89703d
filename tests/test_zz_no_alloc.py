"""hmc_apply_MMdag_noalloc: the operator for callers that cannot allocate device
memory (inside a CUDA-graph capture, beside a framework that owns the device's
memory pool, in loops that cannot pay for an allocation). It takes no context
and allocates nothing; its intermediate lives in the library's static scratch
array. Checked through the C ABI, on two calls in a row, against the oracle's
M M^dagger + sigma (oracle.fermion.apply_MMdag) with the FP64 operator
tolerance of the other tests (1e-12 of the largest entry), and against the
context entry point hmc_apply_MMdag; plus the size limit and the rejection of
partially overlapping vectors. Collected last on purpose."""
import ctypes as C

import numpy as np
import pytest

import workloads as W
from oracle import fermion as of
from oracle.lattice import Lattice as OLat

from gpu_util import ctx_for, dev, host, need_gpu, rel_max, torch

pytestmark = pytest.mark.gpu


def call_noalloc(lib, p, phi_ptr, ms, sigma, x_ptr, out_ptr):
    from paper_1804_07195_gb300 import _abi
    lat = _abi.hmc_lattice(p.n, p.m, p.nt, p.kappa, p.U, p.beta)
    return lib.hmc_apply_MMdag_noalloc(C.byref(lat), C.c_void_p(phi_ptr), ms, sigma, C.c_void_p(x_ptr),
                                       C.c_void_p(out_ptr), C.c_void_p(torch.cuda.current_stream().cuda_stream))


@pytest.mark.parametrize("shape,ms,sigma", [((6, 6, 16), 0.0, 0.0), ((2, 1, 4), 0.5, 0.0),
                                            ((36, 36, 64), 0.3, 0.25)])
def test_noalloc_matches_oracle_twice(shape, ms, sigma):
    need_gpu()
    import paper_1804_07195_gb300 as hmc
    from paper_1804_07195_gb300 import _abi
    lib = hmc.library()
    w = W.small(*shape, seed=900 + sum(shape))
    ol = OLat.from_params(w.lat)
    phi = dev(w.phi)
    hx = [w.b, w.rho[0]]
    xs = [dev(v) for v in hx]
    torch.cuda.synchronize()
    free0 = None
    outs = []
    for k, x in enumerate(xs):
        out = torch.empty_like(x)
        torch.cuda.synchronize()
        if k == 1:
            free0 = torch.cuda.mem_get_info()[0]
        assert call_noalloc(lib, w.lat, phi.data_ptr(), ms, sigma, x.data_ptr(), out.data_ptr()) == _abi.HMC_OK
        torch.cuda.synchronize()
        if k == 1:
            # the second call allocates nothing on the device
            assert torch.cuda.mem_get_info()[0] == free0
        ref = of.apply_MMdag(ol, w.phi, ms, hx[k], sigma)
        assert rel_max(host(out), ref) <= 1e-12
        outs.append(host(out))
    # and the same values as the context entry point
    with ctx_for(w.lat) as ctx:
        for k, x in enumerate(xs):
            assert rel_max(outs[k], host(ctx.apply_MMdag(phi, ms, x, sigma))) <= 1e-12


def test_noalloc_rejects_lattices_beyond_its_scratch():
    need_gpu()
    import paper_1804_07195_gb300 as hmc
    from paper_1804_07195_gb300 import _abi
    lib = hmc.library()
    p = W.L102  # 1,331,712 sites > HMC_NOALLOC_MAX_SITES
    assert p.nsites > _abi.HMC_NOALLOC_MAX_SITES
    phi = torch.zeros(p.nsites, dtype=torch.float64, device="cuda")
    x = torch.zeros(p.nsites, dtype=torch.complex128, device="cuda")
    out = torch.empty_like(x)
    assert call_noalloc(lib, p, phi.data_ptr(), 0.0, 0.0, x.data_ptr(), out.data_ptr()) == _abi.HMC_ERR_NOMEM


def test_noalloc_rejects_partial_overlap():
    """in and out that share part of their range are rejected before any launch."""
    need_gpu()
    import paper_1804_07195_gb300 as hmc
    from paper_1804_07195_gb300 import _abi
    lib = hmc.library()
    w = W.small(3, 3, 8, seed=905)
    N = w.lat.nsites
    phi = dev(w.phi)
    buf = torch.zeros(2 * N, dtype=torch.complex128, device="cuda")
    for shift in (0, 1, N - 1):
        st = call_noalloc(lib, w.lat, phi.data_ptr(), 0.0, 0.0, buf.data_ptr(), buf[shift:].data_ptr())
        assert st == _abi.HMC_ERR_INVALID
    # disjoint halves of the same buffer are fine
    buf[:N] = dev(w.b)
    assert call_noalloc(lib, w.lat, phi.data_ptr(), 0.0, 0.0, buf.data_ptr(), buf[N:].data_ptr()) == _abi.HMC_OK
    torch.cuda.synchronize()
    ref = of.apply_MMdag(OLat.from_params(w.lat), w.phi, 0.0, w.b)
    assert rel_max(host(buf[N:]), ref) <= 1e-12
