"""hmc_apply_MMdag_noalloc: the operator for callers that cannot allocate device
memory (inside a CUDA-graph capture, beside a framework that owns the device's
memory pool, in loops that cannot pay for an allocation). It takes no context
and allocates nothing; its intermediate lives in the library's static scratch
array. Checked through the C ABI against hmc_apply_MMdag on two calls in a row,
with the FP64 operator tolerance of the other tests (1e-12 of the largest
entry), plus the size limit. Collected last on purpose."""
import ctypes as C

import numpy as np
import pytest

import workloads as W

from gpu_util import ctx_for, dev, host, need_gpu, rel_max, torch

pytestmark = pytest.mark.gpu


def call_noalloc(lib, p, phi, ms, sigma, x, out):
    from paper_1804_07195_gb300 import _abi
    lat = _abi.hmc_lattice(p.n, p.m, p.nt, p.kappa, p.U, p.beta)
    return lib.hmc_apply_MMdag_noalloc(C.byref(lat), C.c_void_p(phi.data_ptr()), ms, sigma,
                                       C.c_void_p(x.data_ptr()), C.c_void_p(out.data_ptr()),
                                       C.c_void_p(torch.cuda.current_stream().cuda_stream))


@pytest.mark.parametrize("shape,ms,sigma", [((6, 6, 16), 0.0, 0.0), ((36, 36, 64), 0.3, 0.25)])
def test_noalloc_matches_context_apply_twice(shape, ms, sigma):
    need_gpu()
    import paper_1804_07195_gb300 as hmc
    from paper_1804_07195_gb300 import _abi
    lib = hmc.library()
    w = W.small(*shape, seed=900 + sum(shape))
    phi = dev(w.phi)
    xs = [dev(w.b), dev(w.rho[0])]
    with ctx_for(w.lat) as ctx:
        refs = [host(ctx.apply_MMdag(phi, ms, x, sigma)) for x in xs]
    torch.cuda.synchronize()
    free0 = None
    for k, x in enumerate(xs):
        out = torch.empty_like(x)
        torch.cuda.synchronize()
        if k == 1:
            free0 = torch.cuda.mem_get_info()[0]
        assert call_noalloc(lib, w.lat, phi, ms, sigma, x, out) == _abi.HMC_OK
        torch.cuda.synchronize()
        if k == 1:
            # the second call allocates nothing on the device
            assert torch.cuda.mem_get_info()[0] == free0
        assert rel_max(host(out), refs[k]) <= 1e-12


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
    assert call_noalloc(lib, p, phi, 0.0, 0.0, x, out) == _abi.HMC_ERR_NOMEM
