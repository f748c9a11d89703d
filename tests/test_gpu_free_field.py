"""Full-size parity against the free-field closed form: for a constant field
phi = theta, M M^dagger + sigma is diagonal in plane waves (Eq. ferm_op, anti-
periodic time), so its application and its inverse are known exactly at any
size. On the 102x102, nt = 64 lattice (1.33M sites), in the launch
configurations the benchmark uses:
  - FP64 application element by element within 1e-12 of the largest entry,
    FP32 within 1e-5 (single-precision inputs, phases and sums);
  - FP64 CG, mixed FGMRES (a = 1 and the paper's a = 5) and mixed flexible CG
    to true residual 1e-10 (checked here with the closed form), and their
    solutions within kappa times that residual of the exact solution, kappa
    the exact condition number;
  - the batched solver on uneven lattices, each solution against its own
    lattice's closed form."""
import numpy as np
import pytest

from oracle import free_field
from oracle.lattice import Lattice as OLat

from gpu_util import dev, host, need_gpu, rel_max, torch

pytestmark = pytest.mark.gpu

FULL = (102, 102, 64, 1.0, 3.8, 12.0)
CASES = [(0.0, 0.0, 0.0), (0.3, 0.5, 0.0), (-1.2, 0.1, 0.04)]


def rand_vec(N, seed):
    g = np.random.default_rng(seed)
    return (g.normal(size=N) + 1j * g.normal(size=N)) * np.sqrt(0.5)


def context(shape):
    import paper_1804_07195_gb300 as hmc
    from paper_1804_07195_gb300 import build
    build.build()
    return hmc.Context(hmc.Lattice(*shape))


def true_rel(ol, ms, sigma, theta, x, b):
    return np.linalg.norm(free_field.apply_A(ol, ms, sigma, x, theta) - b) / np.linalg.norm(b)


@pytest.mark.parametrize("theta,ms,sigma", CASES)
def test_full_size_application(theta, ms, sigma):
    need_gpu()
    ol = OLat(*FULL)
    v = rand_vec(ol.N, 1)
    phi = dev(np.full(ol.N, theta))
    ref = free_field.apply_A(ol, ms, sigma, v, theta)
    v32 = v.astype(np.complex64)
    ref32 = free_field.apply_A(ol, ms, sigma, v32.astype(np.complex128), theta)
    with context(FULL) as ctx:
        got = host(ctx.apply_MMdag(phi, ms, dev(v), sigma))
        got32 = host(ctx.apply_MMdag(phi, ms, dev(v32), sigma))
    assert rel_max(got, ref) <= 1e-12
    assert rel_max(got32.astype(np.complex128), ref32) <= 1e-5


@pytest.mark.parametrize("theta,ms,sigma", CASES)
def test_full_size_solves_reach_the_exact_solution(theta, ms, sigma):
    need_gpu()
    ol = OLat(*FULL)
    b = rand_vec(ol.N, 2)
    phi = dev(np.full(ol.N, theta))
    exact = free_field.solve_A(ol, ms, sigma, b, theta)
    kappa = free_field.condition_number(ol, ms, sigma, theta)
    sols = {}
    with context(FULL) as ctx:
        x, _ = ctx.solve_cg(phi, ms, dev(b), sigma=sigma, tol=1e-10)
        sols["cg64"] = host(x)
        for a in (1.0, 5.0):
            x, _ = ctx.solve_fgmres(phi, ms, dev(b), sigma=sigma, tol=1e-10, a=a)
            sols["fgmres a=%g" % a] = host(x)
        x, _ = ctx.solve_fcg(phi, ms, dev(b), sigma=sigma, tol=1e-10, a=1.0)
        sols["fcg"] = host(x)
    for name, x in sols.items():
        rel = true_rel(ol, ms, sigma, theta, x, b)
        assert rel <= 1.0001e-10, (name, rel)
        err = np.linalg.norm(x - exact) / np.linalg.norm(exact)
        assert err <= kappa * rel + 1e-13, (name, err, kappa, rel)


@pytest.mark.parametrize("mixed", [1, 0])
def test_batched_uneven_lattices_reach_the_exact_solutions(mixed):
    need_gpu()
    import paper_1804_07195_gb300 as hmc
    shapes = [(36, 36, 48), (6, 6, 16), (24, 18, 32), (1, 1, 2), (12, 12, 64)]
    params = [(0.0, 0.1, 0.0), (0.7, 0.5, 0.0), (-0.4, 2.0, 0.0), (0.2, 0.0, 0.3), (1.1, 0.0, 0.0)]
    systems, refs = [], []
    for k, (sh, (theta, ms, sigma)) in enumerate(zip(shapes, params)):
        ol = OLat(sh[0], sh[1], sh[2], 1.0, 3.0, 6.0)
        b = rand_vec(ol.N, 10 + k)
        systems.append({"lattice": hmc.Lattice(sh[0], sh[1], sh[2], 1.0, 3.0, 6.0),
                        "phi": dev(np.full(ol.N, theta)), "ms": ms, "sigma": sigma, "b": dev(b),
                        "x": torch.zeros(ol.N, dtype=torch.complex128, device="cuda"), "tol": 1e-10,
                        "maxit": 100000})
        refs.append((ol, theta, ms, sigma, b))
    with context((shapes[0][0], shapes[0][1], shapes[0][2], 1.0, 3.0, 6.0)) as ctx:
        infos = ctx.solve_batched(systems, mixed=bool(mixed))
    for s, (ol, theta, ms, sigma, b), info in zip(systems, refs, infos):
        x = host(s["x"])
        rel = true_rel(ol, ms, sigma, theta, x, b)
        assert rel <= 1.0001e-10, (ol.n, ol.m, ol.nt, rel, info)
        exact = free_field.solve_A(ol, ms, sigma, b, theta)
        err = np.linalg.norm(x - exact) / np.linalg.norm(exact)
        assert err <= free_field.condition_number(ol, ms, sigma, theta) * rel + 1e-13
