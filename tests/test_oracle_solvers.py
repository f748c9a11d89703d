"""Pins of the oracle's solvers (Section 3, Algorithm A.1) against LU solves of
the explicit matrix. CPU only."""
import numpy as np
import pytest

import workloads as W
from oracle import fermion, solvers
from oracle.lattice import Lattice


def problem(shape=(6, 6, 16), seed=1001, ms=0.0, sigma=0.0, U=2.0, beta=4.0):
    w = W.small(*shape, seed=seed, U=U, beta=beta)
    lat = Lattice.from_params(w.lat)
    D = fermion.dense_M(lat, w.phi, ms)
    Amat = D @ D.conj().T + sigma * np.eye(lat.N)
    A64 = lambda v: fermion.apply_MMdag(lat, w.phi, ms, v, sigma)

    def A32(v):
        # the same operator evaluated in complex64 throughout
        return fermion.apply_MMdag(lat, w.phi.astype(np.float32).astype(np.float64), ms,
                                   v.astype(np.complex64), sigma).astype(np.complex64)
    return w, lat, Amat, A64, A32


@pytest.mark.parametrize("ms,sigma", [(0.0, 0.0), (0.3, 0.0), (0.0, 0.09)])
def test_cg_matches_lu(ms, sigma):
    w, lat, Amat, A64, _ = problem(ms=ms, sigma=sigma)
    x_ref = solvers.dense_solve(Amat, w.b)
    res = solvers.cg(A64, w.b, tol=1e-12)
    assert res.converged
    assert solvers.true_rel_residual(A64, res.x, w.b) < 1e-11
    assert np.linalg.norm(res.x - x_ref) < 1e-9 * np.linalg.norm(x_ref)


def test_fgmres_matches_lu_and_uses_inner_solves(paper):
    w, lat, Amat, A64, A32 = problem()
    x_ref = solvers.dense_solve(Amat, w.b)
    res = solvers.fgmres(A64, A32, w.b, tol=1e-10, m=paper["fgmres_restart_m"],
                         a=paper["fgmres_inner_factor_a"])
    assert res.converged
    assert solvers.true_rel_residual(A64, res.x, w.b) <= 1e-10
    assert np.linalg.norm(res.x - x_ref) < 1e-7 * np.linalg.norm(x_ref)
    assert res.inner_iters > 0


def test_fgmres_without_preconditioning_is_gmres():
    """TOL a |b| / ERR >= 1 skips spCG (z_j = v_j): plain restarted GMRES."""
    w, lat, Amat, A64, A32 = problem(shape=(3, 3, 8))
    res = solvers.fgmres(A64, A32, w.b, tol=0.25, m=10, a=5.0)
    assert res.inner_iters == 0
    assert solvers.true_rel_residual(A64, res.x, w.b) <= 0.25


def test_fgmres_residual_estimate_tracks_true_residual():
    """The Givens estimate is the exact GMRES residual of the Arnoldi relation
    A Z = V H; check it against the true residual at each restart."""
    w, lat, Amat, A64, A32 = problem(shape=(3, 3, 8))
    res = solvers.fgmres(A64, A32, w.b, tol=1e-12, m=3, a=5.0, inner_floor=1e-2)
    assert res.converged and res.outer_iters >= 2
    assert solvers.true_rel_residual(A64, res.x, w.b) <= 1e-12


def test_fcg_matches_lu_with_few_outer_steps():
    w, lat, Amat, A64, A32 = problem()
    x_ref = solvers.dense_solve(Amat, w.b)
    res = solvers.fcg(A64, A32, w.b, tol=1e-10)
    assert res.converged and res.inner_iters > 0
    assert solvers.true_rel_residual(A64, res.x, w.b) <= 2e-10
    assert np.linalg.norm(res.x - x_ref) < 1e-7 * np.linalg.norm(x_ref)


def test_fcg_with_exact_preconditioner_is_one_step():
    """With z = A^{-1} r exactly, alpha = 1 and the first step solves the system."""
    w, lat, Amat, A64, A32 = problem(shape=(3, 3, 8))
    exact = lambda v, t: solvers.dense_solve(Amat, v)
    res = solvers.fcg(A64, None, w.b, tol=1e-12, precond=exact)
    assert res.iters == 1 and res.converged


def test_spcg_reaches_single_precision_floor():
    w, lat, Amat, A64, A32 = problem(shape=(3, 3, 8))
    res = solvers.spcg(A32, w.b, tol=1e-6)
    assert res.converged and res.x.dtype == np.complex64
    assert solvers.true_rel_residual(A64, res.x, w.b) < 1e-5


def test_zero_rhs():
    w, lat, Amat, A64, A32 = problem(shape=(2, 1, 4))
    z = np.zeros(lat.N, complex)
    assert np.all(solvers.cg(A64, z).x == 0)
    assert np.all(solvers.fgmres(A64, A32, z).x == 0)
