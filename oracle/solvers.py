"""Linear solvers for A x = b with A = M_{m_s} M_{m_s}^dagger + sigma (Section 3 and
Algorithm A.1).

  dense_solve -- LU factorisation of the explicit matrix (scipy), the plain
                 definition x = A^{-1} b, for tiny lattices.
  cg          -- conjugate gradient in complex128 (Section 3: relative tolerance on
                 the recursive residual).
  spcg        -- the same CG with vectors and operator in complex64 and dot
                 products accumulated in float64 (the single-precision CG of
                 Section 3, used as the preconditioner).
  fgmres      -- flexible GMRES with spCG as preconditioner, Algorithm A.1, with
                 restart length m = 10 and inner tolerance factor a = 5 (Appendix A).
  fcg         -- flexibly preconditioned CG with spCG as preconditioner, the
                 mixed-precision solver Section 3 describes before FGMRES.

Readings taken where Algorithm A.1 is garbled or silent:
  * h and y are complex (the operator is complex Hermitian); h_ij = v_i^H w,
    computed for all i <= j from the same w (classical Gram-Schmidt).
  * the running residual estimate ERR after each Arnoldi step is the GMRES
    residual norm tracked by Givens rotations, |g_{j+1}|.
  * the least-squares problem is solved through the normal equations
    h^H h y = |r| h^H e_1 with a Cholesky factorisation, as the appendix states.
  * the spCG tolerance is max(TOL a |b| / ERR, floor) with floor = 1e-6; the first
    solve uses max(TOL a, floor); spCG stops after at most 2000 iterations.
"""
from __future__ import annotations

from dataclasses import dataclass, field
from typing import Callable, List

import numpy as np
import scipy.linalg as sla


def dense_solve(Amat: np.ndarray, b: np.ndarray) -> np.ndarray:
    """The plain definition x = A^{-1} b (Section 3)."""
    lu = sla.lu_factor(Amat)
    return sla.lu_solve(lu, b)


def vdot64(u: np.ndarray, v: np.ndarray) -> complex:
    """u^H v accumulated in complex128 whatever the storage precision."""
    return complex(np.vdot(u.astype(np.complex128), v.astype(np.complex128)))


def norm2_64(u: np.ndarray) -> float:
    """Section 3."""
    uu = u.astype(np.complex128)
    return float(np.real(np.vdot(uu, uu)))


@dataclass
class SolveResult:
    """Section 3 and Appendix A."""
    x: np.ndarray
    iters: int
    converged: bool
    res_history: List[float] = field(default_factory=list)
    inner_iters: int = 0
    outer_iters: int = 0


def cg(apply_A: Callable, b: np.ndarray, tol: float = 1e-10, maxit: int = 100000,
       x0=None, dtype=np.complex128) -> SolveResult:
    """Textbook CG for a Hermitian positive definite A (Section 3, ref. templates):
        alpha = |r|^2 / <p, A p>;  x += alpha p;  r -= alpha A p;
        beta = |r_new|^2 / |r|^2;  p = r + beta p,
    stopped when |r| <= tol |b| (recursive residual)."""
    b = b.astype(dtype)
    x = np.zeros_like(b) if x0 is None else x0.astype(dtype).copy()
    r = b - apply_A(x) if x0 is not None else b.copy()
    p = r.copy()
    rr = norm2_64(r)
    bb = norm2_64(b)
    hist = [np.sqrt(rr)]
    if bb == 0.0:
        return SolveResult(np.zeros_like(b), 0, True, hist)
    k = 0
    while rr > tol * tol * bb and k < maxit:
        Ap = apply_A(p)
        pAp = float(np.real(vdot64(p, Ap)))
        alpha = rr / pAp
        x = x + dtype(alpha) * p if dtype is np.complex64 else x + alpha * p
        r = r - (np.float32(alpha) if dtype is np.complex64 else alpha) * Ap
        rr_new = norm2_64(r)
        beta = rr_new / rr
        p = r + (np.float32(beta) if dtype is np.complex64 else beta) * p
        rr = rr_new
        k += 1
        hist.append(np.sqrt(rr))
    return SolveResult(x, k, rr <= tol * tol * bb, hist)


def spcg(apply_A32: Callable, b: np.ndarray, tol: float, maxit: int = 2000) -> SolveResult:
    """Single-precision CG (Section 3): complex64 vectors and operator,
    float64 dot products."""
    return cg(apply_A32, b.astype(np.complex64), tol=tol, maxit=maxit, dtype=np.complex64)


def _givens(a: complex, b: complex):
    """A rotation G = [[c, s], [-conj(s), c]] with c real such that
    G [a, b]^T = [r, 0]^T."""
    if b == 0:
        return 1.0, 0.0 + 0.0j
    if a == 0:
        return 0.0, np.conj(b) / abs(b)
    na = abs(a)
    nrm = np.hypot(na, abs(b))
    c = na / nrm
    s = (a / na) * np.conj(b) / nrm
    return c, s


def fgmres(apply_A: Callable, apply_A32: Callable, b: np.ndarray, tol: float = 1e-10,
           m: int = 10, a: float = 5.0, inner_floor: float = 1e-6,
           inner_maxit: int = 2000, max_restarts: int = 1000) -> SolveResult:
    """Flexible GMRES with spCG as preconditioner, Algorithm A.1 (Appendix A)."""
    b = b.astype(np.complex128)
    bnorm = np.sqrt(norm2_64(b))
    hist: List[float] = []
    if bnorm == 0.0:
        return SolveResult(np.zeros_like(b), 0, True, [0.0])
    inner_total = 0

    def precondition(v, err):
        nonlocal inner_total
        t = tol * a * bnorm / err
        if t < 1.0:
            res = spcg(apply_A32, v, max(t, inner_floor), inner_maxit)
            inner_total += res.iters
            return res.x.astype(np.complex128)
        return v.copy()

    # first line of Algorithm A.1: an spCG solve of A x = b (tolerance TOL a, floored;
    # a tolerance >= 1 returns x = 0 after no iteration), then the true residual
    first = spcg(apply_A32, b, max(tol * a, inner_floor), inner_maxit)
    inner_total += first.iters
    x = first.x.astype(np.complex128)
    r = b - apply_A(x)
    err = np.sqrt(norm2_64(r))
    w = r.copy()
    hist.append(err / bnorm)
    outer = 0
    arnoldi = 0
    while err > tol * bnorm and outer < max_restarts:
        rnorm = err
        V: List[np.ndarray] = []
        Z: List[np.ndarray] = []
        H = np.zeros((m + 1, m), dtype=np.complex128)
        rot_c = np.zeros(m)
        rot_s = np.zeros(m, dtype=np.complex128)
        g = np.zeros(m + 1, dtype=np.complex128)
        g[0] = rnorm
        k = 0
        for j in range(m):
            if err < tol * bnorm:
                break
            V.append(w / np.sqrt(norm2_64(w)))
            Z.append(precondition(V[j], err))
            w = apply_A(Z[j])
            for i in range(j + 1):
                H[i, j] = vdot64(V[i], w)
            for i in range(j + 1):
                w = w - H[i, j] * V[i]
            H[j + 1, j] = np.sqrt(norm2_64(w))
            # running residual estimate: rotate column j and update g
            col = H[: j + 2, j].copy()
            for i in range(j):
                c, s = rot_c[i], rot_s[i]
                t0 = c * col[i] + s * col[i + 1]
                col[i + 1] = -np.conj(s) * col[i] + c * col[i + 1]
                col[i] = t0
            c, s = _givens(col[j], col[j + 1])
            rot_c[j], rot_s[j] = c, s
            g[j + 1] = -np.conj(s) * g[j]
            g[j] = c * g[j]
            err = abs(g[j + 1])
            k = j + 1
            arnoldi += 1
        if k == 0:
            break
        h = H[: k + 1, :k]
        # argmin | |r| e_1 - h y |  via  h^H h y = |r| h^H e_1  (Cholesky)
        lhs = h.conj().T @ h
        rhs = rnorm * h[0, :].conj()
        y = sla.cho_solve(sla.cho_factor(lhs), rhs)
        for i in range(k):
            x = x + y[i] * Z[i]
        r = b - apply_A(x)
        err = np.sqrt(norm2_64(r))
        w = r.copy()
        outer += 1
        hist.append(err / bnorm)
    res = SolveResult(x, arnoldi, err <= tol * bnorm, hist)
    res.inner_iters = inner_total
    res.outer_iters = outer
    return res


def fcg(apply_A: Callable, apply_A32: Callable, b: np.ndarray, tol: float = 1e-10, a: float = 5.0,
        inner_floor: float = 1e-6, inner_maxit: int = 2000, maxit: int = 1000,
        precond: Callable = None) -> SolveResult:
    """Flexible CG (Section 3: an FP64 CG whose preconditioner is the spCG
    solve, made flexible because spCG with a tolerance is not a fixed linear
    map; Notay's method). Readings, as the paper gives no detail: one previous
    direction is kept (truncation 1),
        z_i = spCG(r_i),  p_i = z_i - (p_{i-1}^H A z_i / p_{i-1}^H A p_{i-1}) p_{i-1},
        alpha = p_i^H r_i / p_i^H A p_i,  x += alpha p_i,  r -= alpha A p_i,
    with the spCG tolerance max(TOL a |b| / |r_i|, floor) of Algorithm A.1 and
    z_i = r_i once that ratio reaches 1; stop when the recursive residual
    satisfies |r| <= TOL |b|. `precond(r, tol)` replaces the spCG solve when
    given (z = r is still used once TOL a |b| / |r| >= 1)."""
    b = b.astype(np.complex128)
    bnorm = np.sqrt(norm2_64(b))
    if bnorm == 0.0:
        return SolveResult(np.zeros_like(b), 0, True, [0.0])
    x = np.zeros_like(b)
    r = b.copy()
    rnorm = bnorm
    hist = [1.0]
    inner_total = 0
    p_prev = q_prev = None
    pq_prev = None
    k = 0
    while rnorm > tol * bnorm and k < maxit:
        t = tol * a * bnorm / rnorm
        if t < 1.0 and precond is not None:
            z = precond(r, max(t, inner_floor))
        elif t < 1.0:
            res = spcg(apply_A32, r, max(t, inner_floor), inner_maxit)
            inner_total += res.iters
            z = res.x.astype(np.complex128)
        else:
            z = r.copy()
        if p_prev is None:
            p = z
        else:
            beta = vdot64(q_prev, z) / pq_prev   # (A p_prev)^H z / p_prev^H A p_prev
            p = z - beta * p_prev
        q = apply_A(p)
        pq = float(np.real(vdot64(p, q)))
        alpha = vdot64(p, r) / pq
        x = x + alpha * p
        r = r - alpha * q
        rnorm = np.sqrt(norm2_64(r))
        p_prev, q_prev, pq_prev = p, q, pq
        k += 1
        hist.append(rnorm / bnorm)
    out = SolveResult(x, k, rnorm <= tol * bnorm, hist)
    out.inner_iters = inner_total
    return out


def true_rel_residual(apply_A: Callable, x: np.ndarray, b: np.ndarray) -> float:
    """Section 3: the true residual, checked in FP64."""
    r = b.astype(np.complex128) - apply_A(x.astype(np.complex128))
    return float(np.sqrt(norm2_64(r) / norm2_64(b)))
