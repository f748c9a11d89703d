"""GB300 (sm_103a) Hybrid Monte Carlo hot path for the Hubbard model on the
honeycomb lattice (arXiv:1804.07195): the fermion operator M[phi] and its
adjoint (Eq. ferm_op), CG and mixed-precision flexible GMRES solves of
M M^dagger (Section 3, Algorithm A.1), the Hasenbusch-split pseudofermion force
(Section 5.1, Eqs. p_dot, f_chi_i, def_xi_i) and the multi-time-scale MD
trajectory (Sections 2, 4 and 5.2).

The compute lives in libhmc.so (C ABI, include/hmc.h). This package is its
thin binding: `Context` mirrors the hmc_* entry points with the same names
and takes torch CUDA tensors (PyTorch supplies device memory and streams);
`PseudofermionAction` wraps the force as a torch.autograd.Function.
"""
from __future__ import annotations

import ctypes as C
from dataclasses import dataclass
from typing import List, Optional, Sequence

from . import _abi

__all__ = ["Context", "HMCError", "SolverOpts", "Integrator", "Lattice", "PseudofermionAction",
           "library"]


def library():
    return _abi.load()


class HMCError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"hmc status {status}: {msg}")
        self.status = status


@dataclass
class Lattice:
    """n x m honeycomb torus, nt time slices, hopping kappa, coupling U,
    inverse temperature beta (delta = beta / nt)."""
    n: int
    m: int
    nt: int
    kappa: float = 1.0
    U: float = 2.0
    beta: float = 4.0

    @property
    def nsites(self) -> int:
        return 2 * self.n * self.m * self.nt

    @property
    def delta(self) -> float:
        return self.beta / self.nt

    def c(self) -> _abi.hmc_lattice:
        return _abi.hmc_lattice(self.n, self.m, self.nt, self.kappa, self.U, self.beta)


@dataclass
class SolverOpts:
    method: int = _abi.HMC_SOLVER_FGMRES_MIXED
    tol: float = 1e-10
    maxit: int = 100000
    restart: int = 10
    a: float = 5.0
    inner_floor: float = 1e-6
    inner_maxit: int = 2000

    def c(self) -> _abi.hmc_solver_opts:
        return _abi.hmc_solver_opts(self.method, self.tol, self.maxit, self.restart, self.a,
                                    self.inner_floor, self.inner_maxit)


@dataclass
class Integrator:
    kind: int = _abi.HMC_INTEG_NESTED_OMELYAN
    nmd: int = 10
    N: Sequence[int] = ()
    zeta: float = 0.193
    tau: float = 1.0

    def c(self) -> _abi.hmc_integrator:
        arr = (C.c_int * _abi.HMC_MAX_MASSES)(*([int(x) for x in self.N] +
                                                [1] * (_abi.HMC_MAX_MASSES - len(self.N))))
        return _abi.hmc_integrator(self.kind, self.nmd, arr, self.zeta, self.tau)


def _ptr(t, dtype=None, n=None, what="tensor"):
    import torch
    if t is None:
        return None
    if not t.is_cuda:
        raise ValueError(f"{what} must be a CUDA tensor")
    if not t.is_contiguous():
        raise ValueError(f"{what} must be contiguous")
    if dtype is not None and t.dtype != dtype:
        raise TypeError(f"{what} must be {dtype}, got {t.dtype}")
    if n is not None and t.numel() != n:
        raise ValueError(f"{what} must have {n} elements, got {t.numel()}")
    return C.c_void_p(t.data_ptr())


def _prec(t):
    import torch
    if t.dtype == torch.complex128:
        return 64
    if t.dtype == torch.complex64:
        return 32
    raise TypeError("fermion vectors must be complex128 or complex64")


class Context:
    """One lattice on the current CUDA device, bound to a CUDA stream
    (default: torch's current stream). Methods mirror include/hmc.h."""

    def __init__(self, lattice: Lattice, stream=None):
        import torch
        self.lib = library()
        self.lat = lattice
        self.N = lattice.nsites
        if stream is None:
            stream = torch.cuda.current_stream()
        self.stream = stream
        h = C.c_void_p()
        st = self.lib.hmc_create(C.byref(h), C.byref(lattice.c()), C.c_void_p(stream.cuda_stream))
        if st != _abi.HMC_OK:
            raise HMCError(st, "hmc_create failed (invalid lattice or CUDA error)")
        self.h = h

    def close(self):
        if getattr(self, "h", None):
            self.lib.hmc_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def _check(self, st, allow=()):
        if st != _abi.HMC_OK and st not in allow:
            msg = self.lib.hmc_last_error(self.h)
            raise HMCError(st, msg.decode() if msg else "")
        return st

    # --- field and operator -------------------------------------------------
    def load_field(self, phi):
        import torch
        self._check(self.lib.hmc_load_field(self.h, _ptr(phi, torch.float64, self.N, "phi")))

    def _phi(self, phi):
        import torch
        return None if phi is None else _ptr(phi, torch.float64, self.N, "phi")

    def apply_M(self, phi, ms, x, out=None):
        import torch
        out = torch.empty_like(x) if out is None else out
        self._check(self.lib.hmc_apply_M(self.h, self._phi(phi), ms, _ptr(x, n=self.N),
                                         _ptr(out, x.dtype, self.N), _prec(x)))
        return out

    def apply_Mdag(self, phi, ms, x, out=None):
        import torch
        out = torch.empty_like(x) if out is None else out
        self._check(self.lib.hmc_apply_Mdag(self.h, self._phi(phi), ms, _ptr(x, n=self.N),
                                            _ptr(out, x.dtype, self.N), _prec(x)))
        return out

    def apply_MMdag(self, phi, ms, x, sigma=0.0, out=None):
        import torch
        out = torch.empty_like(x) if out is None else out
        self._check(self.lib.hmc_apply_MMdag(self.h, self._phi(phi), ms, sigma, _ptr(x, n=self.N),
                                             _ptr(out, x.dtype, self.N), _prec(x)))
        return out

    # --- solvers ------------------------------------------------------------
    def solve_cg(self, phi, ms, b, x=None, sigma=0.0, tol=1e-10, maxit=100000, allow_fail=False):
        import torch
        x = torch.zeros_like(b) if x is None else x
        info = _abi.hmc_solve_info()
        st = self.lib.hmc_solve_cg(self.h, self._phi(phi), ms, sigma,
                                   _ptr(b, torch.complex128, self.N, "b"),
                                   _ptr(x, torch.complex128, self.N, "x"), tol, maxit, C.byref(info))
        self._check(st, allow=(_abi.HMC_ERR_NOT_CONVERGED,) if allow_fail else ())
        return x, info.as_dict()

    def solve_spcg(self, phi, ms, b, sigma=0.0, tol=1e-6, maxit=2000, allow_fail=False):
        import torch
        x = torch.zeros_like(b)
        info = _abi.hmc_solve_info()
        st = self.lib.hmc_solve_spcg(self.h, self._phi(phi), ms, sigma,
                                     _ptr(b, torch.complex64, self.N, "b"),
                                     _ptr(x, torch.complex64, self.N, "x"), tol, maxit, C.byref(info))
        self._check(st, allow=(_abi.HMC_ERR_NOT_CONVERGED,) if allow_fail else ())
        return x, info.as_dict()

    def solve_fgmres(self, phi, ms, b, sigma=0.0, tol=1e-10, restart=10, a=5.0, inner_prec=32,
                     maxit=100000, allow_fail=False):
        import torch
        x = torch.zeros_like(b)
        info = _abi.hmc_solve_info()
        st = self.lib.hmc_solve_fgmres(self.h, self._phi(phi), ms, sigma,
                                       _ptr(b, torch.complex128, self.N, "b"),
                                       _ptr(x, torch.complex128, self.N, "x"), tol, restart, a,
                                       inner_prec, maxit, C.byref(info))
        self._check(st, allow=(_abi.HMC_ERR_NOT_CONVERGED,) if allow_fail else ())
        return x, info.as_dict()

    def solve_fcg(self, phi, ms, b, sigma=0.0, tol=1e-10, a=5.0, maxit=1000, allow_fail=False):
        import torch
        x = torch.zeros_like(b)
        info = _abi.hmc_solve_info()
        st = self.lib.hmc_solve_fcg(self.h, self._phi(phi), ms, sigma, _ptr(b, torch.complex128, self.N, "b"),
                                    _ptr(x, torch.complex128, self.N, "x"), tol, a, maxit, C.byref(info))
        self._check(st, allow=(_abi.HMC_ERR_NOT_CONVERGED,) if allow_fail else ())
        return x, info.as_dict()

    # --- Hasenbusch terms, force, action --------------------------------------
    def _vecs(self, vs, what):
        import torch
        arr = (C.c_void_p * len(vs))(*[_ptr(v, torch.complex128, self.N, what).value for v in vs])
        return arr

    def make_chi(self, phi, masses, rhos, opts: Optional[SolverOpts] = None):
        import torch
        opts = opts or SolverOpts()
        chis = [torch.empty_like(r) for r in rhos]
        m = (C.c_double * max(1, len(masses)))(*masses)
        info = _abi.hmc_solve_info()
        self._check(self.lib.hmc_make_chi(self.h, self._phi(phi), len(masses), m,
                                          self._vecs(rhos, "rho"), self._vecs(chis, "chi"),
                                          C.byref(opts.c()), C.byref(info)))
        return chis, info.as_dict()

    def force(self, phi, masses, chis, term=-1, flags=_abi.HMC_GAUSSIAN | _abi.HMC_FERMION,
              opts: Optional[SolverOpts] = None, out=None):
        import torch
        opts = opts or SolverOpts()
        out = torch.empty(self.N, dtype=torch.float64, device="cuda") if out is None else out
        m = (C.c_double * max(1, len(masses)))(*masses)
        info = _abi.hmc_solve_info()
        chiv = self._vecs(chis, "chi") if chis else None
        self._check(self.lib.hmc_force(self.h, self._phi(phi), len(masses), m, chiv, term, flags,
                                       C.byref(opts.c()), _ptr(out, torch.float64, self.N, "out"),
                                       C.byref(info)))
        return out, info.as_dict()

    def action(self, phi, masses, chis, term=-1, flags=_abi.HMC_GAUSSIAN | _abi.HMC_FERMION,
               opts: Optional[SolverOpts] = None):
        opts = opts or SolverOpts()
        m = (C.c_double * max(1, len(masses)))(*masses)
        S = C.c_double()
        info = _abi.hmc_solve_info()
        chiv = self._vecs(chis, "chi") if chis else None
        self._check(self.lib.hmc_action(self.h, self._phi(phi), len(masses), m, chiv, term, flags,
                                        C.byref(opts.c()), C.byref(S), C.byref(info)))
        return S.value, info.as_dict()

    def md_trajectory(self, phi, pi, masses, rhos, integ: Integrator, md_opts: SolverOpts,
                      action_opts: SolverOpts):
        """One trajectory; phi and pi (float64 CUDA tensors) are updated in
        place. Returns (H0, H1, info)."""
        import torch
        m = (C.c_double * max(1, len(masses)))(*masses)
        H0, H1 = C.c_double(), C.c_double()
        info = _abi.hmc_solve_info()
        self._check(self.lib.hmc_md_trajectory(
            self.h, _ptr(phi, torch.float64, self.N, "phi"), _ptr(pi, torch.float64, self.N, "pi"),
            len(masses), m, self._vecs(rhos, "rho"), C.byref(integ.c()), C.byref(md_opts.c()),
            C.byref(action_opts.c()), C.byref(H0), C.byref(H1), C.byref(info)))
        return H0.value, H1.value, info.as_dict()

    def md_trajectory_batched(self, chains: List[dict], masses, integ: Integrator, md_opts: SolverOpts,
                              action_opts: SolverOpts):
        """One trajectory for each chain (dicts with lattice, phi, pi, rho), all
        advanced in lockstep with batched solves; phi and pi are updated in
        place. Returns (H0 list, H1 list, info list)."""
        import torch
        K = len(chains)
        arr = (_abi.hmc_chain * K)()
        keep = []
        for k, ch in enumerate(chains):
            lat = ch["lattice"]
            n = lat.nsites
            rho = (C.c_void_p * len(ch["rho"]))(*[_ptr(r, torch.complex128, n, "rho").value for r in ch["rho"]])
            keep.append(rho)
            arr[k] = _abi.hmc_chain(lat.c(), _ptr(ch["phi"], torch.float64, n, "phi"),
                                    _ptr(ch["pi"], torch.float64, n, "pi"), rho)
        m = (C.c_double * max(1, len(masses)))(*masses)
        H0 = (C.c_double * K)()
        H1 = (C.c_double * K)()
        infos = (_abi.hmc_solve_info * K)()
        self._check(self.lib.hmc_md_trajectory_batched(self.h, K, arr, len(masses), m, C.byref(integ.c()),
                                                       C.byref(md_opts.c()), C.byref(action_opts.c()), H0, H1,
                                                       infos))
        return list(H0), list(H1), [i.as_dict() for i in infos]

    def solve_batched(self, systems: List[dict], mixed: bool = True):
        """systems: dicts with lattice (Lattice), phi, ms, sigma, b, x, tol, maxit."""
        import torch
        arr = (_abi.hmc_system * len(systems))()
        for k, s in enumerate(systems):
            lat = s["lattice"]
            n = lat.nsites
            arr[k] = _abi.hmc_system(lat.c(), _ptr(s["phi"], torch.float64, n, "phi"), s.get("ms", 0.0),
                                     s.get("sigma", 0.0), _ptr(s["b"], torch.complex128, n, "b"),
                                     _ptr(s["x"], torch.complex128, n, "x"), s.get("tol", 1e-10),
                                     s.get("maxit", 100000))
        infos = (_abi.hmc_solve_info * len(systems))()
        self._check(self.lib.hmc_solve_batched(self.h, len(systems), arr, 1 if mixed else 0, infos))
        return [i.as_dict() for i in infos]

    def set_cg_variant(self, variant: int):
        """0: autotune over all FP32 CG kernel designs; 1: grid-stride; 2: tiled;
        3: marching; 4: persistent (one cooperative launch per solve); 5:
        grid-stride with two cells per thread; 6: single-reduction (one fused
        kernel per iteration); 7: resident tiles (one cooperative launch, p
        and M^dagger p of each tile in shared memory)."""
        self._check(self.lib.hmc_set_cg_variant(self.h, variant))

    def set_batched_variant(self, variant: int):
        """FP32 CG of the batched solve: 0 = choose by timing (default), 1 =
        graph loop of per-iteration kernels, 2 = one persistent launch."""
        self._check(self.lib.hmc_set_batched_variant(self.h, variant))

    def batched_variant(self) -> int:
        v = C.c_int()
        self._check(self.lib.hmc_batched_variant(self.h, C.byref(v)))
        return v.value

    def set_apply_variant(self, variant: int):
        """M M^dagger applications: 0 = choose by timing (default), 1 = two
        passes through memory, 2 = the fused kernel (u kept on chip)."""
        self._check(self.lib.hmc_set_apply_variant(self.h, variant))

    def apply_variant(self, prec: int) -> int:
        v = C.c_int()
        self._check(self.lib.hmc_apply_variant(self.h, prec, C.byref(v)))
        return v.value

    def set_fused_tile(self, prec: int, Ti: int, Tj: int, Tt: int, depth: int = 2, pairs: int = 0):
        """Pin the fused kernel's tile: Ti x Tj cells and Tt time slices per
        block, `depth` slices staged ahead (2 or 6), pairs = 1 for the FP32
        kernel with two cells per thread (n and Ti even)."""
        self._check(self.lib.hmc_set_fused_tile(self.h, prec, Ti, Tj, Tt, depth, pairs))

    def fused_tile(self, prec: int):
        """(Ti, Tj, Tt, depth, pairs) of the fused kernel in use for precision prec."""
        v = [C.c_int() for _ in range(5)]
        self._check(self.lib.hmc_fused_tile(self.h, prec, *[C.byref(x) for x in v]))
        return tuple(x.value for x in v)

    def set_cg_fused_tile(self, Ti: int, Tj: int, Tt: int, depth: int = 2):
        """Pin the single-reduction FP32 CG kernel's tile (variant 6): Ti x Tj
        cells and Tt time slices per block, `depth` slices staged ahead (2 or
        6); (0, 0, 0) hands the choice back to the tuner."""
        self._check(self.lib.hmc_set_cg_fused_tile(self.h, Ti, Tj, Tt, depth))

    def cg_fused_tile(self):
        """(Ti, Tj, Tt, depth, in_use) of the single-reduction FP32 CG kernel."""
        v = [C.c_int() for _ in range(5)]
        self._check(self.lib.hmc_cg_fused_tile(self.h, *[C.byref(x) for x in v]))
        return tuple(x.value for x in v)

    def graph_mode(self) -> int:
        """2: one graph launch per CG solve (device-side loop); 1: captured
        chunks with host checks; 0: kernels launched one by one."""
        m = C.c_int()
        self._check(self.lib.hmc_graph_mode(self.h, C.byref(m)))
        return m.value

    def set_graph_mode(self, mode: int):
        """2: device-side loop graphs (default); 1: chunks with host checks
        (kernel profilers see the kernels only in this mode)."""
        self._check(self.lib.hmc_set_graph_mode(self.h, mode))

    def set_wait_test(self, extra: int, limit_cycles: int = 0):
        """Test hook: grid barriers of the persistent FP32 CG kernel wait for
        `extra` more arrivals than there are blocks and give up after
        `limit_cycles` SM cycles (0: default); (0, 0) restores normal work."""
        self._check(self.lib.hmc_set_wait_test(self.h, extra, limit_cycles))

    def check_guards(self) -> int:
        """Number of the context's device buffers whose guard bands were
        overwritten (0 when every kernel stayed inside its buffers)."""
        n = C.c_int()
        self._check(self.lib.hmc_check_guards(self.h, C.byref(n)))
        return n.value

    # --- instrumentation ----------------------------------------------------
    def profile(self, timing: bool, reset: bool = True):
        self._check(self.lib.hmc_profile(self.h, 1 if timing else 0, 1 if reset else 0))

    def profile_read(self):
        arr = (_abi.hmc_kernel_stat * _abi.HMC_NKERNELS)()
        cnt = C.c_int()
        self._check(self.lib.hmc_profile_read(self.h, arr, _abi.HMC_NKERNELS, C.byref(cnt)))
        return {arr[i].name.decode(): {"launches": arr[i].launches, "ms": arr[i].ms_total,
                                       "bytes": arr[i].bytes_total,
                                       "threads": arr[i].threads, "waves": arr[i].waves,
                                       "design": arr[i].design}
                for i in range(cnt.value)}


def apply_MMdag_noalloc(lattice: Lattice, phi, ms, x, sigma=0.0, out=None, stream=None):
    """out = (M M^dagger + sigma) x (complex128) through hmc_apply_MMdag_noalloc:
    no context and no device allocation inside the library (the intermediate
    lives in its static scratch array of HMC_NOALLOC_MAX_SITES entries)."""
    import torch
    lib = library()
    n = lattice.nsites
    out = torch.empty_like(x) if out is None else out
    if stream is None:
        stream = torch.cuda.current_stream()
    st = lib.hmc_apply_MMdag_noalloc(C.byref(lattice.c()), _ptr(phi, torch.float64, n, "phi"), ms, sigma,
                                     _ptr(x, torch.complex128, n, "x"), _ptr(out, torch.complex128, n, "out"),
                                     C.c_void_p(stream.cuda_stream))
    if st != _abi.HMC_OK:
        raise HMCError(st, "hmc_apply_MMdag_noalloc failed")
    return out


from .autograd import PseudofermionAction  # noqa: E402
