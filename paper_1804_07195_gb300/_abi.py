"""ctypes declarations of the C ABI in include/hmc.h.

Argument marshalling only: every computation happens in libhmc.so. Loading
fails loudly when the library is missing; there is no fallback.
"""
from __future__ import annotations

import ctypes as C
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "_build", "libhmc.so")

HMC_OK = 0
HMC_ERR_INVALID = -1
HMC_ERR_CUDA = -2
HMC_ERR_NOT_CONVERGED = -3
HMC_ERR_NAN = -4
HMC_ERR_TIMEOUT = -5
HMC_ERR_NOMEM = -6

HMC_MAX_MASSES = 8
HMC_SOLVER_CG64 = 0
HMC_SOLVER_FGMRES_MIXED = 1
HMC_SOLVER_FGMRES_FP64 = 2
HMC_SOLVER_FCG_MIXED = 3
HMC_INTEG_NESTED_OMELYAN = 0
HMC_INTEG_LEAPFROG = 1
HMC_INTEG_FORCE_GRADIENT = 2
HMC_GAUSSIAN = 1
HMC_FERMION = 2
HMC_ACCUMULATE = 4


class hmc_lattice(C.Structure):
    _fields_ = [("n", C.c_int), ("m", C.c_int), ("nt", C.c_int),
                ("kappa", C.c_double), ("U", C.c_double), ("beta", C.c_double)]


class hmc_solve_info(C.Structure):
    _fields_ = [("iters", C.c_int), ("iters_outer", C.c_int), ("iters_inner", C.c_int),
                ("status", C.c_int), ("true_rel_res", C.c_double), ("seconds", C.c_double),
                ("applies64", C.c_longlong), ("applies32", C.c_longlong), ("bytes", C.c_longlong)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class hmc_solver_opts(C.Structure):
    _fields_ = [("method", C.c_int), ("tol", C.c_double), ("maxit", C.c_int),
                ("restart", C.c_int), ("a", C.c_double), ("inner_floor", C.c_double),
                ("inner_maxit", C.c_int)]


class hmc_integrator(C.Structure):
    _fields_ = [("kind", C.c_int), ("nmd", C.c_int), ("N", C.c_int * HMC_MAX_MASSES),
                ("zeta", C.c_double), ("tau", C.c_double)]


class hmc_system(C.Structure):
    _fields_ = [("lat", hmc_lattice), ("phi", C.c_void_p), ("ms", C.c_double),
                ("sigma", C.c_double), ("b", C.c_void_p), ("x", C.c_void_p),
                ("tol", C.c_double), ("maxit", C.c_int)]


class hmc_chain(C.Structure):
    _fields_ = [("lat", hmc_lattice), ("phi", C.c_void_p), ("pi", C.c_void_p), ("rho", C.POINTER(C.c_void_p))]


class hmc_kernel_stat(C.Structure):
    _fields_ = [("name", C.c_char * 48), ("launches", C.c_longlong), ("ms_total", C.c_double),
                ("bytes_total", C.c_double), ("threads", C.c_int), ("waves", C.c_int), ("design", C.c_int)]


HMC_NKERNELS = 40
HMC_NOALLOC_MAX_SITES = 1 << 20

P = C.c_void_p
D = C.c_double
I = C.c_int
S = C.c_int  # hmc_status

# name -> (restype, argtypes), in header order
PROTOTYPES = {
    "hmc_abi_version": (C.c_int, []),
    "hmc_status_string": (C.c_char_p, [S]),
    "hmc_last_error": (C.c_char_p, [P]),
    "hmc_create": (S, [C.POINTER(P), C.POINTER(hmc_lattice), P]),
    "hmc_destroy": (S, [P]),
    "hmc_set_stream": (S, [P, P]),
    "hmc_load_field": (S, [P, P]),
    "hmc_apply_M": (S, [P, P, D, P, P, I]),
    "hmc_apply_Mdag": (S, [P, P, D, P, P, I]),
    "hmc_apply_MMdag": (S, [P, P, D, D, P, P, I]),
    "hmc_solve_cg": (S, [P, P, D, D, P, P, D, I, C.POINTER(hmc_solve_info)]),
    "hmc_solve_spcg": (S, [P, P, D, D, P, P, D, I, C.POINTER(hmc_solve_info)]),
    "hmc_solve_fgmres": (S, [P, P, D, D, P, P, D, I, D, I, I, C.POINTER(hmc_solve_info)]),
    "hmc_solve_fcg": (S, [P, P, D, D, P, P, D, D, I, C.POINTER(hmc_solve_info)]),
    "hmc_solve_batched": (S, [P, I, C.POINTER(hmc_system), I, C.POINTER(hmc_solve_info)]),
    "hmc_make_chi": (S, [P, P, I, C.POINTER(D), C.POINTER(P), C.POINTER(P),
                         C.POINTER(hmc_solver_opts), C.POINTER(hmc_solve_info)]),
    "hmc_force": (S, [P, P, I, C.POINTER(D), C.POINTER(P), I, I, C.POINTER(hmc_solver_opts),
                      P, C.POINTER(hmc_solve_info)]),
    "hmc_action": (S, [P, P, I, C.POINTER(D), C.POINTER(P), I, I, C.POINTER(hmc_solver_opts),
                       C.POINTER(D), C.POINTER(hmc_solve_info)]),
    "hmc_md_trajectory": (S, [P, P, P, I, C.POINTER(D), C.POINTER(P), C.POINTER(hmc_integrator),
                              C.POINTER(hmc_solver_opts), C.POINTER(hmc_solver_opts),
                              C.POINTER(D), C.POINTER(D), C.POINTER(hmc_solve_info)]),
    "hmc_md_trajectory_batched": (S, [P, I, C.POINTER(hmc_chain), I, C.POINTER(D), C.POINTER(hmc_integrator),
                                      C.POINTER(hmc_solver_opts), C.POINTER(hmc_solver_opts), C.POINTER(D),
                                      C.POINTER(D), C.POINTER(hmc_solve_info)]),
    "hmc_set_cg_variant": (S, [P, I]),
    "hmc_set_batched_variant": (S, [P, I]),
    "hmc_batched_variant": (S, [P, C.POINTER(I)]),
    "hmc_set_apply_variant": (S, [P, I]),
    "hmc_apply_variant": (S, [P, I, C.POINTER(I)]),
    "hmc_set_fused_tile": (S, [P, I, I, I, I, I, I]),
    "hmc_fused_tile": (S, [P, I, C.POINTER(I), C.POINTER(I), C.POINTER(I), C.POINTER(I), C.POINTER(I)]),
    "hmc_set_cg_fused_tile": (S, [P, I, I, I, I]),
    "hmc_cg_fused_tile": (S, [P, C.POINTER(I), C.POINTER(I), C.POINTER(I), C.POINTER(I), C.POINTER(I)]),
    "hmc_set_wait_test": (S, [P, I, C.c_longlong]),
    "hmc_graph_mode": (S, [P, C.POINTER(I)]),
    "hmc_set_graph_mode": (S, [P, I]),
    "hmc_check_guards": (S, [P, C.POINTER(I)]),
    "hmc_guard_test_write": (S, [P]),
    "hmc_profile": (S, [P, I, I]),
    "hmc_apply_MMdag_noalloc": (S, [C.POINTER(hmc_lattice), P, D, D, P, P, P]),
    "hmc_profile_read": (S, [P, C.POINTER(hmc_kernel_stat), I, C.POINTER(I)]),
}

_lib = None


def load(path: str = LIB_PATH) -> C.CDLL:
    """Load libhmc.so (built by paper_1804_07195_gb300.build) and declare its
    prototypes. Raises if it is missing."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise RuntimeError(f"libhmc.so not found at {path}: build it with "
                           "`python -m paper_1804_07195_gb300.build` (there is no CPU fallback)")
    lib = C.CDLL(path)
    for name, (res, args) in PROTOTYPES.items():
        f = getattr(lib, name)
        f.restype = res
        f.argtypes = args
    _lib = lib
    return lib
