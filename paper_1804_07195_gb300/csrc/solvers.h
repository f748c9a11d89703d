// Solver drivers shared by the entry points, the force and the trajectory.
#pragma once

#include "kernels.h"

namespace hmc {

struct SolveStats {
  int iters = 0, outer = 0, inner = 0;
  long long applies64 = 0, applies32 = 0;
  double true_rel = 0.0;
  int cg_done = 0;
};

// CG on (M_ms M_ms^dagger + sigma) x = b in precision R on the context's
// lattice and current phase tables. x holds the start vector unless x_zero.
template <typename R>
hmc_status cg_core(hmc_ctx* c, double ms, double sigma, const V2<R>* b, V2<R>* x, bool x_zero,
                   double tol, int maxit, int sc_slot, bool want_true_res, SolveStats* st);

// Algorithm A.1 on the context's lattice and current phase tables.
hmc_status fgmres_core(hmc_ctx* c, double ms, double sigma, const double2* b, double2* x, double tol,
                       int restart, double a, int inner_prec, int maxit, double inner_floor,
                       int inner_maxit, SolveStats* st);

// z = A^{-1} v to relative tolerance t by CG in precision prec (32: through
// float copies; 64: FP64); t >= 1 gives z = v.
hmc_status precondition_solve(hmc_ctx* c, double ms, double sigma, const double2* v64, const float2* v32,
                              double2* z, double t, int prec, int inner_maxit, SolveStats* st);

// Flexible CG with an FP32 CG preconditioner (Section 3).
hmc_status fcg_core(hmc_ctx* c, double ms, double sigma, const double2* b, double2* x, double tol,
                    double a, int maxit, double inner_floor, int inner_maxit, SolveStats* st);

// Dispatch on opts->method; x is the output (start at 0).
hmc_status solve_opts(hmc_ctx* c, double ms, double sigma, const double2* b, double2* x,
                      const hmc_solver_opts* opts, SolveStats* st);

// out = (M_ms M_ms^dagger + sigma) in, FP64, using the context's U64 slot.
hmc_status apply_A64(hmc_ctx* c, double ms, double sigma, const double2* in, double2* out);

void add_stats(hmc_solve_info* info, const SolveStats& s);
hmc_solver_opts default_opts();

}  // namespace hmc
