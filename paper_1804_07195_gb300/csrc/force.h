// Hasenbusch terms: pseudofermion creation, per-term action and force.
#pragma once

#include "solvers.h"

namespace hmc {

hmc_status check_masses(hmc_ctx* c, int nmass, const double* masses);
// grad += dS_i/dphi for term i (the context's phase tables must hold phi).
hmc_status term_grad(hmc_ctx* c, int nmass, const double* masses, const double2* const* chi, int i,
                     const hmc_solver_opts* o, double* grad, SolveStats* st);
// *S_host = S_i (stationary form, synchronises).
hmc_status term_action(hmc_ctx* c, int nmass, const double* masses, const double2* const* chi, int i,
                       const hmc_solver_opts* o, double* S_host, SolveStats* st);
hmc_status make_chi(hmc_ctx* c, int nmass, const double* masses, const double2* const* rho,
                    double2* const* chi, const hmc_solver_opts* o, SolveStats* st);
// grad (+)= phi / (delta U)
hmc_status gauss_grad(hmc_ctx* c, const double* phi, int accumulate, double* grad);

}  // namespace hmc
