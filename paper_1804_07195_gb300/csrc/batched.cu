// Batched solves of many independent systems (placeholder until the batched
// kernels land).
#include "solvers.h"

using namespace hmc;

extern "C" hmc_status hmc_solve_batched(hmc_ctx* c, int nsys, const hmc_system* sys, int mixed,
                                        hmc_solve_info* infos) {
  (void)nsys; (void)sys; (void)mixed; (void)infos;
  return fail(c, HMC_ERR_INVALID, "hmc_solve_batched is not available in this build");
}
