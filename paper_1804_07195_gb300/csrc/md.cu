// One HMC molecular-dynamics trajectory on the device (Section 2's HMC outline,
// Section 4's integrators, Section 5.2's nested time scales).
//
//   Q(c):     phi <- phi + c pi
//   P(k, c):  pi  <- pi - c dS_k/dphi(phi)
// Level k < n is the chi_k Hasenbusch term, level n the Gaussian term plus
// chi_n. Each level keeps its last force with the field version it was
// computed at, so a force is evaluated once per distinct field; momentum
// updates are never merged.
#include <cmath>
#include <cstring>
#include <string>
#include <vector>

#include "force.h"
#include "integrator.h"
#include "trace.h"

namespace hmc {

struct MD {
  hmc_ctx* c;
  double* phi;
  double* pi;
  int nmass;
  const double* masses;
  const double2* const* chi;
  const hmc_solver_opts* o;
  double* cache;   // (nmass + 1) x N forces
  std::vector<long long> cache_ver;
  long long ver = 0;
  long long tables_ver = -1;
  SolveStats st;
  int nforce = 0;
  hmc_status err = HMC_OK;
  double* phit = nullptr;  // force-gradient: the displaced field

  size_t N() const { return (size_t)c->geo.N; }

  hmc_status tables() {
    if (tables_ver == ver) return HMC_OK;
    HMC_TRY(prepare_field(c, phi));
    tables_ver = ver;
    return HMC_OK;
  }

  // dS_k/dphi at the current phi into `out` (level -1: all levels summed).
  hmc_status level_grad(int k, double* out) {
    HMC_TRACE("force level");
    HMC_TRY(tables());
    ++nforce;
    if (k == -1) {
      HMC_TRY(gauss_grad(c, phi, 0, out));
      for (int i = 0; i <= nmass; ++i) HMC_TRY(term_grad(c, nmass, masses, chi, i, o, out, &st));
      return HMC_OK;
    }
    if (k == nmass) {
      HMC_TRY(gauss_grad(c, phi, 0, out));
    } else {
      HMC_CUDA(c, cudaMemsetAsync(out, 0, N() * sizeof(double), c->stream));
    }
    return term_grad(c, nmass, masses, chi, k, o, out, &st);
  }

  void Q(double coef) {
    if (err != HMC_OK) return;
    err = axpy_real_launch(c, (int)N(), coef, pi, phi);
    ++ver;
  }

  // The force of level k at the current field, computed unless cached.
  double* ensure(int k) {
    const int slot = k < 0 ? nmass + 1 : k;
    double* f = cache + (size_t)slot * N();
    if (cache_ver[slot] != ver) {
      err = level_grad(k, f);
      if (err != HMC_OK) return nullptr;
      cache_ver[slot] = ver;
    }
    return f;
  }

  void P(int k, double coef) {
    if (err != HMC_OK) return;
    double* f = ensure(k);
    if (f) err = axpy_real_launch(c, (int)N(), -coef, f, pi);
  }

  bool ok() const { return err == HMC_OK; }

  // The middle kick of the force-gradient integrator (Eq. force_cal): the
  // force at phi_tilde = phi - (h^2/24) dS/dphi(phi) (new field versions, so
  // that neither the tables nor the cache of one field serve the other).
  void fg_kick(double coef, double h) {
    if (err != HMC_OK) return;
    const double* g1 = ensure(-1);
    if (!g1) return;
    if (!phit) {
      err = ws_get(c, WS_MD_PHI0, sizeof(double) * N(), (void**)&phit);
      if (err != HMC_OK) return;
    }
    cudaError_t e = cudaMemcpyAsync(phit, phi, sizeof(double) * N(), cudaMemcpyDeviceToDevice, c->stream);
    if (e != cudaSuccess) {
      err = cuda_fail(c, e, "force-gradient copy");
      return;
    }
    err = axpy_real_launch(c, (int)N(), -(h * h / 24.0), g1, phit);
    if (err != HMC_OK) return;
    double* keep = phi;
    phi = phit;
    ++ver;
    P(-1, coef);
    phi = keep;
    ++ver;
  }
};

}  // namespace hmc

using namespace hmc;

extern "C" hmc_status hmc_md_trajectory(hmc_ctx* c, double* phi, double* pi, int nmass,
                                        const double* masses, const void* const* rho,
                                        const hmc_integrator* integ, const hmc_solver_opts* md_opts,
                                        const hmc_solver_opts* action_opts, double* H0, double* H1,
                                        hmc_solve_info* agg) {
  if (!c) return HMC_ERR_INVALID;
  HMC_TRACE("hmc_md_trajectory");
  if (!phi || !pi || !integ || !md_opts || !action_opts || !H0 || !H1 || !rho)
    return fail(c, HMC_ERR_INVALID, "NULL argument");
  if (((uintptr_t)phi) % 8 || ((uintptr_t)pi) % 8) return fail(c, HMC_ERR_INVALID, "phi/pi misaligned");
  HMC_TRY(check_masses(c, nmass, masses));
  for (int i = 0; i <= nmass; ++i)
    if (!rho[i] || ((uintptr_t)rho[i]) % 16) return fail(c, HMC_ERR_INVALID, "rho entry NULL or misaligned");
  if (integ->nmd < 1 || !(integ->tau > 0.0)) return fail(c, HMC_ERR_INVALID, "bad nmd or tau");
  std::vector<int> steps;
  if (integ->kind == HMC_INTEG_NESTED_OMELYAN) {
    for (int k = 0; k < nmass; ++k) {
      const int Nk = integ->N[k];
      if (Nk < 1) return fail(c, HMC_ERR_INVALID, "time-scale ratio N_k must be >= 1");
      if (k == 0 && integ->nmd % Nk) return fail(c, HMC_ERR_INVALID, "N_0 must divide N_MD");
      if (k > 0 && integ->N[k - 1] % Nk) return fail(c, HMC_ERR_INVALID, "N_k must divide N_{k-1}");
      steps.push_back(integ->nmd / Nk);
    }
    steps.push_back(integ->nmd);
  } else if (integ->kind != HMC_INTEG_LEAPFROG && integ->kind != HMC_INTEG_FORCE_GRADIENT) {
    return fail(c, HMC_ERR_INVALID, "unknown integrator");
  }
  const size_t N = (size_t)c->geo.N;
  const size_t vb = sizeof(double2) * N;
  double2* chibuf;
  double* cache;
  HMC_TRY(ws_get(c, WS_MD_CHI, vb * (nmass + 1), (void**)&chibuf));
  HMC_TRY(ws_get(c, WS_MD_FORCE, sizeof(double) * N * (nmass + 2), (void**)&cache));
  std::vector<double2*> chi(nmass + 1);
  for (int i = 0; i <= nmass; ++i) chi[i] = chibuf + i * N;

  MD md{c, phi, pi, nmass, masses, chi.data(), md_opts, cache};
  md.cache_ver.assign(nmass + 2, -1);
  if (agg) std::memset(agg, 0, sizeof(*agg));

  // pseudofermions from rho at the starting field
  HMC_TRY(md.tables());
  SolveStats chist;
  hmc_status s = make_chi(c, nmass, masses, (const double2* const*)rho, chi.data(), action_opts, &chist);
  if (s != HMC_OK) return s;

  // H0 = phi^2/(2 delta U) + sum rho^dagger rho + pi^2/2
  const double inv_dU = 1.0 / (c->delta * c->lat.U);
  HMC_TRY(half_sq_launch(c, (int)N, phi, inv_dU, pi, c->dscal + 54, c->tickets));
  for (int i = 0; i <= nmass; ++i)
    HMC_TRY(norm2_launch(c, (int)N, (const double2*)rho[i], c->dscal + 56 + i, c->tickets));
  HMC_CUDA(c, cudaMemcpyAsync(c->dscal_host + 54, c->dscal + 54, sizeof(double) * (2 + nmass + 1),
                              cudaMemcpyDeviceToHost, c->stream));
  HMC_CUDA(c, cudaStreamSynchronize(c->stream));
  double h0 = c->dscal_host[54] + c->dscal_host[55];
  for (int i = 0; i <= nmass; ++i) h0 += c->dscal_host[56 + i];

  // molecular dynamics
  run_integrator(md, integ->kind, steps, integ->nmd, integ->zeta, integ->tau);
  if (md.err != HMC_OK) return md.err;

  // H1 = S(phi') + pi'^2/2 with the action solves at action_opts' tolerance
  HMC_TRY(md.tables());
  SolveStats hst;
  double h1 = 0.0;
  for (int i = 0; i <= nmass; ++i) {
    double Si = 0.0;
    s = term_action(c, nmass, masses, chi.data(), i, action_opts, &Si, &hst);
    if (s != HMC_OK) return s;
    h1 += Si;
  }
  HMC_TRY(half_sq_launch(c, (int)N, phi, inv_dU, pi, c->dscal + 54, c->tickets));
  HMC_CUDA(c, cudaMemcpyAsync(c->dscal_host + 54, c->dscal + 54, sizeof(double) * 2,
                              cudaMemcpyDeviceToHost, c->stream));
  HMC_CUDA(c, cudaStreamSynchronize(c->stream));
  h1 += c->dscal_host[54] + c->dscal_host[55];
  *H0 = h0;
  *H1 = h1;
  if (agg) {
    SolveStats all = md.st;
    all.iters += chist.iters + hst.iters;
    all.outer += chist.outer + hst.outer;
    all.inner += chist.inner + hst.inner;
    all.applies64 += chist.applies64 + hst.applies64;
    all.applies32 += chist.applies32 + hst.applies32;
    agg->iters = all.iters;
    agg->iters_outer = all.outer;
    agg->iters_inner = all.inner;
    agg->applies64 = all.applies64;
    agg->applies32 = all.applies32;
    agg->status = HMC_OK;
    agg->true_rel_res = hst.true_rel;
    agg->bytes = (long long)((double)N * (192.0 * all.applies64 + 96.0 * all.applies32));
  }
  return HMC_OK;
}
