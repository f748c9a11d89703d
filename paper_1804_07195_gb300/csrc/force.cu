// Pseudofermions, actions and forces of the Hasenbusch-split determinant
// (Section 5.1: the n-mass splitting, chi creation, Eqs. f_chi_i and def_xi_i;
// Eq. p_dot for the single term).
#include <cmath>
#include <cstring>
#include <string>

#include "force.h"
#include "trace.h"

namespace hmc {

static double lower_mass(const double* masses, int i) { return i == 0 ? 0.0 : masses[i - 1]; }

hmc_status check_masses(hmc_ctx* c, int nmass, const double* masses) {
  if (nmass < 0 || nmass > HMC_MAX_MASSES) return fail(c, HMC_ERR_INVALID, "nmass out of range");
  if (nmass > 0 && masses == nullptr) return fail(c, HMC_ERR_INVALID, "masses is NULL");
  for (int i = 0; i < nmass; ++i) {
    if (!std::isfinite(masses[i])) return fail(c, HMC_ERR_INVALID, "mass not finite");
    if (1.0 - c->delta * masses[i] == 0.0) return fail(c, HMC_ERR_INVALID, "1 - delta*mu == 0");
  }
  return HMC_OK;
}

// src_i and eta_i of term i (see hmc.h): eta = (M_lo M_lo^+)^{-1} src.
static hmc_status term_solve(hmc_ctx* c, int nmass, const double* masses, const double2* const* chi,
                             int i, const hmc_solver_opts* o, const double2** src_out,
                             double2** eta_out, SolveStats* st) {
  const Geo& g = c->geo;
  const size_t vb = sizeof(double2) * (size_t)g.N;
  double2 *src, *eta;
  HMC_TRY(ws_get(c, WS_F_SRC, vb, (void**)&src));
  HMC_TRY(ws_get(c, WS_F_ETA, vb, (void**)&eta));
  const double lo = lower_mass(masses, i);
  const double2* s;
  if (i == nmass) {
    s = chi[nmass];
  } else {
    HMC_TRY(m_launch<double>(c, g, c->delta * masses[i], chi[i], nullptr, 0.0, src));
    s = src;
  }
  hmc_status r = solve_opts(c, lo, 0.0, s, eta, o, st);
  if (r != HMC_OK) return r;
  *src_out = s;
  *eta_out = eta;
  return HMC_OK;
}

hmc_status term_grad(hmc_ctx* c, int nmass, const double* masses, const double2* const* chi, int i,
                     const hmc_solver_opts* o, double* grad, SolveStats* st) {
  HMC_TRACE("force term");
  const Geo& g = c->geo;
  const double2* src;
  double2* eta;
  HMC_TRY(term_solve(c, nmass, masses, chi, i, o, &src, &eta, st));
  double2* xi;
  HMC_TRY(ws_get(c, WS_F_XI, sizeof(double2) * (size_t)g.N, (void**)&xi));
  HMC_TRY(mdag_launch<double>(c, g, c->delta * lower_mass(masses, i), eta, xi));
  return force_launch(c, g, eta, xi, i == nmass ? nullptr : chi[i], grad);
}

// S_i = src^dagger (M_lo M_lo^dagger)^{-1} src, evaluated in the stationary form
//   S_i = 2 Re(src^dagger eta) - |M_lo^dagger eta|^2,
// which equals the definition for the exact eta and, for eta = eta* + e, is off
// by -e^dagger A e only: second order in the solve error instead of first
// order (src^dagger eta alone carries the error eta*^dagger r of any solver
// that is not Galerkin, such as flexible GMRES).
hmc_status term_action(hmc_ctx* c, int nmass, const double* masses, const double2* const* chi, int i,
                       const hmc_solver_opts* o, double* S_host, SolveStats* st) {
  const double2* src;
  double2* eta;
  HMC_TRY(term_solve(c, nmass, masses, chi, i, o, &src, &eta, st));
  double2* xi;
  HMC_TRY(ws_get(c, WS_F_XI, sizeof(double2) * (size_t)c->geo.N, (void**)&xi));
  HMC_TRY(mdag_launch<double>(c, c->geo, c->delta * lower_mass(masses, i), eta, xi));
  HMC_TRY(redot_launch(c, c->geo.N, src, eta, c->dscal + 100, c->tickets));
  HMC_TRY(norm2_launch(c, c->geo.N, xi, c->dscal + 101, c->tickets));
  HMC_CUDA(c, cudaMemcpyAsync(c->dscal_host + 100, c->dscal + 100, 2 * sizeof(double),
                              cudaMemcpyDeviceToHost, c->stream));
  HMC_CUDA(c, cudaStreamSynchronize(c->stream));
  *S_host = 2.0 * c->dscal_host[100] - c->dscal_host[101];
  return HMC_OK;
}

hmc_status make_chi(hmc_ctx* c, int nmass, const double* masses, const double2* const* rho,
                    double2* const* chi, const hmc_solver_opts* o, SolveStats* st) {
  const Geo& g = c->geo;
  const size_t vb = sizeof(double2) * (size_t)g.N;
  double2 *src, *y;
  HMC_TRY(ws_get(c, WS_F_SRC, vb, (void**)&src));
  HMC_TRY(ws_get(c, WS_F_ETA, vb, (void**)&y));
  for (int i = 0; i < nmass; ++i) {
    // chi_i = M_{mu_i}^+ (M_{mu_i} M_{mu_i}^+)^{-1} M_{mu_{i-1}} rho_i
    HMC_TRY(m_launch<double>(c, g, c->delta * lower_mass(masses, i), rho[i], nullptr, 0.0, src));
    hmc_status r = solve_opts(c, masses[i], 0.0, src, y, o, st);
    if (r != HMC_OK) return r;
    HMC_TRY(mdag_launch<double>(c, g, c->delta * masses[i], y, chi[i]));
  }
  // chi_n = M_{mu_{n-1}} rho_n
  const double top = nmass > 0 ? masses[nmass - 1] : 0.0;
  return m_launch<double>(c, g, c->delta * top, rho[nmass], nullptr, 0.0, chi[nmass]);
}

hmc_status gauss_grad(hmc_ctx* c, const double* phi, int accumulate, double* grad) {
  return gauss_grad_launch(c, c->geo.N, phi, 1.0 / (c->delta * c->lat.U), accumulate, grad);
}

}  // namespace hmc

using namespace hmc;

static hmc_status check_chi(hmc_ctx* c, int nmass, const void* const* v, const char* what) {
  if (v == nullptr) return fail(c, HMC_ERR_INVALID, std::string(what) + " is NULL");
  for (int i = 0; i <= nmass; ++i) {
    if (v[i] == nullptr || ((uintptr_t)v[i]) % 16)
      return fail(c, HMC_ERR_INVALID, std::string(what) + " entry is NULL or misaligned");
  }
  return HMC_OK;
}

static hmc_status check_opts(hmc_ctx* c, const hmc_solver_opts* o) {
  if (!o) return fail(c, HMC_ERR_INVALID, "solver options are NULL");
  if (o->method < HMC_SOLVER_CG64 || o->method > HMC_SOLVER_FCG_MIXED)
    return fail(c, HMC_ERR_INVALID, "unknown solver method");
  if (!(o->tol > 0.0) || o->maxit < 1) return fail(c, HMC_ERR_INVALID, "bad tol or maxit");
  if (o->method != HMC_SOLVER_CG64 &&
      (o->restart < 1 || o->restart > kMaxRestart || !(o->a > 0.0) || !(o->inner_floor > 0.0) ||
       o->inner_maxit < 1))
    return fail(c, HMC_ERR_INVALID, "bad FGMRES options");
  return HMC_OK;
}

static void to_info(hmc_solve_info* info, const SolveStats& s, hmc_status st, double N) {
  if (!info) return;
  std::memset(info, 0, sizeof(*info));
  info->iters = s.iters;
  info->iters_outer = s.outer;
  info->iters_inner = s.inner;
  info->status = st;
  info->true_rel_res = s.true_rel;
  info->applies64 = s.applies64;
  info->applies32 = s.applies32;
  info->bytes = (long long)(N * (192.0 * s.applies64 + 96.0 * s.applies32));
}

extern "C" {

hmc_status hmc_make_chi(hmc_ctx* c, const double* phi, int nmass, const double* masses,
                        const void* const* rho, void* const* chi, const hmc_solver_opts* opts,
                        hmc_solve_info* info) {
  if (!c) return HMC_ERR_INVALID;
  HMC_TRACE("hmc_make_chi");
  HMC_TRY(check_masses(c, nmass, masses));
  HMC_TRY(check_chi(c, nmass, rho, "rho"));
  HMC_TRY(check_chi(c, nmass, (const void* const*)chi, "chi"));
  HMC_TRY(check_opts(c, opts));
  HMC_TRY(prepare_field(c, phi));
  SolveStats s;
  hmc_status st = make_chi(c, nmass, masses, (const double2* const*)rho, (double2* const*)chi, opts, &s);
  to_info(info, s, st, c->geo.N);
  if (st == HMC_OK) HMC_CUDA(c, cudaStreamSynchronize(c->stream));
  return st;
}

hmc_status hmc_force(hmc_ctx* c, const double* phi, int nmass, const double* masses,
                     const void* const* chi, int term, int flags, const hmc_solver_opts* opts,
                     double* dSdphi, hmc_solve_info* info) {
  if (!c) return HMC_ERR_INVALID;
  HMC_TRACE("hmc_force");
  if (!dSdphi || ((uintptr_t)dSdphi) % 8) return fail(c, HMC_ERR_INVALID, "dSdphi NULL or misaligned");
  HMC_TRY(check_masses(c, nmass, masses));
  if (term < -1 || term > nmass) return fail(c, HMC_ERR_INVALID, "term out of range");
  const bool fermion = flags & HMC_FERMION;
  if (fermion) {
    HMC_TRY(check_chi(c, nmass, chi, "chi"));
    HMC_TRY(check_opts(c, opts));
  }
  if ((flags & HMC_GAUSSIAN) && phi == nullptr && c->loaded_phi == nullptr)
    return fail(c, HMC_ERR_INVALID, "the Gaussian term needs phi");
  HMC_TRY(prepare_field(c, phi));
  const double* ph = phi ? phi : c->loaded_phi;
  const size_t N = (size_t)c->geo.N;
  const bool acc = flags & HMC_ACCUMULATE;
  if (flags & HMC_GAUSSIAN)
    HMC_TRY(gauss_grad(c, ph, acc ? 1 : 0, dSdphi));
  else if (!acc)
    HMC_CUDA(c, cudaMemsetAsync(dSdphi, 0, N * sizeof(double), c->stream));
  SolveStats s;
  hmc_status st = HMC_OK;
  if (fermion) {
    for (int i = 0; i <= nmass && st == HMC_OK; ++i) {
      if (term != -1 && term != i) continue;
      st = term_grad(c, nmass, masses, (const double2* const*)chi, i, opts, dSdphi, &s);
    }
  }
  to_info(info, s, st, (double)N);
  if (st == HMC_OK) HMC_CUDA(c, cudaStreamSynchronize(c->stream));
  return st;
}

hmc_status hmc_action(hmc_ctx* c, const double* phi, int nmass, const double* masses,
                      const void* const* chi, int term, int flags, const hmc_solver_opts* opts,
                      double* S_out, hmc_solve_info* info) {
  if (!c) return HMC_ERR_INVALID;
  HMC_TRACE("hmc_action");
  if (!S_out) return fail(c, HMC_ERR_INVALID, "S_out is NULL");
  HMC_TRY(check_masses(c, nmass, masses));
  if (term < -1 || term > nmass) return fail(c, HMC_ERR_INVALID, "term out of range");
  const bool fermion = flags & HMC_FERMION;
  if (fermion) {
    HMC_TRY(check_chi(c, nmass, chi, "chi"));
    HMC_TRY(check_opts(c, opts));
  }
  HMC_TRY(prepare_field(c, phi));
  const double* ph = phi ? phi : c->loaded_phi;
  double total = 0.0;
  SolveStats s;
  hmc_status st = HMC_OK;
  if (flags & HMC_GAUSSIAN) {
    if (!ph) return fail(c, HMC_ERR_INVALID, "the Gaussian term needs phi");
    HMC_TRY(half_sq_launch(c, c->geo.N, ph, 1.0 / (c->delta * c->lat.U), nullptr, c->dscal + 50, c->tickets));
    HMC_CUDA(c, cudaMemcpyAsync(c->dscal_host + 50, c->dscal + 50, sizeof(double), cudaMemcpyDeviceToHost, c->stream));
    HMC_CUDA(c, cudaStreamSynchronize(c->stream));
    total += c->dscal_host[50];
  }
  if (fermion) {
    for (int i = 0; i <= nmass && st == HMC_OK; ++i) {
      if (term != -1 && term != i) continue;
      double Si = 0.0;
      st = term_action(c, nmass, masses, (const double2* const*)chi, i, opts, &Si, &s);
      if (st != HMC_OK) break;
      total += Si;
    }
  }
  *S_out = total;
  to_info(info, s, st, c->geo.N);
  return st;
}

}  // extern "C"
