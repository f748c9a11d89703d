// K independent HMC trajectories advanced in lockstep: Section 2's HMC outline
// with the integrators of Sections 4 and 5.2 and the Hasenbusch terms of
// Section 5.1, for Markov chains that may live on lattices of uneven sizes.
//
// All chains follow the same integrator schedule, so at every point of it they
// need the same kind of solve: one per chain (and per Hasenbusch term where a
// force level or the action has several). Those solves run as ONE batched solve
// (hmc_solve_batched: one launch per kernel per CG iteration over all systems,
// converged systems masked, the iteration loop a device-side CUDA-graph loop).
// The stencils, forces and field updates of each chain run on a per-chain
// context (its lattice, phase tables and workspace), all on the caller's
// context's stream. A force is evaluated once per distinct field for all
// chains together, as in the single-chain trajectory.
#include <cmath>
#include <cstring>
#include <string>
#include <vector>

#include "force.h"
#include "integrator.h"
#include "trace.h"
#include "validate.h"

namespace hmc {
namespace {

double lower_mass(const double* masses, int i) { return i == 0 ? 0.0 : masses[i - 1]; }

struct BChain {
  hmc_ctx* c = nullptr;
  double* phi = nullptr;
  double* pi = nullptr;
  double* phi_home = nullptr;  // the caller's field (phi is swapped for the force-gradient kick)
  const double2* rho[HMC_MAX_MASSES + 1] = {};
  double2* chi[HMC_MAX_MASSES + 1] = {};
  double* cache = nullptr;  // (nmass + 2) forces of N doubles
  double* phit = nullptr;
  SolveStats st;
  size_t N() const { return (size_t)c->geo.N; }
};

struct BatchMD {
  hmc_ctx* ctx;
  std::vector<BChain>& ch;
  int nmass;
  const double* masses;
  const hmc_solver_opts* o;
  std::vector<long long> cache_ver;
  long long ver = 0, tables_ver = -1;
  hmc_status err = HMC_OK;
  std::vector<hmc_system> sys;
  std::vector<hmc_solve_info> infos;

  bool ok() const { return err == HMC_OK; }

  hmc_status tables() {
    if (tables_ver == ver) return HMC_OK;
    for (BChain& b : ch) HMC_TRY(prepare_field(b.c, b.phi));
    tables_ver = ver;
    return HMC_OK;
  }

  // eta_c = (M_lo M_lo^dagger)^{-1} src_c for every chain c, one batched solve
  // (FP64 CG for HMC_SOLVER_CG64, else FP32 CG under FP64 defect correction).
  hmc_status solve_all(double ms_lo, const std::vector<const double2*>& src, const std::vector<double2*>& eta,
                       const hmc_solver_opts* so, bool last_res = false) {
    const int K = (int)ch.size();
    sys.resize(K);
    infos.resize(K);
    for (int i = 0; i < K; ++i) {
      hmc_system& y = sys[i];
      y.lat = ch[i].c->lat;
      y.phi = ch[i].phi;
      y.ms = ms_lo;
      y.sigma = 0.0;
      y.b = src[i];
      y.x = eta[i];
      y.tol = so->tol;
      y.maxit = so->maxit;
    }
    const hmc_status s = hmc_solve_batched(ctx, K, sys.data(), so->method == HMC_SOLVER_CG64 ? 0 : 1, infos.data());
    for (int i = 0; i < K; ++i) {
      SolveStats& t = ch[i].st;
      t.iters += infos[i].iters;
      t.outer += infos[i].iters_outer;
      t.inner += infos[i].iters_inner;
      t.applies64 += infos[i].applies64;
      t.applies32 += infos[i].applies32;
      if (last_res) t.true_rel = infos[i].true_rel_res;
    }
    return s;
  }

  // src_i of term i for every chain (M_{mu_i} chi_i, or chi_n for the top term)
  hmc_status sources(int i, std::vector<const double2*>& src, std::vector<double2*>& eta) {
    const int K = (int)ch.size();
    src.resize(K);
    eta.resize(K);
    for (int c = 0; c < K; ++c) {
      BChain& b = ch[c];
      const size_t vb = sizeof(double2) * b.N();
      double2 *s, *e;
      HMC_TRY(ws_get(b.c, WS_F_SRC, vb, (void**)&s));
      HMC_TRY(ws_get(b.c, WS_F_ETA, vb, (void**)&e));
      if (i == nmass) {
        src[c] = b.chi[nmass];
      } else {
        HMC_TRY(m_launch<double>(b.c, b.c->geo, b.c->delta * masses[i], b.chi[i], nullptr, 0.0, s));
        src[c] = s;
      }
      eta[c] = e;
    }
    return HMC_OK;
  }

  // dS_k/dphi of every chain into its cache slot (level -1: all levels).
  hmc_status level_grad(int k, int slot) {
    HMC_TRACE("force level, all chains");
    HMC_TRY(tables());
    for (BChain& b : ch) {
      double* out = b.cache + (size_t)slot * b.N();
      if (k == nmass || k == -1)
        HMC_TRY(gauss_grad(b.c, b.phi, 0, out));
      else
        HMC_CUDA(b.c, cudaMemsetAsync(out, 0, b.N() * sizeof(double), b.c->stream));
    }
    const int i0 = k < 0 ? 0 : k, i1 = k < 0 ? nmass : k;
    std::vector<const double2*> src;
    std::vector<double2*> eta;
    for (int i = i0; i <= i1; ++i) {
      HMC_TRY(sources(i, src, eta));
      HMC_TRY(solve_all(lower_mass(masses, i), src, eta, o));
      for (size_t c = 0; c < ch.size(); ++c) {
        BChain& b = ch[c];
        double2* xi;
        HMC_TRY(ws_get(b.c, WS_F_XI, sizeof(double2) * b.N(), (void**)&xi));
        HMC_TRY(mdag_launch<double>(b.c, b.c->geo, b.c->delta * lower_mass(masses, i), eta[c], xi));
        HMC_TRY(force_launch(b.c, b.c->geo, eta[c], xi, i == nmass ? nullptr : b.chi[i],
                             b.cache + (size_t)slot * b.N()));
      }
    }
    return HMC_OK;
  }

  void Q(double coef) {
    if (err != HMC_OK) return;
    for (BChain& b : ch) {
      err = axpy_real_launch(b.c, (int)b.N(), coef, b.pi, b.phi);
      if (err != HMC_OK) return;
    }
    ++ver;
  }

  int ensure(int k) {
    const int slot = k < 0 ? nmass + 1 : k;
    if (cache_ver[slot] != ver) {
      err = level_grad(k, slot);
      if (err != HMC_OK) return -1;
      cache_ver[slot] = ver;
    }
    return slot;
  }

  void P(int k, double coef) {
    if (err != HMC_OK) return;
    const int slot = ensure(k);
    if (slot < 0) return;
    for (BChain& b : ch) {
      err = axpy_real_launch(b.c, (int)b.N(), -coef, b.cache + (size_t)slot * b.N(), b.pi);
      if (err != HMC_OK) return;
    }
  }

  // The force-gradient middle kick (Eq. force_cal) for every chain.
  void fg_kick(double coef, double h) {
    if (err != HMC_OK) return;
    const int slot = ensure(-1);
    if (slot < 0) return;
    for (BChain& b : ch) {
      if (!b.phit) {
        err = ws_get(b.c, WS_MD_PHI0, sizeof(double) * b.N(), (void**)&b.phit);
        if (err != HMC_OK) return;
      }
      const cudaError_t e =
          cudaMemcpyAsync(b.phit, b.phi, sizeof(double) * b.N(), cudaMemcpyDeviceToDevice, b.c->stream);
      if (e != cudaSuccess) {
        err = cuda_fail(b.c, e, "force-gradient copy");
        return;
      }
      err = axpy_real_launch(b.c, (int)b.N(), -(h * h / 24.0), b.cache + (size_t)slot * b.N(), b.phit);
      if (err != HMC_OK) return;
      b.phi = b.phit;
    }
    ++ver;
    P(-1, coef);
    for (BChain& b : ch) b.phi = b.phi_home;
    ++ver;
  }
};

bool same_lattice(const hmc_lattice& a, const hmc_lattice& b) {
  return a.n == b.n && a.m == b.m && a.nt == b.nt && a.kappa == b.kappa && a.U == b.U && a.beta == b.beta;
}

}  // namespace
}  // namespace hmc

using namespace hmc;

static hmc_status trajectory_batched(hmc_ctx* ctx, int nchains, const hmc_chain* chains, int nmass,
                                     const double* masses, const hmc_integrator* integ,
                                     const hmc_solver_opts* md_opts, const hmc_solver_opts* action_opts, double* H0,
                                     double* H1, hmc_solve_info* infos);

extern "C" hmc_status hmc_md_trajectory_batched(hmc_ctx* ctx, int nchains, const hmc_chain* chains, int nmass,
                                                const double* masses, const hmc_integrator* integ,
                                                const hmc_solver_opts* md_opts, const hmc_solver_opts* action_opts,
                                                double* H0, double* H1, hmc_solve_info* infos) {
  if (!ctx) return HMC_ERR_INVALID;
  HMC_TRACE("hmc_md_trajectory_batched");
  ctx->err.clear();
  const hmc_status s =
      trajectory_batched(ctx, nchains, chains, nmass, masses, integ, md_opts, action_opts, H0, H1, infos);
  if (s != HMC_OK && ctx->err.empty()) {
    // the failing step ran on a chain's context: report its message here
    for (size_t i = 0; i < ctx->subs.size(); ++i)
      if (ctx->subs[i] && !ctx->subs[i]->err.empty()) {
        ctx->err = "chain " + std::to_string(i) + ": " + ctx->subs[i]->err;
        break;
      }
  }
  return s;
}

static hmc_status trajectory_batched(hmc_ctx* ctx, int nchains, const hmc_chain* chains, int nmass,
                                     const double* masses, const hmc_integrator* integ,
                                     const hmc_solver_opts* md_opts, const hmc_solver_opts* action_opts, double* H0,
                                     double* H1, hmc_solve_info* infos) {
  if (nchains < 1 || !chains || !integ || !md_opts || !action_opts || !H0 || !H1)
    return fail(ctx, HMC_ERR_INVALID, "NULL argument or no chain");
  if (nmass < 0 || nmass > HMC_MAX_MASSES || (nmass > 0 && !masses))
    return fail(ctx, HMC_ERR_INVALID, "nmass out of range or masses NULL");
  for (const hmc_solver_opts* so : {md_opts, action_opts})
    if (so->method < HMC_SOLVER_CG64 || so->method > HMC_SOLVER_FCG_MIXED || !(so->tol > 0.0) || so->maxit < 1)
      return fail(ctx, HMC_ERR_INVALID, "bad solver options");
  if (integ->nmd < 1 || !(integ->tau > 0.0)) return fail(ctx, HMC_ERR_INVALID, "bad nmd or tau");
  std::vector<int> steps;
  if (integ->kind == HMC_INTEG_NESTED_OMELYAN) {
    for (int k = 0; k < nmass; ++k) {
      const int Nk = integ->N[k];
      if (Nk < 1) return fail(ctx, HMC_ERR_INVALID, "time-scale ratio N_k must be >= 1");
      if (k == 0 && integ->nmd % Nk) return fail(ctx, HMC_ERR_INVALID, "N_0 must divide N_MD");
      if (k > 0 && integ->N[k - 1] % Nk) return fail(ctx, HMC_ERR_INVALID, "N_k must divide N_{k-1}");
      steps.push_back(integ->nmd / Nk);
    }
    steps.push_back(integ->nmd);
  } else if (integ->kind != HMC_INTEG_LEAPFROG && integ->kind != HMC_INTEG_FORCE_GRADIENT) {
    return fail(ctx, HMC_ERR_INVALID, "unknown integrator");
  }
  for (int i = 0; i < nchains; ++i) {
    const hmc_chain& y = chains[i];
    if (bad_lattice(&y.lat)) return fail(ctx, HMC_ERR_INVALID, "bad lattice in chain " + std::to_string(i));
    if (!y.phi || !y.pi || !y.rho || ((uintptr_t)y.phi) % 8 || ((uintptr_t)y.pi) % 8)
      return fail(ctx, HMC_ERR_INVALID, "chain " + std::to_string(i) + ": NULL or misaligned phi, pi or rho");
    for (int k = 0; k <= nmass; ++k)
      if (!y.rho[k] || ((uintptr_t)y.rho[k]) % 16)
        return fail(ctx, HMC_ERR_INVALID, "chain " + std::to_string(i) + ": rho entry NULL or misaligned");
  }
  // one context per chain, kept for the next call while the lattice stays
  if ((int)ctx->subs.size() < nchains) ctx->subs.resize(nchains, nullptr);
  std::vector<BChain> ch(nchains);
  for (int i = 0; i < nchains; ++i) {
    hmc_ctx*& sc = ctx->subs[i];
    if (sc && !same_lattice(sc->lat, chains[i].lat)) {
      hmc_destroy(sc);
      sc = nullptr;
    }
    if (!sc) {
      const hmc_status s = hmc_create(&sc, &chains[i].lat, ctx->stream);
      if (s != HMC_OK) return fail(ctx, s, "per-chain context creation failed");
    }
    sc->stream = ctx->stream;
    sc->err.clear();
    HMC_TRY(check_masses(sc, nmass, masses));
    BChain& b = ch[i];
    b.c = sc;
    b.phi = b.phi_home = chains[i].phi;
    b.pi = chains[i].pi;
    for (int k = 0; k <= nmass; ++k) b.rho[k] = (const double2*)chains[i].rho[k];
    const size_t N = b.N();
    double2* chibuf;
    HMC_TRY(ws_get(sc, WS_MD_CHI, sizeof(double2) * N * (nmass + 1), (void**)&chibuf));
    HMC_TRY(ws_get(sc, WS_MD_FORCE, sizeof(double) * N * (nmass + 2), (void**)&b.cache));
    for (int k = 0; k <= nmass; ++k) b.chi[k] = chibuf + k * N;
  }
  BatchMD md{ctx, ch, nmass, masses, md_opts};
  md.cache_ver.assign(nmass + 2, -1);

  // pseudofermions from rho at the starting fields (Section 5.1):
  //   chi_i = M_{mu_i}^dagger (M_{mu_i} M_{mu_i}^dagger)^{-1} M_{mu_{i-1}} rho_i,  chi_n = M_{mu_{n-1}} rho_n
  HMC_TRY(md.tables());
  {
    std::vector<const double2*> src(nchains);
    std::vector<double2*> y(nchains);
    for (int i = 0; i < nmass; ++i) {
      for (int c = 0; c < nchains; ++c) {
        BChain& b = ch[c];
        const size_t vb = sizeof(double2) * b.N();
        double2 *s, *e;
        HMC_TRY(ws_get(b.c, WS_F_SRC, vb, (void**)&s));
        HMC_TRY(ws_get(b.c, WS_F_ETA, vb, (void**)&e));
        HMC_TRY(m_launch<double>(b.c, b.c->geo, b.c->delta * lower_mass(masses, i), b.rho[i], nullptr, 0.0, s));
        src[c] = s;
        y[c] = e;
      }
      HMC_TRY(md.solve_all(masses[i], src, y, action_opts));
      for (int c = 0; c < nchains; ++c)
        HMC_TRY(mdag_launch<double>(ch[c].c, ch[c].c->geo, ch[c].c->delta * masses[i], y[c], ch[c].chi[i]));
    }
    const double top = nmass > 0 ? masses[nmass - 1] : 0.0;
    for (BChain& b : ch)
      HMC_TRY(m_launch<double>(b.c, b.c->geo, b.c->delta * top, b.rho[nmass], nullptr, 0.0, b.chi[nmass]));
  }

  // H0 = phi^2/(2 delta U) + sum rho^dagger rho + pi^2/2, per chain
  for (BChain& b : ch) {
    const double inv_dU = 1.0 / (b.c->delta * b.c->lat.U);
    HMC_TRY(half_sq_launch(b.c, (int)b.N(), b.phi, inv_dU, b.pi, b.c->dscal + 54, b.c->tickets));
    for (int i = 0; i <= nmass; ++i)
      HMC_TRY(norm2_launch(b.c, (int)b.N(), b.rho[i], b.c->dscal + 56 + i, b.c->tickets));
    HMC_CUDA(b.c, cudaMemcpyAsync(b.c->dscal_host + 54, b.c->dscal + 54, sizeof(double) * (2 + nmass + 1),
                                  cudaMemcpyDeviceToHost, b.c->stream));
  }
  HMC_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
  for (int c = 0; c < nchains; ++c) {
    const double* d = ch[c].c->dscal_host;
    double h0 = d[54] + d[55];
    for (int i = 0; i <= nmass; ++i) h0 += d[56 + i];
    H0[c] = h0;
  }

  // molecular dynamics, all chains in lockstep
  run_integrator(md, integ->kind, steps, integ->nmd, integ->zeta, integ->tau);
  if (md.err != HMC_OK) return md.err;

  // H1 = S(phi') + pi'^2/2 with the action solves at action_opts' tolerance,
  // each S_i in the stationary form 2 Re(src^dagger eta) - |M_lo^dagger eta|^2
  HMC_TRY(md.tables());
  std::vector<double> h1(nchains, 0.0);
  {
    std::vector<const double2*> src;
    std::vector<double2*> eta;
    for (int i = 0; i <= nmass; ++i) {
      HMC_TRY(md.sources(i, src, eta));
      HMC_TRY(md.solve_all(lower_mass(masses, i), src, eta, action_opts, true));
      for (int c = 0; c < nchains; ++c) {
        BChain& b = ch[c];
        double2* xi;
        HMC_TRY(ws_get(b.c, WS_F_XI, sizeof(double2) * b.N(), (void**)&xi));
        HMC_TRY(mdag_launch<double>(b.c, b.c->geo, b.c->delta * lower_mass(masses, i), eta[c], xi));
        HMC_TRY(redot_launch(b.c, b.c->geo.N, src[c], eta[c], b.c->dscal + 100, b.c->tickets));
        HMC_TRY(norm2_launch(b.c, b.c->geo.N, xi, b.c->dscal + 101, b.c->tickets));
        HMC_CUDA(b.c, cudaMemcpyAsync(b.c->dscal_host + 100, b.c->dscal + 100, 2 * sizeof(double),
                                      cudaMemcpyDeviceToHost, b.c->stream));
      }
      HMC_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
      for (int c = 0; c < nchains; ++c) h1[c] += 2.0 * ch[c].c->dscal_host[100] - ch[c].c->dscal_host[101];
    }
  }
  for (BChain& b : ch) {
    const double inv_dU = 1.0 / (b.c->delta * b.c->lat.U);
    HMC_TRY(half_sq_launch(b.c, (int)b.N(), b.phi, inv_dU, b.pi, b.c->dscal + 54, b.c->tickets));
    HMC_CUDA(b.c, cudaMemcpyAsync(b.c->dscal_host + 54, b.c->dscal + 54, sizeof(double) * 2, cudaMemcpyDeviceToHost,
                                  b.c->stream));
  }
  HMC_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
  for (int c = 0; c < nchains; ++c) {
    H1[c] = h1[c] + ch[c].c->dscal_host[54] + ch[c].c->dscal_host[55];
    if (infos) {
      const SolveStats& s = ch[c].st;
      hmc_solve_info& f = infos[c];
      std::memset(&f, 0, sizeof(f));
      f.iters = s.iters;
      f.iters_outer = s.outer;
      f.iters_inner = s.inner;
      f.status = HMC_OK;
      f.true_rel_res = s.true_rel;
      f.applies64 = s.applies64;
      f.applies32 = s.applies32;
      f.bytes = (long long)((double)ch[c].N() * (192.0 * s.applies64 + 96.0 * s.applies32));
    }
  }
  return HMC_OK;
}
