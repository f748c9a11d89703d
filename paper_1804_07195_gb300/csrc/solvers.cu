// Krylov solvers for A x = b, A = M_ms M_ms^dagger + sigma (Section 3 and
// Algorithm A.1): CG in FP64 or FP32, and flexible GMRES with an FP32 CG
// preconditioner. The iteration runs on the device; the host checks the
// convergence flag every few iterations and only reads back small scalars.
#include <cmath>
#include <complex>
#include <vector>

#include "solvers.h"

namespace hmc {

hmc_solver_opts default_opts() {
  hmc_solver_opts o;
  o.method = HMC_SOLVER_FGMRES_MIXED;
  o.tol = 1e-10;
  o.maxit = 100000;
  o.restart = 10;
  o.a = 5.0;
  o.inner_floor = 1e-6;
  o.inner_maxit = 2000;
  return o;
}

void add_stats(hmc_solve_info* info, const SolveStats& s) {
  if (!info) return;
  info->iters += s.iters;
  info->iters_outer += s.outer;
  info->iters_inner += s.inner;
  info->applies64 += s.applies64;
  info->applies32 += s.applies32;
  info->true_rel_res = s.true_rel;
}

template <typename R>
static hmc_status vec_slots(hmc_ctx* c, V2<R>** r, V2<R>** p, V2<R>** u) {
  const size_t bytes = sizeof(V2<R>) * (size_t)c->geo.N;
  const bool d = sizeof(R) == 8;
  HMC_TRY(ws_get(c, d ? WS_CG_R64 : WS_CG_R32, bytes, (void**)r));
  HMC_TRY(ws_get(c, d ? WS_CG_P64 : WS_CG_P32, bytes, (void**)p));
  HMC_TRY(ws_get(c, d ? WS_U64 : WS_U32, bytes, (void**)u));
  return HMC_OK;
}

// Launch-shape autotuner of the CG kernels of one precision: every candidate
// (threads per block x grid waves, the same for all kernels of the iteration)
// runs a few timed iterations on scratch vectors with this solve's right-hand
// side; the fastest is kept for the context. Runs once per context and
// precision. Results of later solves are reproducible for the chosen shape
// (the shape fixes the reduction order).
template <typename R>
hmc_status cg_core(hmc_ctx* c, double ms, double sigma, const V2<R>* b, V2<R>* x, bool x_zero,
                   double tol, int maxit, int sc_slot, bool want_true_res, SolveStats* st);

template <typename R>
static hmc_status tune_cg(hmc_ctx* c, double ms, double sigma, const V2<R>* b) {
  bool& done = sizeof(R) == 4 ? c->tuned32 : c->tuned64;
  if (done) return HMC_OK;
  done = true;
  const Geo& g = c->geo;
  const size_t bytes = sizeof(V2<R>) * (size_t)g.N;
  V2<R> *r, *p, *u, *x, *q = nullptr;
  HMC_TRY(vec_slots<R>(c, &r, &p, &u));
  HMC_TRY(ws_get(c, sizeof(R) == 4 ? WS_CG_X32 : WS_CG_X64, bytes, (void**)&x));
  if (sizeof(R) == 4) HMC_TRY(ws_get(c, WS_CG_Q32, bytes, (void**)&q));
  CGScal* sc = c->sc + 2;
  unsigned* tk = c->tickets;
  const int ids32[2] = {K_CG_MDAG32, K_CG_M32};
  const int ids64[3] = {K_CG_MDAG64, K_CG_M64, K_CG_P64};
  const int* ids = sizeof(R) == 4 ? ids32 : ids64;
  const int nk = sizeof(R) == 4 ? 2 : 3;
  auto iter = [&](int n) -> hmc_status {
    for (int i = 0; i < n; ++i) {
      if constexpr (sizeof(R) == 4) {
        float2* po = (i & 1) ? (float2*)q : (float2*)p;
        float2* pn = (i & 1) ? (float2*)p : (float2*)q;
        HMC_TRY(cg32_pmdag_launch(c, g, (const float2*)r, po, pn, (float2*)u, sc, tk));
        HMC_TRY(cg32_m_launch(c, g, (const float2*)u, pn, (float2*)x, (float2*)r, sc, tk));
      } else {
        HMC_TRY(cg_mdag_launch<R>(c, g, p, u, sc, tk));
        HMC_TRY(cg_m_launch<R>(c, g, u, p, x, r, sc, tk));
        HMC_TRY(cg_p_launch<R>(c, g.N, r, p, sc));
      }
    }
    return HMC_OK;
  };
  cudaEvent_t e0, e1;
  HMC_CUDA(c, cudaEventCreate(&e0));
  HMC_CUDA(c, cudaEventCreate(&e1));
  // candidates: {threads, waves, tiled, time slices per tile}
  std::vector<Shape> cands;
  const int var = c->cg32_variant;
  const bool want_tiled = sizeof(R) == 4 && (var == 0 || var == 2 || var == 3 || var == 4);
  if (want_tiled && var != 3)
    for (int tc : {256, 512, 1024})
      for (int tt : {2, 4, 8})
        if (cg32_tiled_ok(c, g, tc, tt)) {
          Shape sh;
          sh.threads = tc;
          sh.tiled = 1;
          sh.tt = tt;
          cands.push_back(sh);
        }
  if (want_tiled && var != 2)
    for (int th : {128, 256, 512})
      for (int tt : {2, 4, 8})
        if (cg32_march_ok(c, g, th, tt)) {
          Shape sh;
          sh.threads = th;
          sh.tiled = 2;
          sh.tt = tt;
          cands.push_back(sh);
        }
  // variants 2 and 3 keep the grid-stride candidates only where none of theirs fits
  // (variant 5, two cells per thread, falls back to variant 1 where n is odd)
  if (!(sizeof(R) == 4 && var >= 2 && var <= 4 && !cands.empty()))
    for (int pairs : {0, 1})
      for (int th : {128, 256, 512})
        for (int wv : {1, 2, 4, 0}) {
          const bool pairs_ok = sizeof(R) == 4 && !(g.n & 1);
          if (pairs && !(pairs_ok && (var == 0 || var == 5))) continue;
          if (!pairs && sizeof(R) == 4 && var == 5 && pairs_ok) continue;
          Shape sh;
          sh.threads = th;
          sh.waves = wv;
          sh.tiled = pairs ? 4 : 0;
          cands.push_back(sh);
        }
  float best = 1e30f;
  Shape keep[3];
  // the fastest shape of each kernel family (tiled: 0 grid-stride, 1 tiled,
  // 2 marching, 4 grid-stride with two cells per thread)
  float fam_t[5] = {1e30f, 1e30f, 1e30f, 1e30f, 1e30f};
  Shape fam[5][3];
  for (const Shape& cand : cands) {
    {
      for (int k = 0; k < nk; ++k) {
        Shape& sh = c->shape[ids[k]];
        sh = cand;
        sh.occ = (cand.tiled && cand.tiled != 4) ? 1 : cg_kernel_occupancy(ids[k], cand.threads, cand.tiled == 4);
      }
      // tolerance 0: no candidate stops early
      HMC_TRY(init0_launch<R>(c, g.N, b, x, r, p, sc, 0.0, 1 << 30, sigma, tk, c->delta * ms));
      HMC_TRY(iter(2));
      HMC_CUDA(c, cudaEventRecord(e0, c->stream));
      HMC_TRY(iter(4));
      HMC_CUDA(c, cudaEventRecord(e1, c->stream));
      HMC_CUDA(c, cudaEventSynchronize(e1));
      float ms_ = 0.f;
      cudaEventElapsedTime(&ms_, e0, e1);
      if (ms_ < best) {
        best = ms_;
        for (int k = 0; k < nk; ++k) keep[k] = c->shape[ids[k]];
      }
      const int f = cand.tiled;
      if (f >= 0 && f < 5 && ms_ < fam_t[f]) {
        fam_t[f] = ms_;
        for (int k = 0; k < nk; ++k) fam[f][k] = c->shape[ids[k]];
      }
    }
  }
  for (int k = 0; k < nk; ++k) c->shape[ids[k]] = keep[k];
  // FP32: the single-reduction kernel's tile (variants 0 and 6), then the
  // designs against each other through the solver path they would run in
  // (graph replay with programmatic dependent launch; 48 iterations, twice
  // each, best kept): the fastest pair of each kernel family (timed above
  // with plain launches, which rank the families differently), the
  // persistent kernel, the single-reduction kernel
  if constexpr (sizeof(R) == 4) {
    c->persist32 = false;
    c->cg1_32 = false;
    c->resident32 = false;
    bool cg1_fit = false;
    if ((var == 0 || var == 6) && !c->capturing) {
      const CG1Bufs B = cg1_bufs(c, (float2*)r);
      if (B.r[1] != nullptr) {
        if (c->cg1_pinned)
          cg1_fit = cg1_ok(c, g, c->cg1_shape);
        else
          cg1_fit = cg1_tune(c, g, B, (float2*)p, (float2*)x, sc, [&] {
            return init0_launch<R>(c, g.N, b, x, r, p, sc, 0.0, 1 << 30, sigma, tk, c->delta * ms);
          });
      }
      HMC_CUDA(c, cudaGetLastError());
      c->err.clear();
    }
    if (var == 6) c->cg1_32 = cg1_fit;
    if (var == 0 && !c->capturing) {
      struct Design {
        bool persist, cg1, resident;
        int fam;  // pair family whose shapes the design runs (-1: the overall fastest)
      };
      std::vector<Design> designs;
      for (int f = 0; f < 5; ++f)
        if (fam_t[f] < 1e30f) designs.push_back({false, false, false, f});
      if (designs.empty()) designs.push_back({false, false, false, -1});
      if (cg32_persist_ok(c, g)) designs.push_back({true, false, false, -1});
      if (cg1_fit) designs.push_back({false, true, false, -1});
      if (cg32_resident_ok(c, g)) designs.push_back({false, false, true, -1});
      auto use_shapes = [&](int f) {
        for (int k = 0; k < nk; ++k) c->shape[ids[k]] = f >= 0 ? fam[f][k] : keep[k];
      };
      float best_t = 1e30f;
      Design best_d = designs[0];
      for (size_t k = 0; designs.size() > 1 && k < designs.size(); ++k) {
        c->persist32 = designs[k].persist;
        c->cg1_32 = designs[k].cg1;
        c->resident32 = designs[k].resident;
        use_shapes(designs[k].fam);
        destroy_graphs(c);  // graphs hold the launch shapes they were captured with
        float tm = 1e30f;
        for (int rep = 0; rep < 2; ++rep) {
          SolveStats tmp;
          HMC_CUDA(c, cudaEventRecord(e0, c->stream));
          const hmc_status st = cg_core<R>(c, ms, sigma, b, x, true, 1e-30, 48, 2, false, &tmp);
          HMC_CUDA(c, cudaEventRecord(e1, c->stream));
          HMC_CUDA(c, cudaEventSynchronize(e1));
          if (st != HMC_OK && st != HMC_ERR_NOT_CONVERGED) {
            c->persist32 = false;
            c->cg1_32 = false;
            c->resident32 = false;
            cudaEventDestroy(e0);
            cudaEventDestroy(e1);
            return st;
          }
          c->err.clear();
          float t = 0.f;
          cudaEventElapsedTime(&t, e0, e1);
          tm = std::min(tm, t);
        }
        if (tm < best_t) {
          best_t = tm;
          best_d = designs[k];
        }
      }
      c->persist32 = best_d.persist;
      c->cg1_32 = best_d.cg1;
      c->resident32 = best_d.resident;
      use_shapes(best_d.fam);
      destroy_graphs(c);
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  return HMC_OK;
}

template <typename R>
hmc_status cg_core(hmc_ctx* c, double ms, double sigma, const V2<R>* b, V2<R>* x, bool x_zero,
                   double tol, int maxit, int sc_slot, bool want_true_res, SolveStats* st) {
  const Geo& g = c->geo;
  if (!c->capturing) HMC_TRY(tune_cg<R>(c, ms, sigma, b));
  const R dm = (R)(c->delta * ms);
  V2<R> *r, *p, *u;
  HMC_TRY(vec_slots<R>(c, &r, &p, &u));
  CGScal* sc = c->sc + sc_slot;
  CGScal* sch = c->sc_host + sc_slot;
  unsigned* tk = c->tickets;
  const double tol2 = tol * tol;
  const double ddm = c->delta * ms;
  if (x_zero) {
    HMC_TRY(init0_launch<R>(c, g.N, b, x, r, p, sc, tol2, maxit, sigma, tk, ddm));
  } else {
    HMC_TRY(mdag_launch<R>(c, g, dm, x, u));
    HMC_TRY(resid_launch<R>(c, g, dm, u, x, b, sigma, r, p, sc, tol2, maxit, nullptr, tk, ddm));
    if (sizeof(R) == 8) st->applies64++; else st->applies32++;
  }
  // FP32: two kernels per iteration with a second direction buffer q
  // (p and q alternate as p_old / p_new); every chunk has an even length, so
  // the newest direction is in p whenever a chunk ends.
  V2<R>* q = nullptr;
  if (sizeof(R) == 4)
    HMC_TRY(ws_get(c, WS_CG_Q32, sizeof(V2<R>) * (size_t)g.N, (void**)&q));
  bool single = false;  // FP32 single-reduction design (decided below)
  CG1Bufs B{};
  auto iterate = [&](int n) -> hmc_status {
    for (int i = 0; i < n; ++i) {
      if constexpr (sizeof(R) == 4) {
        if (single) {
          HMC_TRY(cg1_iter_launch(c, g, B, (float2*)p, (float2*)x, sc, i & 1));
          continue;
        }
        float2* pold = (i & 1) ? (float2*)q : (float2*)p;
        float2* pnew = (i & 1) ? (float2*)p : (float2*)q;
        HMC_TRY(cg32_pmdag_launch(c, g, (const float2*)r, pold, pnew, (float2*)u, sc, tk));
        HMC_TRY(cg32_m_launch(c, g, (const float2*)u, pnew, (float2*)x, (float2*)r, sc, tk));
      } else {
        HMC_TRY(cg_mdag_launch<R>(c, g, p, u, sc, tk));
        HMC_TRY(cg_m_launch<R>(c, g, u, p, x, r, sc, tk));
        HMC_TRY(cg_p_launch<R>(c, g.N, r, p, sc));
      }
    }
    return HMC_OK;
  };
  // Iterations run in chunks of kChunk, replayed from a captured CUDA graph
  // (one per buffer set) unless per-kernel timing is on; the host reads the
  // state after 1, 1, 2, 4, 4, ... chunks.
  constexpr int kChunk = 8;
  // FP32: the whole solve in one persistent launch when the tuner (or the
  // pinned variant) chose it
  bool persistent = false;
  if constexpr (sizeof(R) == 4) {
    // the resident-tile kernel (one launch per solve, p and M^dagger p of
    // each tile in shared memory) when the tuner or the pinned variant chose it
    const bool resident = !c->capturing &&
                          (c->cg32_variant == 7 || (c->cg32_variant == 0 && c->resident32)) &&
                          cg32_resident_ok(c, g);
    persistent = resident || (!c->capturing && (c->cg32_variant == 4 || (c->cg32_variant == 0 && c->persist32)) &&
                              cg32_persist_ok(c, g));
    if (persistent) {
      if (resident)
        HMC_TRY(cg32_resident_launch(c, g, (float2*)x, (float2*)r, (float2*)p, (float2*)q, (float2*)u, sc));
      else
        HMC_TRY(cg32_persist_launch(c, g, (float2*)x, (float2*)r, (float2*)p, (float2*)q, (float2*)u, sc));
      HMC_CUDA(c, cudaMemcpyAsync(sch, sc, sizeof(CGScal), cudaMemcpyDeviceToHost, c->stream));
      HMC_CUDA(c, cudaStreamSynchronize(c->stream));
      // the algorithmic bytes of one FP32 CG iteration per site, whatever the
      // design keeps on chip: the operator with its dot (p and phi read, A p
      // written: 20 B, here rounded with the dot to 24 B), x and r updated
      // with the norm (48 B), p updated (24 B)
      c->prof.bytes[resident ? K_CG_RES32 : K_CG_PERSIST32] += 96.0 * g.N * sch->iter;
    }
  }
  // FP32: one single-reduction launch per iteration when the tuner (or the
  // pinned variant) chose it; it starts from w_0 = A r_0
  if constexpr (sizeof(R) == 4) {
    single = !persistent && (c->cg32_variant == 0 || c->cg32_variant == 6) && c->cg1_32 &&
             cg1_ok(c, g, c->cg1_shape);
    if (single) {
      B = cg1_bufs(c, (float2*)r);
      if (B.r[1] == nullptr) return fail(c, HMC_ERR_NOMEM, "single-reduction CG vectors");
      HMC_TRY(cg1_prime_launch(c, g, B, (float2*)p, (float2*)x, sc));
      st->applies32++;
    }
  }
  int kid[3] = {sizeof(R) == 4 ? K_CG_MDAG32 : K_CG_MDAG64, sizeof(R) == 4 ? K_CG_M32 : K_CG_M64, K_CG_P64};
  double kbytes[3] = {sizeof(R) == 4 ? 36.0 : 48.0, sizeof(R) == 4 ? 52.0 : 112.0, 48.0};
  int nk = sizeof(R) == 4 ? 2 : 3;
  if (single) {
    kid[0] = K_CG1_32;
    kbytes[0] = kKernelBytesPerSite[K_CG1_32];
    nk = 1;
  }
  // The whole solve as one graph launch: chunks of kChunk iterations repeated
  // by a device-side while loop until the done flag is set (or the trip bound,
  // maxit / kChunk + 2, is reached); the host waits once, at the end.
  bool looped = false;
  if (!persistent && c->use_graphs && c->use_loop_graphs && !c->prof.timing && !c->capturing) {
    const void* key[6] = {sc, r, p, q, u, x};
    const int kind = (sizeof(R) == 4 ? 32 : 64) + 1000 + (single ? 500 : 0);
    GraphEntry* le = find_graph(c, kind, key);
    if (!le) {
      cudaGraphExec_t exec;
      if (capture_loop_graph(c, [&](cudaGraphConditionalHandle h) -> hmc_status {
            HMC_TRY(iterate(kChunk));
            return loop_continue_launch(c, h, sc);
          }, &exec) == HMC_OK) {
        le = add_graph(c, kind, key, exec);
      } else {
        c->use_loop_graphs = false;  // chunked replay from now on
        c->err.clear();
      }
    }
    if (le) {
      c->loop_trips_host[0] = 0u;
      c->loop_trips_host[1] = (unsigned)(maxit / kChunk + 2);
      HMC_CUDA(c, cudaMemcpyAsync(c->loop_trips, c->loop_trips_host, 2 * sizeof(unsigned), cudaMemcpyHostToDevice,
                                  c->stream));
      HMC_CUDA(c, cudaGraphLaunch(le->exec, c->stream));
      HMC_CUDA(c, cudaMemcpyAsync(sch, sc, sizeof(CGScal), cudaMemcpyDeviceToHost, c->stream));
      HMC_CUDA(c, cudaMemcpyAsync(c->loop_trips_host, c->loop_trips, sizeof(unsigned), cudaMemcpyDeviceToHost,
                                  c->stream));
      HMC_CUDA(c, cudaStreamSynchronize(c->stream));
      // the loop ran trips x kChunk iterations, of which sch->iter did work
      // (the rest found the done flag set and returned at entry)
      const double its = (double)sch->iter;
      for (int k = 0; k < nk; ++k) {
        c->prof.launches[kid[k]] += (long long)its;
        c->prof.bytes[kid[k]] += its * kbytes[k] * g.N;
      }
      looped = true;
    }
  }
  GraphEntry* ge = nullptr;
  if (!persistent && !looped && c->use_graphs && !c->prof.timing) {
    const void* key[6] = {sc, r, p, q, u, x};
    const int kind = (sizeof(R) == 4 ? 32 : 64) + (single ? 500 : 0);
    ge = find_graph(c, kind, key);
    if (!ge) {
      cudaGraphExec_t exec;
      if (capture_graph(c, [&] { return iterate(kChunk); }, &exec) == HMC_OK) {
        ge = add_graph(c, kind, key, exec);
      } else {
        c->use_graphs = false;  // launch the same kernels one by one from now on
        c->err.clear();
      }
    }
  }
  int per_check = 1, checks = 0;
  long long launched = 0;
  for (; !persistent && !looped;) {
    for (int i = 0; i < per_check; ++i) {
      if (ge) {
        HMC_CUDA(c, cudaGraphLaunch(ge->exec, c->stream));
        for (int k = 0; k < nk; ++k) {
          c->prof.launches[kid[k]] += kChunk;
          c->prof.bytes[kid[k]] += kChunk * kbytes[k] * g.N;
        }
      } else {
        HMC_TRY(iterate(kChunk));
      }
    }
    launched += (long long)per_check * kChunk;
    HMC_CUDA(c, cudaMemcpyAsync(sch, sc, sizeof(CGScal), cudaMemcpyDeviceToHost, c->stream));
    HMC_CUDA(c, cudaStreamSynchronize(c->stream));
    if (sch->done != CG_RUNNING) break;
    if (launched > (long long)maxit + 2 * kChunk) break;  // cannot happen: the device stops at maxit
    // with per-launch timing on, check after every chunk so that few launches
    // run past convergence
    if (++checks >= 2 && per_check < 4 && !c->prof.timing) per_check *= 2;
  }
  // Launches after convergence return at entry: drop them from the counters,
  // the algorithmic bytes and the per-launch timings, so these cover exactly
  // the sch->iter iterations that ran.
  if (!persistent && !looped)
    for (int k = 0; k < nk; ++k) prof_discard_last(c, kid[k], launched - (long long)sch->iter, kbytes[k] * g.N);
  st->iters += sch->iter;
  if (sizeof(R) == 8) st->applies64 += sch->iter; else st->applies32 += sch->iter;
  st->cg_done = sch->done;
  if (want_true_res) {
    HMC_TRY(mdag_launch<R>(c, g, dm, x, u));
    HMC_TRY(resid_launch<R>(c, g, dm, u, x, b, sigma, r, nullptr, nullptr, 0.0, 0, c->dscal, tk, ddm));
    HMC_CUDA(c, cudaMemcpyAsync(c->dscal_host, c->dscal, 2 * sizeof(double),
                                cudaMemcpyDeviceToHost, c->stream));
    HMC_CUDA(c, cudaStreamSynchronize(c->stream));
    const double rr = c->dscal_host[0], bb = c->dscal_host[1];
    st->true_rel = bb > 0 ? std::sqrt(rr / bb) : 0.0;
    if (sizeof(R) == 8) st->applies64++; else st->applies32++;
  }
  if (sch->done == CG_TIMEOUT) return fail(c, HMC_ERR_TIMEOUT, "persistent CG: a grid barrier wait gave up");
  if (sch->done == CG_BREAKDOWN) return fail(c, HMC_ERR_NAN, "CG breakdown: non-positive or non-finite curvature/residual");
  if (sch->done == CG_MAXIT) return fail(c, HMC_ERR_NOT_CONVERGED, "CG reached its iteration limit");
  return HMC_OK;
}

template hmc_status cg_core<double>(hmc_ctx*, double, double, const double2*, double2*, bool, double,
                                    int, int, bool, SolveStats*);
template hmc_status cg_core<float>(hmc_ctx*, double, double, const float2*, float2*, bool, double,
                                   int, int, bool, SolveStats*);

hmc_status apply_A64(hmc_ctx* c, double ms, double sigma, const double2* in, double2* out) {
  double2* u;
  HMC_TRY(ws_get(c, WS_U64, sizeof(double2) * (size_t)c->geo.N, (void**)&u));
  const double dm = c->delta * ms;
  HMC_TRY(mdag_launch<double>(c, c->geo, dm, in, u));
  return m_launch<double>(c, c->geo, dm, u, sigma != 0.0 ? in : nullptr, sigma, out);
}

// Solve the small least-squares problem of Algorithm A.1 through the normal
// equations (h^H h) y = |r| h^H e1 with a Cholesky factorisation (Appendix A).
// h is (k+1) x k, column-major in H[i + j*(ldh)].
static bool normal_eq_cholesky(const std::vector<std::complex<double>>& H, int ldh, int k,
                               double rnorm, std::vector<std::complex<double>>& y) {
  using cd = std::complex<double>;
  std::vector<cd> G((size_t)k * k), rhs(k);
  for (int a = 0; a < k; ++a) {
    for (int b = 0; b < k; ++b) {
      cd s = 0;
      for (int i = 0; i <= k; ++i) s += std::conj(H[i + a * ldh]) * H[i + b * ldh];
      G[a + b * k] = s;
    }
    rhs[a] = rnorm * std::conj(H[0 + a * ldh]);
  }
  // G = L L^H
  std::vector<cd> L((size_t)k * k, 0.0);
  for (int j = 0; j < k; ++j) {
    double d = std::real(G[j + j * k]);
    for (int p = 0; p < j; ++p) d -= std::norm(L[j + p * k]);
    if (!(d > 0.0)) return false;
    const double ljj = std::sqrt(d);
    L[j + j * k] = ljj;
    for (int i = j + 1; i < k; ++i) {
      cd s = G[i + j * k];
      for (int p = 0; p < j; ++p) s -= L[i + p * k] * std::conj(L[j + p * k]);
      L[i + j * k] = s / ljj;
    }
  }
  std::vector<cd> z(k);
  for (int i = 0; i < k; ++i) {
    cd s = rhs[i];
    for (int p = 0; p < i; ++p) s -= L[i + p * k] * z[p];
    z[i] = s / L[i + i * k];
  }
  y.assign(k, 0.0);
  for (int i = k - 1; i >= 0; --i) {
    cd s = z[i];
    for (int p = i + 1; p < k; ++p) s -= std::conj(L[p + i * k]) * y[p];
    y[i] = s / std::real(L[i + i * k]);
  }
  return true;
}

// Preconditioner solve z = A^{-1} v to relative tolerance t in precision prec
// (32: spCG through float copies; 64: FP64 CG). t >= 1 gives z = v.
hmc_status precondition_solve(hmc_ctx* c, double ms, double sigma, const double2* v64,
                               const float2* v32, double2* z, double t, int prec, int inner_maxit,
                               SolveStats* st) {
  const int N = c->geo.N;
  if (t >= 1.0) {
    HMC_CUDA(c, cudaMemcpyAsync(z, v64, sizeof(double2) * N, cudaMemcpyDeviceToDevice, c->stream));
    return HMC_OK;
  }
  SolveStats in;
  hmc_status s;
  if (prec == 32) {
    float2 *b32, *x32;
    HMC_TRY(ws_get(c, WS_CG_B32, sizeof(float2) * N, (void**)&b32));
    HMC_TRY(ws_get(c, WS_CG_X32, sizeof(float2) * N, (void**)&x32));
    if (v32 == nullptr) {
      HMC_TRY(to32_launch(c, N, v64, b32));
      v32 = b32;
    }
    s = cg_core<float>(c, ms, sigma, v32, x32, true, t, inner_maxit, 1, false, &in);
    if (s != HMC_OK && s != HMC_ERR_NOT_CONVERGED) return s;
    HMC_TRY(to64_launch(c, N, x32, z));
  } else {
    s = cg_core<double>(c, ms, sigma, v64, z, true, t, inner_maxit, 1, false, &in);
    if (s != HMC_OK && s != HMC_ERR_NOT_CONVERGED) return s;
  }
  c->err.clear();
  st->inner += in.iters;
  st->applies32 += in.applies32;
  st->applies64 += in.applies64;
  return HMC_OK;
}

hmc_status fgmres_core(hmc_ctx* c, double ms, double sigma, const double2* b, double2* x, double tol,
                       int restart, double a, int inner_prec, int maxit, double inner_floor,
                       int inner_maxit, SolveStats* st) {
  using cd = std::complex<double>;
  const Geo& g = c->geo;
  const int N = g.N;
  const double dm = c->delta * ms;
  const size_t vb = sizeof(double2) * (size_t)N;
  double2 *r, *w, *u, *Vb, *Zb;
  float2* v32 = nullptr;
  HMC_TRY(ws_get(c, WS_FG_R, vb, (void**)&r));
  HMC_TRY(ws_get(c, WS_FG_W, vb, (void**)&w));
  HMC_TRY(ws_get(c, WS_U64, vb, (void**)&u));
  HMC_TRY(ws_get(c, WS_FG_V, vb * restart, (void**)&Vb));
  HMC_TRY(ws_get(c, WS_FG_Z, vb * restart, (void**)&Zb));
  if (inner_prec == 32) HMC_TRY(ws_get(c, WS_CG_B32, sizeof(float2) * N, (void**)&v32));
  unsigned* tk = c->tickets;
  double* hdev = c->dscal;            // 2*restart doubles: h column; then |w|^2 at [40]
  double* hhost = c->dscal_host;

  // |b|
  HMC_TRY(norm2_launch(c, N, b, hdev + 40, tk));
  HMC_CUDA(c, cudaMemcpyAsync(hhost + 40, hdev + 40, sizeof(double), cudaMemcpyDeviceToHost, c->stream));
  HMC_CUDA(c, cudaStreamSynchronize(c->stream));
  const double bnorm = std::sqrt(hhost[40]);
  if (!std::isfinite(bnorm)) return fail(c, HMC_ERR_NAN, "FGMRES: right-hand side is not finite");
  if (bnorm == 0.0) {
    HMC_CUDA(c, cudaMemsetAsync(x, 0, vb, c->stream));
    st->true_rel = 0.0;
    return HMC_OK;
  }
  // first line of Algorithm A.1: spCG solve of A x = b (tolerance tol*a, floored)
  HMC_TRY(precondition_solve(c, ms, sigma, b, nullptr, x, std::max(tol * a, inner_floor), inner_prec,
                       inner_maxit, st));
  if (tol * a >= 1.0) HMC_CUDA(c, cudaMemsetAsync(x, 0, vb, c->stream));
  // r = b - A x, ERR = |r|
  auto true_residual = [&](double* err) -> hmc_status {
    HMC_TRY(mdag_launch<double>(c, g, dm, x, u));
    HMC_TRY(resid_launch<double>(c, g, dm, u, x, b, sigma, r, nullptr, nullptr, 0.0, 0, hdev + 40, tk));
    HMC_CUDA(c, cudaMemcpyAsync(hhost + 40, hdev + 40, 2 * sizeof(double), cudaMemcpyDeviceToHost, c->stream));
    HMC_CUDA(c, cudaStreamSynchronize(c->stream));
    st->applies64++;
    *err = std::sqrt(hhost[40]);
    return HMC_OK;
  };
  double err;
  HMC_TRY(true_residual(&err));
  if (!std::isfinite(err)) return fail(c, HMC_ERR_NAN, "FGMRES: residual is not finite");
  int arnoldi = 0;
  const int ldh = restart + 1;
  std::vector<cd> H((size_t)ldh * restart), gvec(restart + 1), rs(restart);
  std::vector<double> rc(restart);
  while (err > tol * bnorm && arnoldi < maxit) {
    const double rnorm = err;
    std::fill(H.begin(), H.end(), cd(0));
    std::fill(gvec.begin(), gvec.end(), cd(0));
    gvec[0] = rnorm;
    int k = 0;
    double wnorm = rnorm;
    const double2* wsrc = r;
    for (int j = 0; j < restart; ++j) {
      if (err < tol * bnorm) break;
      double2* Vj = Vb + (size_t)j * N;
      double2* Zj = Zb + (size_t)j * N;
      // v_j = w / |w|
      HMC_TRY(scale_launch(c, N, 1.0 / wnorm, wsrc, Vj, v32));
      // z_j: spCG with tolerance TOL a |b| / ERR, or z_j = v_j
      const double t = tol * a * bnorm / err;
      HMC_TRY(precondition_solve(c, ms, sigma, Vj, v32, Zj, t < 1.0 ? std::max(t, inner_floor) : 1.0,
                           inner_prec, inner_maxit, st));
      // w = A z_j, h_ij = v_i^H w (i <= j), w -= sum h_ij v_i, h_{j+1,j} = |w|
      HMC_TRY(apply_A64(c, ms, sigma, Zj, w));
      st->applies64++;
      VecList V;
      for (int i = 0; i <= j; ++i) V.v[i] = Vb + (size_t)i * N;
      HMC_TRY(mdot_launch(c, N, V, j + 1, w, hdev, tk));
      HMC_TRY(gsupd_launch(c, N, V, j + 1, hdev, w, hdev + 40, tk));
      HMC_CUDA(c, cudaMemcpyAsync(hhost, hdev, 41 * sizeof(double), cudaMemcpyDeviceToHost, c->stream));
      HMC_CUDA(c, cudaStreamSynchronize(c->stream));
      for (int i = 0; i <= j; ++i) H[i + j * ldh] = cd(hhost[2 * i], hhost[2 * i + 1]);
      wnorm = std::sqrt(hhost[40]);
      H[j + 1 + j * ldh] = wnorm;
      if (!std::isfinite(wnorm)) return fail(c, HMC_ERR_NAN, "FGMRES: Arnoldi vector is not finite");
      // running residual estimate by Givens rotations
      std::vector<cd> col(j + 2);
      for (int i = 0; i <= j + 1; ++i) col[i] = H[i + j * ldh];
      for (int i = 0; i < j; ++i) {
        cd t0 = rc[i] * col[i] + rs[i] * col[i + 1];
        col[i + 1] = -std::conj(rs[i]) * col[i] + rc[i] * col[i + 1];
        col[i] = t0;
      }
      double cr;
      cd sr;
      if (std::abs(col[j + 1]) == 0.0) {
        cr = 1.0;
        sr = 0.0;
      } else if (std::abs(col[j]) == 0.0) {
        cr = 0.0;
        sr = std::conj(col[j + 1]) / std::abs(col[j + 1]);
      } else {
        const double na = std::abs(col[j]);
        const double nrm = std::hypot(na, std::abs(col[j + 1]));
        cr = na / nrm;
        sr = (col[j] / na) * std::conj(col[j + 1]) / nrm;
      }
      rc[j] = cr;
      rs[j] = sr;
      gvec[j + 1] = -std::conj(sr) * gvec[j];
      gvec[j] = cr * gvec[j];
      err = std::abs(gvec[j + 1]);
      k = j + 1;
      wsrc = w;
      ++arnoldi;
      if (arnoldi >= maxit) break;
    }
    if (k == 0) break;
    std::vector<cd> y;
    if (!normal_eq_cholesky(H, ldh, k, rnorm, y))
      return fail(c, HMC_ERR_NAN, "FGMRES: normal equations not positive definite");
    VecList Z;
    CoefList coef;
    for (int i = 0; i < k; ++i) {
      Z.v[i] = Zb + (size_t)i * N;
      coef.re[i] = y[i].real();
      coef.im[i] = y[i].imag();
    }
    HMC_TRY(xupd_launch(c, N, Z, coef, k, x));
    HMC_TRY(true_residual(&err));
    st->outer++;
  }
  st->iters += arnoldi;
  st->true_rel = err / bnorm;
  if (!(err <= tol * bnorm)) return fail(c, HMC_ERR_NOT_CONVERGED, "FGMRES reached its step limit");
  return HMC_OK;
}

hmc_status fcg_core(hmc_ctx* c, double ms, double sigma, const double2* b, double2* x, double tol,
                    double a, int maxit, double inner_floor, int inner_maxit, SolveStats* st) {
  using cd = std::complex<double>;
  const int N = c->geo.N;
  const size_t vb = sizeof(double2) * (size_t)N;
  double2 *r, *z, *buf, *u;
  HMC_TRY(ws_get(c, WS_FG_R, vb, (void**)&r));
  HMC_TRY(ws_get(c, WS_FG_W, vb, (void**)&z));
  HMC_TRY(ws_get(c, WS_FG_V, vb * 4, (void**)&buf));
  HMC_TRY(ws_get(c, WS_U64, vb, (void**)&u));
  double2* p = buf;
  double2* q = buf + N;
  double2* pp = buf + 2 * (size_t)N;  // previous direction and its image
  double2* qp = buf + 3 * (size_t)N;
  unsigned* tk = c->tickets;
  double* d = c->dscal;
  double* h = c->dscal_host;
  auto fetch = [&](int n) -> hmc_status {
    HMC_CUDA(c, cudaMemcpyAsync(h + 80, d + 80, n * sizeof(double), cudaMemcpyDeviceToHost, c->stream));
    HMC_CUDA(c, cudaStreamSynchronize(c->stream));
    return HMC_OK;
  };
  HMC_TRY(norm2_launch(c, N, b, d + 80, tk));
  HMC_TRY(fetch(1));
  const double bnorm = std::sqrt(h[80]);
  if (!std::isfinite(bnorm)) return fail(c, HMC_ERR_NAN, "FCG: right-hand side is not finite");
  HMC_CUDA(c, cudaMemsetAsync(x, 0, vb, c->stream));
  if (bnorm == 0.0) {
    st->true_rel = 0.0;
    return HMC_OK;
  }
  HMC_CUDA(c, cudaMemcpyAsync(r, b, vb, cudaMemcpyDeviceToDevice, c->stream));
  double rnorm = bnorm, pq_prev = 0.0;
  int k = 0;
  while (rnorm > tol * bnorm && k < maxit) {
    const double t = tol * a * bnorm / rnorm;
    HMC_TRY(precondition_solve(c, ms, sigma, r, nullptr, z, t < 1.0 ? std::max(t, inner_floor) : 1.0, 32,
                               inner_maxit, st));
    HMC_CUDA(c, cudaMemcpyAsync(p, z, vb, cudaMemcpyDeviceToDevice, c->stream));
    if (k > 0) {
      // beta = (A p_prev)^H z / (p_prev^H A p_prev);  p = z - beta p_prev
      VecList V;
      V.v[0] = qp;
      HMC_TRY(mdot_launch(c, N, V, 1, z, d + 80, tk));
      HMC_TRY(fetch(2));
      const cd beta = cd(h[80], h[81]) / pq_prev;
      VecList P;
      P.v[0] = pp;
      CoefList co;
      co.re[0] = -beta.real();
      co.im[0] = -beta.imag();
      HMC_TRY(xupd_launch(c, N, P, co, 1, p));
    }
    HMC_TRY(apply_A64(c, ms, sigma, p, q));
    st->applies64++;
    VecList V;
    V.v[0] = p;
    HMC_TRY(redot_launch(c, N, p, q, d + 82, tk));
    HMC_TRY(mdot_launch(c, N, V, 1, r, d + 80, tk));
    HMC_TRY(fetch(3));
    const double pq = h[82];
    if (!(pq > 0.0) || !std::isfinite(pq)) return fail(c, HMC_ERR_NAN, "FCG: non-positive curvature");
    const cd alpha = cd(h[80], h[81]) / pq;
    VecList P, Q;
    P.v[0] = p;
    Q.v[0] = q;
    CoefList ca, cm;
    ca.re[0] = alpha.real();
    ca.im[0] = alpha.imag();
    cm.re[0] = -alpha.real();
    cm.im[0] = -alpha.imag();
    HMC_TRY(xupd_launch(c, N, P, ca, 1, x));
    HMC_TRY(xupd_launch(c, N, Q, cm, 1, r));
    HMC_TRY(norm2_launch(c, N, r, d + 80, tk));
    HMC_TRY(fetch(1));
    rnorm = std::sqrt(h[80]);
    if (!std::isfinite(rnorm)) return fail(c, HMC_ERR_NAN, "FCG: residual is not finite");
    std::swap(p, pp);
    std::swap(q, qp);
    pq_prev = pq;
    ++k;
  }
  st->iters += k;
  // true residual in FP64
  HMC_TRY(mdag_launch<double>(c, c->geo, c->delta * ms, x, u));
  HMC_TRY(resid_launch<double>(c, c->geo, c->delta * ms, u, x, b, sigma, r, nullptr, nullptr, 0.0, 0, d + 80, tk));
  HMC_TRY(fetch(2));
  st->applies64++;
  st->true_rel = std::sqrt(h[80] / h[81]);
  if (!(rnorm <= tol * bnorm)) return fail(c, HMC_ERR_NOT_CONVERGED, "FCG reached its step limit");
  return HMC_OK;
}

hmc_status solve_opts(hmc_ctx* c, double ms, double sigma, const double2* b, double2* x,
                      const hmc_solver_opts* o, SolveStats* st) {
  if (o->method == HMC_SOLVER_CG64)
    return cg_core<double>(c, ms, sigma, b, x, true, o->tol, o->maxit, 0, true, st);
  if (o->method == HMC_SOLVER_FGMRES_MIXED || o->method == HMC_SOLVER_FGMRES_FP64)
    return fgmres_core(c, ms, sigma, b, x, o->tol, o->restart, o->a,
                       o->method == HMC_SOLVER_FGMRES_MIXED ? 32 : 64, o->maxit, o->inner_floor,
                       o->inner_maxit, st);
  if (o->method == HMC_SOLVER_FCG_MIXED)
    return fcg_core(c, ms, sigma, b, x, o->tol, o->a, o->maxit, o->inner_floor, o->inner_maxit, st);
  return fail(c, HMC_ERR_INVALID, "unknown solver method");
}

}  // namespace hmc
