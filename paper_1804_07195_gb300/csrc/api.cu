// C ABI entry points of libhmc: context management, argument validation,
// operator applications, solves and instrumentation. The operations and their
// passages in the paper are listed in include/hmc.h.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstdint>
#include <cstring>
#include <string>

#include "solvers.h"
#include "trace.h"
#include "validate.h"

using namespace hmc;

namespace hmc {

hmc_status fail(hmc_ctx* c, hmc_status s, const std::string& msg) {
  if (c) c->err = msg;
  return s;
}

hmc_status cuda_fail(hmc_ctx* c, cudaError_t e, const char* what) {
  if (c) c->err = std::string(what) + ": " + cudaGetErrorString(e);
  return HMC_ERR_CUDA;
}

hmc_status guarded_alloc(hmc_ctx* c, size_t bytes, void** user) {
  *user = nullptr;
  unsigned char* base = nullptr;
  cudaError_t e = cudaMalloc((void**)&base, bytes + 2 * kGuardBytes);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return fail(c, HMC_ERR_NOMEM, std::string("device allocation failed: ") + cudaGetErrorString(e));
  }
  // cudaMalloc returns 256-byte aligned memory, so the caller's part keeps that alignment
  e = cudaMemset(base, kGuardByte, kGuardBytes);
  if (e == cudaSuccess) e = cudaMemset(base + kGuardBytes + bytes, kGuardByte, kGuardBytes);
  if (e != cudaSuccess) {
    cudaFree(base);
    return cuda_fail(c, e, "guard bands");
  }
  *user = base + kGuardBytes;
  return HMC_OK;
}

void guarded_free(void* user) {
  if (user) cudaFree((unsigned char*)user - kGuardBytes);
}

hmc_status ws_get(hmc_ctx* c, int slot, size_t bytes, void** out) {
  if (c->ws_bytes[slot] < bytes) {
    if (c->ws[slot]) {
      cudaStreamSynchronize(c->stream);
      destroy_graphs(c);
      guarded_free(c->ws[slot]);
      c->ws[slot] = nullptr;
      c->ws_bytes[slot] = 0;
    }
    void* p = nullptr;
    HMC_TRY(guarded_alloc(c, bytes, &p));
    c->ws[slot] = p;
    c->ws_bytes[slot] = bytes;
  }
  *out = c->ws[slot];
  return HMC_OK;
}

void prof_begin(hmc_ctx* c, int id, cudaEvent_t* a) {
  c->prof.launches[id]++;
  if (!c->prof.timing) return;
  if (c->prof.free_events.empty()) {
    cudaEvent_t e;
    cudaEventCreate(&e);
    c->prof.free_events.push_back(e);
  }
  *a = c->prof.free_events.back();
  c->prof.free_events.pop_back();
  cudaEventRecord(*a, c->stream);
}

static void prof_drain(hmc_ctx* c, size_t keep) {
  // resolve the oldest pending pairs until at most `keep` remain
  auto& P = c->prof.pending;
  size_t n = P.size() > keep ? P.size() - keep : 0;
  for (size_t i = 0; i < n; ++i) {
    cudaEventSynchronize(P[i].b);
    float ms = 0.f;
    cudaEventElapsedTime(&ms, P[i].a, P[i].b);
    c->prof.ms[P[i].id] += ms;
    c->prof.free_events.push_back(P[i].a);
    c->prof.free_events.push_back(P[i].b);
  }
  P.erase(P.begin(), P.begin() + n);
}

void prof_end(hmc_ctx* c, int id, cudaEvent_t a) {
  if (!c->prof.timing || a == nullptr) return;
  if (c->prof.free_events.empty()) {
    cudaEvent_t e;
    cudaEventCreate(&e);
    c->prof.free_events.push_back(e);
  }
  cudaEvent_t b = c->prof.free_events.back();
  c->prof.free_events.pop_back();
  cudaEventRecord(b, c->stream);
  c->prof.pending.push_back(Pending{a, b, id});
  if (c->prof.pending.size() > 16384) prof_drain(c, 8192);
}

void prof_discard_last(hmc_ctx* c, int id, long long n, double bytes_each) {
  if (n <= 0) return;
  c->prof.launches[id] -= n;
  c->prof.bytes[id] -= bytes_each * (double)n;
  auto& P = c->prof.pending;
  long long left = n;
  for (size_t i = P.size(); i-- > 0 && left > 0;) {
    if (P[i].id != id) continue;
    c->prof.free_events.push_back(P[i].a);
    c->prof.free_events.push_back(P[i].b);
    P.erase(P.begin() + i);
    --left;
  }
}

hmc_status capture_graph(hmc_ctx* c, const std::function<hmc_status()>& body, cudaGraphExec_t* out) {
  *out = nullptr;
  if (!c->cap_stream) HMC_CUDA(c, cudaStreamCreateWithFlags(&c->cap_stream, cudaStreamNonBlocking));
  cudaStream_t saved = c->stream;
  c->stream = c->cap_stream;
  c->capturing = true;
  c->pdl_armed = false;
  cudaError_t e = cudaStreamBeginCapture(c->cap_stream, cudaStreamCaptureModeThreadLocal);
  hmc_status st = e == cudaSuccess ? body() : cuda_fail(c, e, "cudaStreamBeginCapture");
  cudaGraph_t graph = nullptr;
  if (e == cudaSuccess) {
    cudaError_t e2 = cudaStreamEndCapture(c->cap_stream, &graph);
    if (e2 != cudaSuccess && st == HMC_OK) st = cuda_fail(c, e2, "cudaStreamEndCapture");
  }
  c->capturing = false;
  c->pdl_armed = false;
  c->stream = saved;
  if (st == HMC_OK && graph) {
    e = cudaGraphInstantiate(out, graph, 0);
    if (e != cudaSuccess) st = cuda_fail(c, e, "cudaGraphInstantiate");
  }
  if (graph) cudaGraphDestroy(graph);
  if (st != HMC_OK) cudaGetLastError();  // a failed capture leaves no error behind
  return st;
}

hmc_status capture_loop_graph(hmc_ctx* c, const std::function<hmc_status(cudaGraphConditionalHandle)>& body,
                              cudaGraphExec_t* out) {
  *out = nullptr;
  if (!c->cap_stream) HMC_CUDA(c, cudaStreamCreateWithFlags(&c->cap_stream, cudaStreamNonBlocking));
  cudaGraph_t graph = nullptr;
  cudaError_t e = cudaGraphCreate(&graph, 0);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return cuda_fail(c, e, "cudaGraphCreate");
  }
  cudaGraphConditionalHandle h{};
  cudaGraph_t body_graph = nullptr;
  e = cudaGraphConditionalHandleCreate(&h, graph, 1, cudaGraphCondAssignDefault);
  if (e == cudaSuccess) {
    cudaGraphNodeParams p{};
    p.type = cudaGraphNodeTypeConditional;
    p.conditional.handle = h;
    p.conditional.type = cudaGraphCondTypeWhile;
    p.conditional.size = 1;
    cudaGraphNode_t node;
    e = cudaGraphAddNode(&node, graph, nullptr, nullptr, 0, &p);
    if (e == cudaSuccess) body_graph = p.conditional.phGraph_out[0];
  }
  hmc_status st = HMC_OK;
  if (e != cudaSuccess) {
    st = cuda_fail(c, e, "conditional graph node");
  } else {
    cudaStream_t saved = c->stream;
    c->stream = c->cap_stream;
    c->capturing = true;
    c->pdl_armed = false;
    e = cudaStreamBeginCaptureToGraph(c->cap_stream, body_graph, nullptr, nullptr, 0,
                                      cudaStreamCaptureModeThreadLocal);
    st = e == cudaSuccess ? body(h) : cuda_fail(c, e, "cudaStreamBeginCaptureToGraph");
    if (e == cudaSuccess) {
      cudaGraph_t captured = nullptr;  // the body graph itself, owned by the node
      cudaError_t e2 = cudaStreamEndCapture(c->cap_stream, &captured);
      if (e2 != cudaSuccess && st == HMC_OK) st = cuda_fail(c, e2, "cudaStreamEndCapture");
    }
    c->capturing = false;
    c->pdl_armed = false;
    c->stream = saved;
  }
  if (st == HMC_OK) {
    e = cudaGraphInstantiate(out, graph, 0);
    if (e != cudaSuccess) st = cuda_fail(c, e, "cudaGraphInstantiate");
  }
  cudaGraphDestroy(graph);
  if (st != HMC_OK) cudaGetLastError();  // a failed capture leaves no error behind
  return st;
}

GraphEntry* find_graph(hmc_ctx* c, int kind, const void* const key[6]) {
  for (auto& g : c->graphs) {
    if (g.kind != kind) continue;
    bool same = true;
    for (int i = 0; i < 6; ++i) same = same && g.key[i] == key[i];
    if (same) {
      g.last_use = ++c->graph_clock;
      return &g;
    }
  }
  return nullptr;
}

GraphEntry* add_graph(hmc_ctx* c, int kind, const void* const key[6], cudaGraphExec_t exec) {
  constexpr size_t kMaxGraphs = 16;
  if (c->graphs.size() >= kMaxGraphs) {  // evict the least recently used
    size_t old = 0;
    for (size_t i = 1; i < c->graphs.size(); ++i)
      if (c->graphs[i].last_use < c->graphs[old].last_use) old = i;
    cudaGraphExecDestroy(c->graphs[old].exec);
    c->graphs.erase(c->graphs.begin() + old);
  }
  GraphEntry g;
  g.kind = kind;
  for (int i = 0; i < 6; ++i) g.key[i] = key[i];
  g.exec = exec;
  g.last_use = ++c->graph_clock;
  c->graphs.push_back(g);
  return &c->graphs.back();
}

void destroy_graphs(hmc_ctx* c) {
  for (auto& g : c->graphs) cudaGraphExecDestroy(g.exec);
  c->graphs.clear();
}

hmc_status prepare_field(hmc_ctx* c, const double* phi) {
  if (phi == nullptr) {
    if (!c->field_loaded) return fail(c, HMC_ERR_INVALID, "phi is NULL and no field was loaded");
    return HMC_OK;
  }
  if (((uintptr_t)phi) % 8) return fail(c, HMC_ERR_INVALID, "phi is not 8-byte aligned");
  c->field_loaded = false;
  return k_phase_launch(c, phi);
}

}  // namespace hmc

static hmc_status check_vec(hmc_ctx* c, const void* p, int prec, const char* what) {
  if (p == nullptr) return fail(c, HMC_ERR_INVALID, std::string(what) + " is NULL");
  const uintptr_t al = prec == 64 ? 16 : 8;
  if (((uintptr_t)p) % al) return fail(c, HMC_ERR_INVALID, std::string(what) + " is misaligned");
  return HMC_OK;
}

static hmc_status check_mass(hmc_ctx* c, double ms) {
  if (!std::isfinite(ms)) return fail(c, HMC_ERR_INVALID, "staggered mass is not finite");
  if (1.0 - c->delta * ms == 0.0) return fail(c, HMC_ERR_INVALID, "1 - delta*m_s == 0: the time hop vanishes");
  return HMC_OK;
}

// Bytes of one complex vector of the context's lattice in precision prec.
static size_t vec_bytes(const hmc_ctx* c, int prec) { return (size_t)c->geo.N * (prec == 64 ? 16 : 8); }

static hmc_status check_prec(hmc_ctx* c, int prec) {
  if (prec != 32 && prec != 64) return fail(c, HMC_ERR_INVALID, "prec must be 32 or 64");
  return HMC_OK;
}

// (M M^dagger + sigma) in, in two passes (u = M^dagger in through memory) or
// with the fused kernel (u on chip).
template <typename R>
static hmc_status apply_A_variant(hmc_ctx* c, int variant, double ms, double sigma, const V2<R>* in,
                                  V2<R>* out) {
  const R dm = (R)(c->delta * ms);
  if (variant == 2) return mmdag_fused_launch<R>(c, c->geo, dm, (R)sigma, in, out);
  if constexpr (sizeof(R) == 8) {
    return apply_A64(c, ms, sigma, in, out);
  } else {
    float2* u;
    HMC_TRY(ws_get(c, WS_U32, sizeof(float2) * (size_t)c->geo.N, (void**)&u));
    HMC_TRY(mdag_launch<float>(c, c->geo, dm, in, u));
    return m_launch<float>(c, c->geo, dm, u, sigma != 0.0 ? in : nullptr, (float)sigma, out);
  }
}

// The variant in use: pinned by hmc_set_apply_variant, else chosen on the
// first application in each precision by timing both (after tuning the fused
// kernel's tile on the same operands).
template <typename R>
static hmc_status apply_A(hmc_ctx* c, double ms, double sigma, const V2<R>* in, V2<R>* out) {
  const int pi = sizeof(R) == 4 ? 0 : 1;
  int v = c->apply_variant;
  if (v == 0) {
    if (c->apply_choice[pi] == 0) {
      float best = 1e30f;
      cudaEvent_t e0, e1;
      HMC_CUDA(c, cudaEventCreate(&e0));
      HMC_CUDA(c, cudaEventCreate(&e1));
      for (int cand = 1; cand <= 2; ++cand) {
        HMC_TRY(apply_A_variant<R>(c, cand, ms, sigma, in, out));  // warm (and tune)
        HMC_CUDA(c, cudaEventRecord(e0, c->stream));
        for (int rep = 0; rep < 3; ++rep) HMC_TRY(apply_A_variant<R>(c, cand, ms, sigma, in, out));
        HMC_CUDA(c, cudaEventRecord(e1, c->stream));
        HMC_CUDA(c, cudaEventSynchronize(e1));
        float t = 0.f;
        cudaEventElapsedTime(&t, e0, e1);
        if (t < best) {
          best = t;
          c->apply_choice[pi] = cand;
        }
      }
      cudaEventDestroy(e0);
      cudaEventDestroy(e1);
    }
    v = c->apply_choice[pi];
  }
  return apply_A_variant<R>(c, v, ms, sigma, in, out);
}

extern "C" {

int hmc_abi_version(void) { return HMC_ABI_VERSION; }

const char* hmc_status_string(hmc_status s) {
  switch (s) {
    case HMC_OK: return "ok";
    case HMC_ERR_INVALID: return "invalid argument";
    case HMC_ERR_CUDA: return "CUDA error";
    case HMC_ERR_NOT_CONVERGED: return "solver did not converge";
    case HMC_ERR_NAN: return "NaN, Inf or breakdown in a reduction";
    case HMC_ERR_TIMEOUT: return "device wait timed out";
    case HMC_ERR_NOMEM: return "out of device memory";
  }
  return "unknown status";
}

const char* hmc_last_error(const hmc_ctx* ctx) { return ctx ? ctx->err.c_str() : ""; }

hmc_status hmc_create(hmc_ctx** out, const hmc_lattice* lat, void* stream) {
  if (!out) return HMC_ERR_INVALID;
  *out = nullptr;
  if (bad_lattice(lat)) return HMC_ERR_INVALID;
  hmc_ctx* c = new hmc_ctx();
  c->lat = *lat;
  c->delta = lat->beta / lat->nt;
  c->geo = make_geo(lat->n, lat->m, lat->nt, c->delta, lat->kappa);
  c->stream = (cudaStream_t)stream;
  auto bail = [&](cudaError_t e) {
    cudaGetLastError();
    hmc_destroy(c);
    return e == cudaErrorMemoryAllocation ? HMC_ERR_NOMEM : HMC_ERR_CUDA;
  };
  cudaError_t e = cudaGetDevice(&c->device);
  if (e != cudaSuccess) return bail(e);
  e = cudaDeviceGetAttribute(&c->nsm, cudaDevAttrMultiProcessorCount, c->device);
  if (e != cudaSuccess) return bail(e);
  c->max_grid = c->nsm * kMaxGridPerSM;
  for (int k = 0; k < K_COUNT; ++k) c->shape[k] = Shape{};
  const size_t N = (size_t)c->geo.N;
  if (guarded_alloc(c, N * sizeof(double2), &c->ws[WS_E]) != HMC_OK) return bail(cudaErrorMemoryAllocation);
  c->ws_bytes[WS_E] = N * sizeof(double2);
  if (guarded_alloc(c, N * sizeof(float), &c->ws[WS_PHI32]) != HMC_OK) return bail(cudaErrorMemoryAllocation);
  c->ws_bytes[WS_PHI32] = N * sizeof(float);
  const size_t npart = (size_t)kMaxRed * std::max(c->max_grid, c->nsm * kOneItemBlocksPerSM);
  if ((e = cudaMalloc(&c->partials, sizeof(double) * npart)) != cudaSuccess) return bail(e);
  if ((e = cudaMalloc(&c->partA, sizeof(double) * c->nsm * 2 * kOneItemBlocksPerSM)) != cudaSuccess) return bail(e);
  if ((e = cudaMalloc(&c->partB, sizeof(double) * c->nsm * 2 * kOneItemBlocksPerSM)) != cudaSuccess) return bail(e);
  if ((e = cudaMalloc(&c->tickets, sizeof(unsigned) * kTickets)) != cudaSuccess) return bail(e);
  if ((e = cudaMemset(c->tickets, 0, sizeof(unsigned) * kTickets)) != cudaSuccess) return bail(e);
  if ((e = cudaMalloc(&c->sc, sizeof(CGScal) * 4)) != cudaSuccess) return bail(e);
  if ((e = cudaMalloc(&c->gbar, sizeof(GridBar))) != cudaSuccess) return bail(e);
  if ((e = cudaMalloc(&c->loop_trips, 2 * sizeof(unsigned))) != cudaSuccess) return bail(e);
  if ((e = cudaMallocHost(&c->loop_trips_host, 2 * sizeof(unsigned))) != cudaSuccess) return bail(e);
  if ((e = cudaMemset(c->gbar, 0, sizeof(GridBar))) != cudaSuccess) return bail(e);
  if ((e = cudaMemset(c->sc, 0, sizeof(CGScal) * 4)) != cudaSuccess) return bail(e);
  // one-item grids of the tuned kernels may reach nsm * 128 blocks of 128 threads
  if ((e = cudaFree(c->partials)) != cudaSuccess) return bail(e);
  if ((e = cudaMalloc(&c->partials, sizeof(double) * kMaxRed * c->nsm * 2 * kOneItemBlocksPerSM)) != cudaSuccess)
    return bail(e);
  if ((e = cudaMallocHost(&c->sc_host, sizeof(CGScal) * 4)) != cudaSuccess) return bail(e);
  if ((e = cudaMalloc(&c->dscal, sizeof(double) * 128)) != cudaSuccess) return bail(e);
  if ((e = cudaMallocHost(&c->dscal_host, sizeof(double) * 128)) != cudaSuccess) return bail(e);
  *out = c;
  return HMC_OK;
}

hmc_status hmc_destroy(hmc_ctx* c) {
  if (!c) return HMC_ERR_INVALID;
  for (hmc_ctx* sc : c->subs)
    if (sc) hmc_destroy(sc);
  c->subs.clear();
  if (c->stream || c->device >= 0) cudaStreamSynchronize(c->stream);
  destroy_graphs(c);
  if (c->cap_stream) cudaStreamDestroy(c->cap_stream);
  for (int i = 0; i < WS_COUNT; ++i)
    if (c->ws[i]) guarded_free(c->ws[i]);
  if (c->partials) cudaFree(c->partials);
  if (c->partA) cudaFree(c->partA);
  if (c->partB) cudaFree(c->partB);
  if (c->tickets) cudaFree(c->tickets);
  if (c->sc) cudaFree(c->sc);
  if (c->gbar) cudaFree(c->gbar);
  if (c->loop_trips) cudaFree(c->loop_trips);
  if (c->loop_trips_host) cudaFreeHost(c->loop_trips_host);
  for (int i = 0; i < hmc_ctx::kBatchSlots; ++i)
    if (c->bpool[i]) guarded_free(c->bpool[i]);
  for (int i = 0; i < 4; ++i)
    if (c->bpool_host[i]) cudaFreeHost(c->bpool_host[i]);
  if (c->sc_host) cudaFreeHost(c->sc_host);
  if (c->dscal) cudaFree(c->dscal);
  if (c->dscal_host) cudaFreeHost(c->dscal_host);
  for (auto& p : c->prof.pending) {
    cudaEventDestroy(p.a);
    cudaEventDestroy(p.b);
  }
  for (auto e : c->prof.free_events) cudaEventDestroy(e);
  delete c;
  return HMC_OK;
}

hmc_status hmc_set_stream(hmc_ctx* c, void* stream) {
  if (!c) return HMC_ERR_INVALID;
  c->stream = (cudaStream_t)stream;
  return HMC_OK;
}

hmc_status hmc_load_field(hmc_ctx* c, const double* phi) {
  if (!c) return HMC_ERR_INVALID;
  if (!phi) return fail(c, HMC_ERR_INVALID, "phi is NULL");
  HMC_TRY(prepare_field(c, phi));
  c->field_loaded = true;
  c->loaded_phi = phi;
  return HMC_OK;
}

hmc_status hmc_apply_M(hmc_ctx* c, const double* phi, double ms, const void* in, void* out, int prec) {
  if (!c) return HMC_ERR_INVALID;
  HMC_TRACE("hmc_apply_M");
  HMC_TRY(check_prec(c, prec));
  HMC_TRY(check_vec(c, in, prec, "in"));
  HMC_TRY(check_vec(c, out, prec, "out"));
  HMC_TRY(check_mass(c, ms));
  if (ranges_overlap(in, out, vec_bytes(c, prec))) return fail(c, HMC_ERR_INVALID, "in and out must not overlap");
  HMC_TRY(prepare_field(c, phi));
  if (prec == 64)
    return m_launch<double>(c, c->geo, c->delta * ms, (const double2*)in, nullptr, 0.0, (double2*)out);
  return m_launch<float>(c, c->geo, (float)(c->delta * ms), (const float2*)in, nullptr, 0.f, (float2*)out);
}

hmc_status hmc_apply_Mdag(hmc_ctx* c, const double* phi, double ms, const void* in, void* out, int prec) {
  if (!c) return HMC_ERR_INVALID;
  HMC_TRACE("hmc_apply_Mdag");
  HMC_TRY(check_prec(c, prec));
  HMC_TRY(check_vec(c, in, prec, "in"));
  HMC_TRY(check_vec(c, out, prec, "out"));
  HMC_TRY(check_mass(c, ms));
  if (ranges_overlap(in, out, vec_bytes(c, prec))) return fail(c, HMC_ERR_INVALID, "in and out must not overlap");
  HMC_TRY(prepare_field(c, phi));
  if (prec == 64) return mdag_launch<double>(c, c->geo, c->delta * ms, (const double2*)in, (double2*)out);
  return mdag_launch<float>(c, c->geo, (float)(c->delta * ms), (const float2*)in, (float2*)out);
}

hmc_status hmc_apply_MMdag(hmc_ctx* c, const double* phi, double ms, double sigma, const void* in,
                           void* out, int prec) {
  if (!c) return HMC_ERR_INVALID;
  HMC_TRACE("hmc_apply_MMdag");
  HMC_TRY(check_prec(c, prec));
  HMC_TRY(check_vec(c, in, prec, "in"));
  HMC_TRY(check_vec(c, out, prec, "out"));
  HMC_TRY(check_mass(c, ms));
  if (!(sigma >= 0.0) || !std::isfinite(sigma)) return fail(c, HMC_ERR_INVALID, "sigma must be finite and >= 0");
  if (ranges_overlap(in, out, vec_bytes(c, prec))) return fail(c, HMC_ERR_INVALID, "in and out must not overlap");
  HMC_TRY(prepare_field(c, phi));
  if (prec == 64) return apply_A<double>(c, ms, sigma, (const double2*)in, (double2*)out);
  return apply_A<float>(c, ms, sigma, (const float2*)in, (float2*)out);
}

static hmc_status solve_checks(hmc_ctx* c, double ms, double sigma, const void* b, void* x, int prec,
                               double tol, int maxit) {
  HMC_TRY(check_vec(c, b, prec, "b"));
  HMC_TRY(check_vec(c, x, prec, "x"));
  HMC_TRY(check_mass(c, ms));
  if (!(sigma >= 0.0) || !std::isfinite(sigma)) return fail(c, HMC_ERR_INVALID, "sigma must be finite and >= 0");
  if (!(tol > 0.0) || !std::isfinite(tol)) return fail(c, HMC_ERR_INVALID, "tol must be positive");
  if (maxit < 1) return fail(c, HMC_ERR_INVALID, "maxit must be >= 1");
  if (ranges_overlap(b, x, vec_bytes(c, prec))) return fail(c, HMC_ERR_INVALID, "b and x must not overlap");
  return HMC_OK;
}

static double now_s() {
  return std::chrono::duration<double>(std::chrono::steady_clock::now().time_since_epoch()).count();
}

static void fill_info(hmc_solve_info* info, const SolveStats& s, hmc_status st, double t0,
                      double bytes_per_apply_site, double N) {
  if (!info) return;
  std::memset(info, 0, sizeof(*info));
  info->iters = s.iters;
  info->iters_outer = s.outer;
  info->iters_inner = s.inner;
  info->status = st;
  info->true_rel_res = s.true_rel;
  info->seconds = now_s() - t0;
  info->applies64 = s.applies64;
  info->applies32 = s.applies32;
  (void)bytes_per_apply_site;
  // algorithmic bytes: one CG iteration moves 192 B/site in FP64 and 96 B/site in FP32
  info->bytes = (long long)(N * (192.0 * s.applies64 + 96.0 * s.applies32));
}

hmc_status hmc_solve_cg(hmc_ctx* c, const double* phi, double ms, double sigma, const void* b, void* x,
                        double tol, int maxit, hmc_solve_info* info) {
  if (!c) return HMC_ERR_INVALID;
  HMC_TRACE("hmc_solve_cg");
  const double t0 = now_s();
  HMC_TRY(solve_checks(c, ms, sigma, b, x, 64, tol, maxit));
  HMC_TRY(prepare_field(c, phi));
  SolveStats s;
  hmc_status st = cg_core<double>(c, ms, sigma, (const double2*)b, (double2*)x, false, tol, maxit, 0, true, &s);
  fill_info(info, s, st, t0, 0, c->geo.N);
  return st;
}

hmc_status hmc_solve_spcg(hmc_ctx* c, const double* phi, double ms, double sigma, const void* b, void* x,
                          double tol, int maxit, hmc_solve_info* info) {
  if (!c) return HMC_ERR_INVALID;
  HMC_TRACE("hmc_solve_spcg");
  const double t0 = now_s();
  HMC_TRY(solve_checks(c, ms, sigma, b, x, 32, tol, maxit));
  HMC_TRY(prepare_field(c, phi));
  SolveStats s;
  // the kernels with two cells per thread access x in 16-byte units: an x
  // that is only 8-byte aligned is solved in a workspace vector and copied
  float2* xs = (float2*)x;
  if ((uintptr_t)x % 16) HMC_TRY(ws_get(c, WS_CG_X32, sizeof(float2) * (size_t)c->geo.N, (void**)&xs));
  hmc_status st = cg_core<float>(c, ms, sigma, (const float2*)b, xs, true, tol, maxit, 1, true, &s);
  if (xs != (float2*)x)
    HMC_CUDA(c, cudaMemcpyAsync(x, xs, sizeof(float2) * (size_t)c->geo.N, cudaMemcpyDeviceToDevice, c->stream));
  fill_info(info, s, st, t0, 0, c->geo.N);
  return st;
}

hmc_status hmc_solve_fgmres(hmc_ctx* c, const double* phi, double ms, double sigma, const void* b, void* x,
                            double tol, int restart, double a, int inner_prec, int maxit,
                            hmc_solve_info* info) {
  if (!c) return HMC_ERR_INVALID;
  HMC_TRACE("hmc_solve_fgmres");
  const double t0 = now_s();
  HMC_TRY(solve_checks(c, ms, sigma, b, x, 64, tol, maxit));
  if (restart < 1 || restart > kMaxRestart) return fail(c, HMC_ERR_INVALID, "restart must be in [1, 16]");
  if (!(a > 0.0)) return fail(c, HMC_ERR_INVALID, "a must be positive");
  if (inner_prec != 32 && inner_prec != 64) return fail(c, HMC_ERR_INVALID, "inner_prec must be 32 or 64");
  HMC_TRY(prepare_field(c, phi));
  SolveStats s;
  hmc_status st = fgmres_core(c, ms, sigma, (const double2*)b, (double2*)x, tol, restart, a, inner_prec,
                              maxit, 1e-6, 2000, &s);
  fill_info(info, s, st, t0, 0, c->geo.N);
  return st;
}

hmc_status hmc_solve_fcg(hmc_ctx* c, const double* phi, double ms, double sigma, const void* b, void* x,
                         double tol, double a, int maxit, hmc_solve_info* info) {
  if (!c) return HMC_ERR_INVALID;
  HMC_TRACE("hmc_solve_fcg");
  const double t0 = now_s();
  HMC_TRY(solve_checks(c, ms, sigma, b, x, 64, tol, maxit));
  if (!(a > 0.0)) return fail(c, HMC_ERR_INVALID, "a must be positive");
  HMC_TRY(prepare_field(c, phi));
  SolveStats s;
  hmc_status st = fcg_core(c, ms, sigma, (const double2*)b, (double2*)x, tol, a, maxit, 1e-6, 2000, &s);
  fill_info(info, s, st, t0, 0, c->geo.N);
  return st;
}

hmc_status hmc_set_cg_variant(hmc_ctx* c, int variant) {
  if (!c) return HMC_ERR_INVALID;
  if (variant < 0 || variant > 7) return fail(c, HMC_ERR_INVALID, "variant must be 0 to 7");
  c->cg32_variant = variant;
  c->tuned32 = false;
  c->persist32 = false;
  c->cg1_32 = false;
  c->resident32 = false;
  destroy_graphs(c);
  return HMC_OK;
}

hmc_status hmc_set_batched_variant(hmc_ctx* c, int variant) {
  if (!c) return HMC_ERR_INVALID;
  if (variant < 0 || variant > 2) return fail(c, HMC_ERR_INVALID, "variant must be 0, 1 or 2");
  c->batch_variant = variant;
  c->batch_choice = 0;
  c->batch_us[0] = c->batch_us[1] = 0.f;
  return HMC_OK;
}

hmc_status hmc_batched_variant(hmc_ctx* c, int* variant) {
  if (!c || !variant) return HMC_ERR_INVALID;
  *variant = c->batch_variant ? c->batch_variant : c->batch_choice;
  return HMC_OK;
}

hmc_status hmc_set_apply_variant(hmc_ctx* c, int variant) {
  if (!c) return HMC_ERR_INVALID;
  if (variant < 0 || variant > 2) return fail(c, HMC_ERR_INVALID, "variant must be 0, 1 or 2");
  c->apply_variant = variant;
  c->apply_choice[0] = c->apply_choice[1] = 0;
  return HMC_OK;
}

hmc_status hmc_apply_variant(hmc_ctx* c, int prec, int* variant) {
  if (!c || !variant) return HMC_ERR_INVALID;
  HMC_TRY(check_prec(c, prec));
  *variant = c->apply_variant ? c->apply_variant : c->apply_choice[prec == 32 ? 0 : 1];
  return HMC_OK;
}

hmc_status hmc_set_fused_tile(hmc_ctx* c, int prec, int Ti, int Tj, int Tt, int depth, int pairs) {
  if (!c) return HMC_ERR_INVALID;
  HMC_TRY(check_prec(c, prec));
  if (Ti < 1 || Tj < 1 || Tt < 1) return fail(c, HMC_ERR_INVALID, "tile sizes must be >= 1");
  if (pairs != 0 && pairs != 1) return fail(c, HMC_ERR_INVALID, "pairs must be 0 or 1");
  return set_fused_shape(c, prec, Ti, Tj, Tt, depth, pairs);
}

hmc_status hmc_fused_tile(hmc_ctx* c, int prec, int* Ti, int* Tj, int* Tt, int* depth, int* pairs) {
  if (!c || !Ti || !Tj || !Tt || !depth || !pairs) return HMC_ERR_INVALID;
  HMC_TRY(check_prec(c, prec));
  const FusedShape& fs = c->fshape[prec == 32 ? 0 : 1];
  *Ti = fs.Ti;
  *Tj = fs.Tj;
  *Tt = fs.Tt;
  *depth = fs.D;
  *pairs = fs.pairs;
  return HMC_OK;
}

hmc_status hmc_set_cg_fused_tile(hmc_ctx* c, int Ti, int Tj, int Tt, int depth) {
  if (!c) return HMC_ERR_INVALID;
  if (Ti == 0 && Tj == 0 && Tt == 0) {  // back to the tuner
    c->cg1_pinned = false;
    c->tuned32 = false;
    c->cg1_32 = false;
    destroy_graphs(c);
    return HMC_OK;
  }
  if (Ti < 1 || Tj < 1 || Tt < 1) return fail(c, HMC_ERR_INVALID, "tile sizes must be >= 1");
  HMC_TRY(set_cg1_shape(c, Ti, Tj, Tt, depth));
  c->tuned32 = false;
  c->cg1_32 = false;
  destroy_graphs(c);
  return HMC_OK;
}

hmc_status hmc_cg_fused_tile(hmc_ctx* c, int* Ti, int* Tj, int* Tt, int* depth, int* in_use) {
  if (!c || !Ti || !Tj || !Tt || !depth || !in_use) return HMC_ERR_INVALID;
  const FusedShape& fs = c->cg1_shape;
  *Ti = fs.Ti;
  *Tj = fs.Tj;
  *Tt = fs.Tt;
  *depth = fs.D;
  *in_use = c->cg1_32 ? 1 : 0;
  return HMC_OK;
}

hmc_status hmc_graph_mode(hmc_ctx* c, int* mode) {
  if (!c || !mode) return HMC_ERR_INVALID;
  *mode = (!c->use_graphs || c->prof.timing) ? 0 : (c->use_loop_graphs ? 2 : 1);
  return HMC_OK;
}

hmc_status hmc_set_graph_mode(hmc_ctx* c, int mode) {
  if (!c) return HMC_ERR_INVALID;
  if (mode != 1 && mode != 2) return fail(c, HMC_ERR_INVALID, "graph mode must be 1 or 2");
  c->use_loop_graphs = (mode == 2);
  return HMC_OK;
}

hmc_status hmc_set_wait_test(hmc_ctx* c, int extra, long long limit_cycles) {
  if (!c) return HMC_ERR_INVALID;
  if (extra < 0 || limit_cycles < 0) return fail(c, HMC_ERR_INVALID, "extra and limit_cycles must be >= 0");
  c->bar_extra = extra;
  c->bar_limit = limit_cycles;
  return HMC_OK;
}

hmc_status hmc_check_guards(hmc_ctx* c, int* nbad) {
  if (!c || !nbad) return HMC_ERR_INVALID;
  *nbad = 0;
  HMC_CUDA(c, cudaStreamSynchronize(c->stream));
  std::string first;
  unsigned char band[2][kGuardBytes];
  auto check = [&](void* user, size_t bytes, const std::string& what) -> hmc_status {
    if (!user) return HMC_OK;
    const unsigned char* u = (const unsigned char*)user;
    HMC_CUDA(c, cudaMemcpy(band[0], u - kGuardBytes, kGuardBytes, cudaMemcpyDeviceToHost));
    HMC_CUDA(c, cudaMemcpy(band[1], u + bytes, kGuardBytes, cudaMemcpyDeviceToHost));
    for (int h = 0; h < 2; ++h)
      for (size_t k = 0; k < kGuardBytes; ++k)
        if (band[h][k] != kGuardByte) {
          ++*nbad;
          if (first.empty()) first = what + (h ? " (after its end)" : " (before its start)");
          break;
        }
    return HMC_OK;
  };
  for (int i = 0; i < WS_COUNT; ++i) HMC_TRY(check(c->ws[i], c->ws_bytes[i], "workspace slot " + std::to_string(i)));
  for (int i = 0; i < hmc_ctx::kBatchSlots; ++i)
    HMC_TRY(check(c->bpool[i], c->bpool_bytes[i], "batched buffer " + std::to_string(i)));
  if (*nbad) c->err = std::to_string(*nbad) + " guard band(s) overwritten, first: " + first;
  return HMC_OK;
}

hmc_status hmc_guard_test_write(hmc_ctx* c) {
  if (!c || !c->ws[WS_E]) return HMC_ERR_INVALID;
  // one byte just past the end of the phase table: inside its guard band
  HMC_CUDA(c, cudaMemset((unsigned char*)c->ws[WS_E] + c->ws_bytes[WS_E], 0, 1));
  return HMC_OK;
}

hmc_status hmc_profile(hmc_ctx* c, int timing_on, int reset) {
  if (!c) return HMC_ERR_INVALID;
  if (reset) {
    prof_drain(c, 0);
    for (int i = 0; i < K_COUNT; ++i) {
      c->prof.launches[i] = 0;
      c->prof.ms[i] = 0.0;
      c->prof.bytes[i] = 0.0;
    }
  }
  c->prof.timing = timing_on != 0;
  return HMC_OK;
}

static_assert(K_COUNT <= HMC_NKERNELS, "hmc_profile_read must be able to report every kernel group");

hmc_status hmc_profile_read(hmc_ctx* c, hmc_kernel_stat* out, int max, int* count) {
  if (!c || !out || !count) return HMC_ERR_INVALID;
  prof_drain(c, 0);
  int n = 0;
  for (int i = 0; i < K_COUNT && n < max; ++i) {
    std::memset(&out[n], 0, sizeof(hmc_kernel_stat));
    std::strncpy(out[n].name, kKernelNames[i], sizeof(out[n].name) - 1);
    out[n].launches = c->prof.launches[i];
    out[n].ms_total = c->prof.ms[i];
    out[n].bytes_total = c->prof.bytes[i];
    out[n].threads = c->shape[i].threads;
    const Shape& sh = c->shape[i];
    out[n].waves = (sh.tiled == 1 || sh.tiled == 2) ? -(sh.tt + (sh.tiled == 2 ? 1000 : 0)) : sh.waves;
    out[n].design = sh.tiled;
    ++n;
  }
  *count = n;
  return HMC_OK;
}

}  // extern "C"
