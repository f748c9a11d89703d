// Internal definition of the library context: stream, geometry, phase tables,
// workspace pool, reduction scratch and launch instrumentation.
#pragma once

#include <cuda_runtime.h>

#include <functional>
#include <string>
#include <vector>

#include "common.cuh"
#include "hmc.h"

namespace hmc {

// Kernel identifiers for the launch counters and event timing.
enum KernelId {
  K_PHASE = 0,
  K_MDAG64,
  K_M64,
  K_MDAG32,
  K_M32,
  K_CG_MDAG64,
  K_CG_M64,
  K_CG_P64,
  K_CG_MDAG32,
  K_CG_M32,
  K_CG_P32,
  K_RESID64,
  K_RESID32,
  K_INIT0,
  K_CONVERT,
  K_NORM,
  K_MDOT,
  K_GSUPD,
  K_SCALE,
  K_XUPD,
  K_FORCE,
  K_AXPY,
  K_MD,
  K_BATCH_CG64,
  K_BATCH_CG32,
  K_BATCH_INIT,
  K_BATCH_RESID,
  K_BATCH_MISC,
  K_CG_PERSIST32,
  K_MMDAG_FUSED32,
  K_MMDAG_FUSED64,
  K_CG1_32,
  K_CG_RES32,
  K_COUNT
};

extern const char* const kKernelNames[K_COUNT];
extern const double kKernelBytesPerSite[K_COUNT];

// Named workspace slots owned by the context.
enum WsSlot {
  WS_E = 0,      // e^{i phi} table, complex128
  WS_PHI32,      // phi rounded to float
  WS_U64,        // M^dagger intermediate, complex128
  WS_U32,
  WS_CG_R64, WS_CG_P64, WS_CG_X64,
  WS_CG_R32, WS_CG_P32, WS_CG_X32, WS_CG_B32, WS_CG_Q32,
  WS_CG1_R1, WS_CG1_W0, WS_CG1_W1, WS_CG1_S0, WS_CG1_S1,  // single-reduction FP32 CG
  WS_FG_R, WS_FG_W, WS_FG_X, WS_FG_V, WS_FG_Z,  // FGMRES vectors; V, Z hold `restart` each
  WS_F_ETA, WS_F_XI, WS_F_SRC, WS_F_TMP,        // force / action temporaries
  WS_MD_CHI, WS_MD_GRAD, WS_MD_FORCE,           // trajectory: pseudofermions, level forces
  WS_MD_PHI0,
  WS_BATCH,
  WS_COUNT
};

struct Pending {
  cudaEvent_t a, b;
  int id;
};

// A captured chunk of solver iterations, keyed by the buffers it touches.
struct GraphEntry {
  int kind = 0;
  const void* key[6] = {};
  cudaGraphExec_t exec = nullptr;
  long long last_use = 0;
};

// Launch shape of a tuned kernel: threads per block and grid waves
// (waves <= 0: one work item per thread).
struct Shape {
  int threads = 256;
  int waves = 1;
  int occ = 8;     // resident blocks per SM at this block size
  int tiled = 0;   // FP32 CG pair: 1 = shared-memory tiled kernels, 2 = marching kernels
                   // (threads = cells per block), 4 = grid-stride kernels with two cells
                   // per thread (16-byte accesses; n even)
  int tt = 1;      // tiled or marching: time slices per block
};

// Tile of the fused M M^dagger kernel (fused.cu): Ti x Tj cells per block
// (plus a one-cell ring), Tt time slices per block.
struct FusedShape {
  int Ti = 0, Tj = 0, Tt = 0;
  int tiles_i = 0, tiles_j = 0, tiles_t = 0;
  int D = 2;  // time slices staged ahead of the one in use
  int pairs = 0;  // FP32: two cells per thread (n and Ti even; 16-byte aligned vectors)
};

struct ProfileState {
  bool timing = false;
  long long launches[K_COUNT] = {};
  double ms[K_COUNT] = {};
  double bytes[K_COUNT] = {};  // algorithmic bytes summed over launches
  std::vector<Pending> pending;
  std::vector<cudaEvent_t> free_events;
};

}  // namespace hmc

struct hmc_ctx {
  int device = 0;
  int nsm = 0;
  cudaStream_t stream = nullptr;
  hmc_lattice lat{};
  hmc::Geo geo{};
  double delta = 0.0;
  std::string err;

  bool field_loaded = false;  // E / phi32 hold the field given to hmc_load_field
  const double* loaded_phi = nullptr;

  void* ws[hmc::WS_COUNT] = {};
  size_t ws_bytes[hmc::WS_COUNT] = {};

  double* partials = nullptr;      // reduction partials, kPartials doubles
  double* partA = nullptr;         // per-block partials of the FP32 CG M^dagger kernel
  double* partB = nullptr;         // per-block partials of the FP32 CG M kernel
  unsigned int* tickets = nullptr; // one ticket per concurrent reduction site
  hmc::CGScal* sc = nullptr;       // device CG state (two: FP64 outer, FP32 inner)
  hmc::GridBar* gbar = nullptr;    // grid barrier of the persistent FP32 CG kernel
  hmc::CGScal* sc_host = nullptr;  // pinned mirror
  double* dscal = nullptr;         // device scalar results (64 doubles)
  double* dscal_host = nullptr;    // pinned mirror
  int max_grid = 0;

  hmc::ProfileState prof;

  // CUDA graphs of CG iteration chunks (replayed on `stream`; captured on the
  // private non-blocking `cap_stream`, since the legacy stream cannot capture)
  hmc::Shape shape[hmc::K_COUNT];
  bool tuned32 = false, tuned64 = false;
  int cg32_variant = 0;  // 0 autotune over all designs, 1 grid-stride, 2 tiled, 3 marching,
                         // 4 persistent
  bool persist32 = false;  // the tuner found the persistent FP32 CG kernel fastest
  bool cg1_32 = false;     // the tuner found the single-reduction FP32 CG fastest
  bool resident32 = false;  // the tuner found the resident-tile FP32 CG fastest
  bool cg1_pinned = false;  // its tile was set by the caller
  hmc::FusedShape cg1_shape;  // tile of the single-reduction FP32 CG kernel
  // M M^dagger applications: 0 = choose per precision by timing on first use,
  // 1 = two passes (M^dagger to memory, then M), 2 = the fused kernel
  int apply_variant = 0;
  int apply_choice[2] = {0, 0};     // FP32, FP64: the variant in use (0 = not chosen yet)
  hmc::FusedShape fshape[2];        // FP32, FP64 tiles of the fused kernel
  bool fused_tuned[2] = {false, false};
  // device and pinned host buffers of the batched solver, kept across calls
  // (slot i holds the i-th buffer a call asks for; grown when too small)
  static constexpr int kBatchSlots = 40;
  void* bpool[kBatchSlots] = {};
  size_t bpool_bytes[kBatchSlots] = {};
  void* bpool_host[4] = {};
  size_t bpool_host_bytes[4] = {};
  int bar_extra = 0;         // test hook: extra arrivals every grid barrier waits for
  long long bar_limit = 0;   // test hook: barrier wait limit in SM cycles (0: default)

  // batched FP32 CG: 0 = choose by timing, 1 = graph loop of per-iteration
  // kernels, 2 = one persistent cooperative launch per solve
  int batch_variant = 0;
  int batch_choice = 0;                // the variant chosen (0: not yet)
  float batch_us[2] = {0.f, 0.f};      // us per iteration measured for 1 and 2
  // per-chain contexts of hmc_md_trajectory_batched (slot i: chain i of the
  // last call; recreated when a chain's lattice changes), destroyed with ctx
  std::vector<hmc_ctx*> subs;

  bool use_graphs = true;
  bool use_loop_graphs = true;   // whole solves as one graph with a device-side while loop
  unsigned* loop_trips = nullptr;       // device: [0] trips of the loop so far, [1] bound
  unsigned* loop_trips_host = nullptr;  // pinned mirror
  bool capturing = false;
  bool pdl_armed = false;  // a kernel precedes the next launch in the capture
  cudaStream_t cap_stream = nullptr;
  std::vector<hmc::GraphEntry> graphs;
  long long graph_clock = 0;
};

namespace hmc {

constexpr int kThreads = 256;
constexpr int kMaxGridPerSM = 8;
constexpr int kOneItemBlocksPerSM = 64;
constexpr int kMaxThreads = 512;  // largest block of the tuned CG kernels
constexpr int kMaxRed = 40;  // values reduced at once at most
constexpr int kTickets = 16;

// Record an error message on ctx and return the status.
hmc_status fail(hmc_ctx* c, hmc_status s, const std::string& msg);
// Turn a CUDA error into HMC_ERR_CUDA with a message.
hmc_status cuda_fail(hmc_ctx* c, cudaError_t e, const char* what);

#define HMC_CUDA(ctx, call)                                        \
  do {                                                             \
    cudaError_t e_ = (call);                                       \
    if (e_ != cudaSuccess) return hmc::cuda_fail((ctx), e_, #call); \
  } while (0)

#define HMC_TRY(expr)                  \
  do {                                 \
    hmc_status s_ = (expr);            \
    if (s_ != HMC_OK) return s_;       \
  } while (0)

// Workspace slot of at least `bytes` bytes (grown on demand, never shrunk).
hmc_status ws_get(hmc_ctx* c, int slot, size_t bytes, void** out);

// Device buffers of the context carry guard bands: kGuardBytes before and
// after the `bytes` the caller asked for, filled with kGuardByte. A write past
// either end of a buffer changes a band, which hmc_check_guards reports.
constexpr size_t kGuardBytes = 256;
constexpr unsigned char kGuardByte = 0xA5;
hmc_status guarded_alloc(hmc_ctx* c, size_t bytes, void** user);
void guarded_free(void* user);

// Grid size for a grid-stride kernel over `work` threads.
inline int grid_for(const hmc_ctx* c, long long work) {
  long long g = (work + kThreads - 1) / kThreads;
  if (g > c->max_grid) g = c->max_grid;
  if (g < 1) g = 1;
  return (int)g;
}

// Grid with one thread per work item (up to a cap), for kernels whose loop
// should run once per thread so the block scheduler balances the load.
inline int grid_one(const hmc_ctx* c, long long work) {
  long long g = (work + kThreads - 1) / kThreads;
  const long long cap = (long long)c->nsm * kOneItemBlocksPerSM;
  if (g > cap) g = cap;
  if (g < 1) g = 1;
  return (int)g;
}

// Number of float2 reduction partials the FP32 CG buffers partA / partB hold.
inline long long cg32_part_capacity(const hmc_ctx* c) { return (long long)c->nsm * 2 * kOneItemBlocksPerSM; }

// Grid of a tuned kernel over `work` items.
inline int shape_grid(const hmc_ctx* c, int id, long long work) {
  const Shape& s = c->shape[id];
  if (s.tiled == 4) work = (work + 1) / 2;  // one work item per pair of cells
  if (s.tiled && s.tiled != 4) {  // blocks of the tiled FP32 CG kernels (their reduction partials)
    const Geo& g = c->geo;
    return ((g.V + s.threads - 1) / s.threads) * ((g.nt + s.tt - 1) / s.tt);
  }
  long long g = (work + s.threads - 1) / s.threads;
  if (s.waves > 0) {
    const long long cap = (long long)c->nsm * s.occ * s.waves;
    if (g > cap) g = cap;
  } else {
    const long long cap = (long long)c->nsm * kOneItemBlocksPerSM * 256 / s.threads;
    if (g > cap) g = cap;
  }
  return g < 1 ? 1 : (int)g;
}

// Instrumented launch: counts, and brackets with events when timing is on.
void prof_begin(hmc_ctx* c, int id, cudaEvent_t* a);
void prof_end(hmc_ctx* c, int id, cudaEvent_t a);
// Forget the last n launches of kernel id (counters, algorithmic bytes and any
// pending event pair): launches that found the solve finished and returned at
// entry, so that the counters and timings cover only work that was done.
void prof_discard_last(hmc_ctx* c, int id, long long n, double bytes_each);

// `bytes`: algorithmic bytes of this launch; negative = the kernel's bytes per
// site times the context's site count.
template <typename F>
inline hmc_status launch_b(hmc_ctx* c, int id, double bytes, F&& f) {
  if (c->capturing) {  // recorded into a graph: counted when the graph is replayed
    f();
    cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? HMC_OK : cuda_fail(c, e, kKernelNames[id]);
  }
  cudaEvent_t a = nullptr;
  c->prof.bytes[id] += bytes >= 0 ? bytes : kKernelBytesPerSite[id] * (double)c->geo.N;
  prof_begin(c, id, &a);
  f();
  prof_end(c, id, a);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return cuda_fail(c, e, kKernelNames[id]);
  return HMC_OK;
}

template <typename F>
inline hmc_status launch(hmc_ctx* c, int id, F&& f) {
  return launch_b(c, id, -1.0, f);
}

// Capture the kernels `body` launches into a graph (on cap_stream) and return
// the instantiated executable; the context's stream is restored afterwards.
hmc_status capture_graph(hmc_ctx* c, const std::function<hmc_status()>& body, cudaGraphExec_t* out);
// A graph whose single node is a while loop: `body(handle)` is captured as the
// loop body and must end with a launch that sets the loop condition through
// `handle` (loop_continue_launch); the body repeats while that value is 1.
hmc_status capture_loop_graph(hmc_ctx* c, const std::function<hmc_status(cudaGraphConditionalHandle)>& body,
                              cudaGraphExec_t* out);
// Cached executable for (kind, key) or NULL.
GraphEntry* find_graph(hmc_ctx* c, int kind, const void* const key[6]);
GraphEntry* add_graph(hmc_ctx* c, int kind, const void* const key[6], cudaGraphExec_t exec);
void destroy_graphs(hmc_ctx* c);

// Build the phase tables of phi (or reuse the loaded field when phi is NULL).
hmc_status prepare_field(hmc_ctx* c, const double* phi);

}  // namespace hmc
