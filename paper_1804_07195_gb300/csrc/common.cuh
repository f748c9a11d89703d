// Device-side building blocks shared by the libhmc kernels: lattice geometry
// in the canonical layout, complex arithmetic in float/double, and
// deterministic grid reductions.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace hmc {

// ---------------------------------------------------------------------------
// Unsigned division by a runtime constant d >= 1 for numerators x < 2^31,
// by multiply-high: q = (umulhi(x, mul) + x) >> shift with shift = ceil(log2 d)
// and mul = floor(2^32 (2^shift - d) / d) + 1 (Granlund and Montgomery, 1994).
struct FastDiv {
  uint32_t d, mul, shift;
};

inline FastDiv make_fastdiv(uint32_t d) {
  FastDiv f;
  f.d = d;
  uint32_t s = 0;
  while ((1ull << s) < d) ++s;
  f.shift = s;
  f.mul = (uint32_t)(((1ull << 32) * ((1ull << s) - d)) / d + 1ull);
  return f;
}

inline uint32_t fastdiv_host(uint32_t x, const FastDiv& f) {
  uint32_t hi = (uint32_t)(((uint64_t)x * f.mul) >> 32);
  return (hi + x) >> f.shift;
}

__device__ __forceinline__ uint32_t fdiv(uint32_t x, const FastDiv& f) {
  return (__umulhi(x, f.mul) + x) >> f.shift;
}

// ---------------------------------------------------------------------------
// Geometry of one n x m x nt lattice in the canonical layout
//   idx = ((s*nt + t)*m + j)*n + i.
// Kernels run one thread per "cell-time" q = (t*m + j)*n + i in [0, H) and
// handle the A site q and the B site H + q together.
struct Geo {
  int n, m, nt;
  int V;   // n*m cells per time slice
  int H;   // nt*V sites per sublattice
  int N;   // 2H
  FastDiv fV, fn;
  double dk;  // delta * kappa
  float dkf;  // the same, rounded once on the host for the FP32 kernels
};

__device__ __forceinline__ double geo_dk(const Geo& g, double) { return g.dk; }
__device__ __forceinline__ float geo_dk(const Geo& g, float) { return g.dkf; }

inline Geo make_geo(int n, int m, int nt, double delta, double kappa) {
  Geo g;
  g.n = n;
  g.m = m;
  g.nt = nt;
  g.V = n * m;
  g.H = nt * g.V;
  g.N = 2 * g.H;
  g.fV = make_fastdiv((uint32_t)g.V);
  g.fn = make_fastdiv((uint32_t)n);
  g.dk = delta * kappa;
  g.dkf = (float)g.dk;
  return g;
}

// Indices of everything a thread at cell-time q touches.
struct Nbr {
  int q;             // A(i,j,t); B(i,j,t) is H + q
  int tm, tp;        // same cell at t-1, t+1 (wrapped), within a sublattice half
  int im1, jm1;      // A-row partners: cells (i-1,j), (i,j-1) at t
  int ip1, jp1;      // B-row partners: cells (i+1,j), (i,j+1) at t
  bool wrap_tm;      // t == 0: the t-1 hop wraps (anti-periodic: sign -1)
  bool wrap_tp;      // t == nt-1: the t+1 hop wraps
};

__device__ __forceinline__ Nbr neighbours(const Geo& g, int q) {
  Nbr b;
  b.q = q;
  int t = (int)fdiv((uint32_t)q, g.fV);
  int c = q - t * g.V;
  int j = (int)fdiv((uint32_t)c, g.fn);
  int i = c - j * g.n;
  b.wrap_tm = (t == 0);
  b.wrap_tp = (t == g.nt - 1);
  b.tm = q - g.V + (b.wrap_tm ? g.H : 0);
  b.tp = q + g.V - (b.wrap_tp ? g.H : 0);
  b.im1 = q - 1 + (i == 0 ? g.n : 0);
  b.jm1 = q - g.n + (j == 0 ? g.V : 0);
  b.ip1 = q + 1 - (i == g.n - 1 ? g.n : 0);
  b.jp1 = q + g.n - (j == g.m - 1 ? g.V : 0);
  return b;
}

// ---------------------------------------------------------------------------
// Complex values in the compute precision R (float or double).
template <typename R>
struct Cx {
  R re, im;
};

template <typename R>
struct Vec2;
template <>
struct Vec2<float> {
  using type = float2;
};
template <>
struct Vec2<double> {
  using type = double2;
};

template <typename R>
__device__ __forceinline__ Cx<R> ld(const float2* p, int k) {
  float2 v = p[k];
  return Cx<R>{(R)v.x, (R)v.y};
}
template <typename R>
__device__ __forceinline__ Cx<R> ld(const double2* p, int k) {
  double2 v = p[k];
  return Cx<R>{(R)v.x, (R)v.y};
}
__device__ __forceinline__ void st(float2* p, int k, Cx<float> v) { p[k] = make_float2(v.re, v.im); }
__device__ __forceinline__ void st(float2* p, int k, Cx<double> v) {
  p[k] = make_float2((float)v.re, (float)v.im);
}
__device__ __forceinline__ void st(double2* p, int k, Cx<double> v) { p[k] = make_double2(v.re, v.im); }
__device__ __forceinline__ void st(double2* p, int k, Cx<float> v) {
  p[k] = make_double2((double)v.re, (double)v.im);
}

template <typename R>
__device__ __forceinline__ Cx<R> cneg_if(Cx<R> a, bool neg) {
  return neg ? Cx<R>{-a.re, -a.im} : a;
}

template <typename R>
__device__ __forceinline__ R norm2(Cx<R> a) {
  return a.re * a.re + a.im * a.im;
}

// ---------------------------------------------------------------------------
// Deterministic grid reductions.
//
// Every block reduces its threads' values in a fixed shuffle/shared-memory
// order and writes one partial per value to partials[v * gridDim.x + block].
// The last block to arrive (atomic ticket) sums the partials of every value in
// a fixed order and hands the totals to a finisher run by its thread 0. The
// result therefore does not depend on block scheduling.
constexpr int kMaxBlockThreads = 256;

template <int K>
__device__ __forceinline__ void block_sum(double (&v)[K], double* smem /* K * 32 */) {
#pragma unroll
  for (int k = 0; k < K; ++k) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v[k] += __shfl_xor_sync(0xffffffffu, v[k], o);
  }
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
  if (lane == 0) {
#pragma unroll
    for (int k = 0; k < K; ++k) smem[k * 32 + warp] = v[k];
  }
  __syncthreads();
  if (warp == 0) {
#pragma unroll
    for (int k = 0; k < K; ++k) {
      double x = lane < nw ? smem[k * 32 + lane] : 0.0;
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
      v[k] = x;
    }
  }
  __syncthreads();
}

// Returns true in the last block after the totals were written to `tot` (valid
// in thread 0 of that block only).
template <int K>
__device__ __forceinline__ bool grid_sum(double (&v)[K], double* partials, unsigned int* ticket,
                                         double (&tot)[K]) {
  __shared__ double smem[K * 32];
  __shared__ bool am_last;
  block_sum<K>(v, smem);
  if (threadIdx.x == 0) {
#pragma unroll
    for (int k = 0; k < K; ++k) partials[k * gridDim.x + blockIdx.x] = v[k];
    __threadfence();
    unsigned int t = atomicAdd(ticket, 1u);
    am_last = (t == gridDim.x - 1);
  }
  __syncthreads();
  if (!am_last) return false;
  __threadfence();
  double w[K];
#pragma unroll
  for (int k = 0; k < K; ++k) {
    double acc = 0.0;
    for (int b = threadIdx.x; b < (int)gridDim.x; b += blockDim.x)
      acc += __ldcg(&partials[k * gridDim.x + b]);
    w[k] = acc;
  }
  block_sum<K>(w, smem);
  if (threadIdx.x == 0) {
#pragma unroll
    for (int k = 0; k < K; ++k) tot[k] = w[k];
    *ticket = 0u;
  }
  return true;
}

// ---------------------------------------------------------------------------
// Programmatic dependent launch (sm_90+): a kernel launched with the
// programmatic-serialization attribute may be scheduled before the previous
// kernel in the stream has finished; pdl_wait() blocks until that kernel has
// completed and its memory is visible, and pdl_trigger() lets the next kernel
// start launching once every block of this one has passed it. Both are no-ops
// for an ordinary launch.
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void pdl_trigger() { asm volatile("griddepcontrol.launch_dependents;" :::); }

// ---------------------------------------------------------------------------
// Device-side scalar state of one CG solve (shared by the FP64 and FP32 paths).
struct CGScal {
  double rr;     // |r|^2 of the current residual
  double pAp;    // <p, A p>
  double alpha, beta;
  double bb;     // |b|^2
  double thresh; // stop when rr <= thresh (= tol^2 |b|^2)
  double sigma;  // shift of the operator
  double dm;     // delta * m_s of the operator (read by the iteration kernels)
  double rr_cur; // FP32 pair: |r|^2 of the iteration in progress
  int iter, maxit;
  int done;      // 0 running, 1 converged, 2 iteration limit, 3 breakdown (pAp <= 0 / NaN)
  int first;     // FP32 pair: no direction yet (beta = 0)
  float dm32, sigma32;  // dm and sigma rounded once for the FP32 kernels
  // single-reduction FP32 CG: gamma = |r|^2, alpha and the iteration count,
  // in two slots that successive launches read and write alternately
  double cg1_gamma[2], cg1_alpha[2];
  int cg1_it[2];
  // rr, rr_cur and thresh rounded to float for the FP32 CG kernels
  float rr32, rr_cur32, thresh32;
};

enum { CG_RUNNING = 0, CG_CONVERGED = 1, CG_MAXIT = 2, CG_BREAKDOWN = 3, CG_TIMEOUT = 4 };

// State of a grid-wide barrier between the co-resident blocks of a cooperative
// launch: one arrival word, `count`, whose top bit flips each time every block
// has arrived (`gen` is unused); `err` is set when a wait gave up (every later
// barrier then returns at once). The host zeroes it before each launch.
struct GridBar {
  unsigned count;
  unsigned gen;
  int err;
  int pad;
};

__device__ __forceinline__ unsigned ld_acquire_gpu(const unsigned* p) {
  unsigned v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ unsigned atom_add_release_gpu(unsigned* p, unsigned x) {
  unsigned v;
  asm volatile("atom.release.gpu.global.add.u32 %0, [%1], %2;" : "=r"(v) : "l"(p), "r"(x) : "memory");
  return v;
}

// Barrier over all blocks of a cooperative launch. One atomic per block and
// no reset: block 0 adds 2^31 - (nblocks - 1), every other block adds 1, so
// the word grows by exactly 2^31 per barrier and its top bit changes only
// when the last block arrives; a block waits until the top bit differs from
// the one its own atomic returned. Its add is a release and its polls are
// acquires, so every write before the barrier is visible after it. The wait
// of each block is bounded by `limit` SM clock cycles: a block that gives up
// sets gb->err, and every later barrier returns false at once, so the kernel
// can leave cleanly (the host reports a timeout). Returns true when the
// barrier was passed.
__device__ __forceinline__ bool grid_barrier(GridBar* gb, unsigned nblocks, long long limit) {
  __shared__ int s_ok;
  __syncthreads();
  if (threadIdx.x == 0 && threadIdx.y == 0 && threadIdx.z == 0) {
    volatile int* verr = &gb->err;
    int ok = (*verr == 0);
    if (ok) {
      const bool lead = blockIdx.x == 0 && blockIdx.y == 0 && blockIdx.z == 0;
      __threadfence();  // the block's writes (ordered before this thread by __syncthreads) at GPU scope
      const unsigned old = atom_add_release_gpu(&gb->count, lead ? 0x80000000u - (nblocks - 1u) : 1u);
      const long long t0 = clock64();
      unsigned spins = 0;
      while (((ld_acquire_gpu(&gb->count) ^ old) & 0x80000000u) == 0u) {
        if ((++spins & 31u) == 0u) {
          if (*verr) {
            ok = 0;
            break;
          }
          if (clock64() - t0 > limit) {
            atomicExch(&gb->err, 1);
            ok = 0;
            break;
          }
        }
      }
    }
    s_ok = ok;
  }
  __syncthreads();
  return s_ok != 0;
}

// ---------------------------------------------------------------------------
// The FP32 kernels' copy of the field: phi reduced to [-pi, pi] in FP64, then
// rounded to float. The kernels evaluate e^{i phi} from it with the hardware
// sine and cosine, whose error bound is stated for that interval, and need
// no reduction of their own; a field of any size keeps the float's full
// relative precision on its phase.
__device__ __forceinline__ float phi_to_f32(double x) {
  return (float)fma(-6.283185307179586, rint(x * 0.15915494309189535), x);
}

// ---------------------------------------------------------------------------
// Float-float sums for the FP32 kernels. GB300 executes FP64 at 1/58 of the FP32
// rate, so the single-precision kernels keep their reductions off the FP64
// pipe: a value is an unevaluated pair (hi, lo) of floats, and two pairs add
// with Knuth's TwoSum plus a renormalisation (about 48 significant bits).
__device__ __forceinline__ float2 ff_add(float2 a, float2 b) {
  const float s = a.x + b.x;
  const float v = s - a.x;
  float e = (a.x - (s - v)) + (b.x - v);
  e += a.y + b.y;
  const float hi = s + e;
  return make_float2(hi, e - (hi - s));
}

// Block sum of v in a fixed order; the result is valid in thread 0.
__device__ __forceinline__ float2 ff_block_sum(float2 v) {
  __shared__ float2 sm[32];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    float2 w = make_float2(__shfl_xor_sync(0xffffffffu, v.x, o), __shfl_xor_sync(0xffffffffu, v.y, o));
    v = ff_add(v, w);
  }
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
  if (lane == 0) sm[warp] = v;
  __syncthreads();
  if (warp == 0) {
    v = lane < nw ? sm[lane] : make_float2(0.f, 0.f);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      float2 w = make_float2(__shfl_xor_sync(0xffffffffu, v.x, o), __shfl_xor_sync(0xffffffffu, v.y, o));
      v = ff_add(v, w);
    }
  }
  return v;
}

// Thread 0 writes the block's sum of loc to part[blockIdx.x].
__device__ __forceinline__ void ff_write_partial(float loc, float2* part) {
  float2 v = ff_block_sum(make_float2(loc, 0.f));
  if (threadIdx.x == 0) part[blockIdx.x] = v;
}

// Sum of G float-float partials in a fixed order (identical in every block);
// valid in thread 0 of the calling block, as a double.
// The pair is returned to every thread; only the thread that forms the
// block's scalars widens it to double (ff_to_double), so no other thread
// issues an FP64 instruction.
__device__ __forceinline__ float2 ff_sum_partials(const float2* __restrict__ part, int G) {
  float2 v = make_float2(0.f, 0.f);
  for (int b = threadIdx.x; b < G; b += blockDim.x) v = ff_add(v, __ldcg(part + b));
  return ff_block_sum(v);
}
__device__ __forceinline__ double ff_to_double(float2 v) { return (double)v.x + (double)v.y; }

// Scalars of the FP32 CG pair, formed by thread 0 of every block of the
// kernel in FP32 (on this GPU the FP64 pipe is slow, and the rest of the block
// waits for them); the lead block also records them in FP64 for the host.
// First kernel of an iteration: |r|^2 from the second kernel's partials (the
// init kernel's value on the first iteration), the convergence and limit
// checks and beta; returns the CG state (CG_RUNNING to go on).
__device__ __forceinline__ int cg32_scalars_first(CGScal* sc, bool first, float2 rr_pair, bool lead, float* beta) {
  const float rr = first ? sc->rr_cur32 : rr_pair.x + rr_pair.y;
  int done = CG_RUNNING;
  if (!isfinite(rr))
    done = CG_BREAKDOWN;
  else if (rr <= sc->thresh32)
    done = CG_CONVERGED;
  else if (sc->iter >= sc->maxit)
    done = CG_MAXIT;
  const float b = first ? 0.f : rr / sc->rr32;
  *beta = b;
  if (lead) {
    sc->rr_cur32 = rr;
    sc->rr_cur = rr;
    sc->beta = b;
    if (done) {
      sc->rr32 = rr;
      sc->rr = rr;
      sc->done = done;
    }
  }
  return done;
}
// Second kernel: <p, A p> from the first kernel's partials and alpha;
// returns true on a breakdown (non-positive or non-finite curvature).
__device__ __forceinline__ bool cg32_scalars_second(CGScal* sc, float2 pAp_pair, bool lead, float* alpha) {
  const float pAp = pAp_pair.x + pAp_pair.y;
  const float rr = sc->rr_cur32;
  const bool bad = !(pAp > 0.f) || !isfinite(pAp);
  const float a = bad ? 0.f : rr / pAp;
  *alpha = a;
  if (lead) {
    sc->pAp = pAp;
    sc->rr32 = rr;
    sc->rr = sc->rr_cur;
    sc->first = 0;
    if (bad) {
      sc->alpha = 0.0;
      sc->done = CG_BREAKDOWN;
    } else {
      sc->alpha = a;
      sc->iter += 1;
    }
  }
  return bad;
}

}  // namespace hmc
