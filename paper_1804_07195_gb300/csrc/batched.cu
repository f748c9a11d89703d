// Batched solves of many independent systems (M_s M_s^dagger + sigma_s) x_s = b_s,
// lattices of uneven sizes, in one launch per kernel: the CG of Section 3 and
// the FGMRES of Algorithm A.1 run for every system at once, each with its own
// operator of Eq. ferm_op (lattice, phases, staggered mass).
//
// Layout: the systems' vectors are concatenated; system s occupies sites
// [off_s, off_s + N_s) in its own canonical order. Every block belongs to one
// system (a block table maps block -> system), so a block's reduction partial
// is per system and the last block of a system (per-system ticket) finishes
// that system's scalars. A system that has converged is masked: its blocks
// return at once. Chunks of CG iterations are captured into a CUDA graph and
// replayed until every system is done.
//
// mixed = 0: CG in FP64 to |r| <= tol |b|.
// mixed = 1: FP64 defect correction: r = b - A x in FP64, an FP32 CG solve of
//            A e = r, x += e, repeated until the FP64 true residual meets tol.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <map>
#include <vector>

#include "operator.cuh"
#include "solvers.h"
#include "trace.h"
#include "validate.h"

namespace hmc {

struct BSys {
  Geo g;
  long long off;     // first site of the system in the concatenated vectors
  int block0, nblocks;
  double dm, sigma;
  const double* phi; // the caller's field (phase kernel only)
  int maxit;         // iteration limit of this system's CG
  float dm32, sigma32;  // dm and sigma rounded to float for the FP32 kernels
};

struct BState {
  CGScal cg;
  int active;  // 1 while the system takes part in the current inner solve
  float alpha32, beta32;  // cg.alpha and cg.beta rounded to float, written once per system
};

// Sum K values over the blocks [base, base + count) of one system, in a fixed
// order; true in the last block of the group (totals in thread 0).
template <int K>
__device__ __forceinline__ bool group_sum(double (&v)[K], double* partials, int base, int count,
                                          unsigned* ticket, double (&tot)[K]) {
  __shared__ double smem[K * 32];
  __shared__ bool am_last;
  block_sum<K>(v, smem);
  if (threadIdx.x == 0) {
#pragma unroll
    for (int k = 0; k < K; ++k) partials[(size_t)k * gridDim.x + blockIdx.x] = v[k];
    __threadfence();
    unsigned t = atomicAdd(ticket, 1u);
    am_last = (t == (unsigned)count - 1u);
  }
  __syncthreads();
  if (!am_last) return false;
  __threadfence();
  double w[K];
#pragma unroll
  for (int k = 0; k < K; ++k) {
    double acc = 0.0;
    for (int b = threadIdx.x; b < count; b += blockDim.x) acc += __ldcg(&partials[(size_t)k * gridDim.x + base + b]);
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

// Block total of per-thread partial sums, valid in thread 0: FP32 sums use the
// float-float reduction (no FP64 instruction per thread), FP64 sums the
// double shuffle reduction.
__device__ __forceinline__ double block_total(float v) {
  float2 t = ff_block_sum(make_float2(v, 0.f));
  return threadIdx.x == 0 ? ff_to_double(t) : 0.0;
}
__device__ __forceinline__ double block_total(double v) {
  __shared__ double sm[32];
  double a[1] = {v};
  block_sum<1>(a, sm);
  return a[0];
}

// Second half of group_sum: thread 0 holds the block total; the last block of
// the system's group sums the partials (in FP64, that block only).
__device__ __forceinline__ bool group_finish(double blocktot, double* partials, int base, int count,
                                             unsigned* ticket, double* tot, int vb) {
  __shared__ bool am_last;
  if (threadIdx.x == 0) {
    partials[vb] = blocktot;
    __threadfence();
    unsigned t = atomicAdd(ticket, 1u);
    am_last = (t == (unsigned)count - 1u);
  }
  __syncthreads();
  if (!am_last) return false;
  __threadfence();
  __shared__ double sm[32];
  double w[1] = {0.0};
  for (int b = threadIdx.x; b < count; b += blockDim.x) w[0] += __ldcg(&partials[base + b]);
  block_sum<1>(w, sm);
  if (threadIdx.x == 0) {
    *tot = w[0];
    *ticket = 0u;
  }
  return true;
}

// Scalars of a system in the compute precision, read once per block by
// thread 0: the FP32 kernels read float copies written once per system, so
// no block waits on FP64 conversions (slow on this GPU) in its prologue.
template <typename R>
struct BScal {
  R dm, sigma, coef;
  static __device__ __forceinline__ void from(const BSys& S, const BState& st, bool alpha, BScal* out) {
    if constexpr (sizeof(R) == 4) {
      out->dm = S.dm32;
      out->sigma = S.sigma32;
      out->coef = alpha ? st.alpha32 : st.beta32;
    } else {
      out->dm = S.dm;
      out->sigma = S.sigma;
      out->coef = alpha ? st.cg.alpha : st.cg.beta;
    }
  }
};

#define BLOCK_SYS()                                  \
  __shared__ BSys S_;                                \
  const int s_ = bsys[blockIdx.x];                   \
  if (threadIdx.x == 0) S_ = sys[s_];                \
  __syncthreads();                                   \
  const Geo& g = S_.g;                               \
  const int lb = blockIdx.x - S_.block0;             \
  const int stride = S_.nblocks * blockDim.x

// The same for virtual block vb of a persistent launch, whose blocks take one
// virtual block after another (the leading barrier keeps the previous one's
// readers of the shared copy ahead of the new write).
#define VBLOCK_SYS(vb)                               \
  __shared__ BSys S_;                                \
  const int s_ = bsys[vb];                           \
  __syncthreads();                                   \
  if (threadIdx.x == 0) S_ = sys[s_];                \
  __syncthreads();                                   \
  const Geo& g = S_.g;                               \
  const int lb = (vb) - S_.block0;                   \
  const int stride = S_.nblocks * blockDim.x

// VBLOCK_SYS for the CG iteration kernels, with the system's state: thread 0
// issues the loads of the descriptor, the done flag and the scalars together
// (one L2 round trip after the block's system index, not two), then one
// barrier publishes S_, sc and skip.
#define VBLOCK_SYS_CG(vb, ALPHA)                     \
  __shared__ BSys S_;                                \
  __shared__ BScal<R> sc;                            \
  __shared__ int skip;                               \
  const int s_ = bsys[vb];                           \
  __syncthreads();                                   \
  if (threadIdx.x == 0) {                            \
    const BSys sl = sys[s_];                         \
    skip = bst[s_].cg.done;                          \
    BScal<R>::from(sl, bst[s_], ALPHA, &sc);         \
    S_ = sl;                                         \
  }                                                  \
  __syncthreads();                                   \
  const Geo& g = S_.g;                               \
  const int lb = (vb) - S_.block0;                   \
  const int stride = S_.nblocks * blockDim.x

__global__ void kb_phase(const BSys* __restrict__ sys, const int* __restrict__ bsys,
                         double2* __restrict__ E, float* __restrict__ phi32) {
  BLOCK_SYS();
  for (int k = lb * blockDim.x + threadIdx.x; k < g.N; k += stride) {
    double x = S_.phi[k], s, c;
    sincos(x, &s, &c);
    E[S_.off + k] = make_double2(c, s);
    phi32[S_.off + k] = phi_to_f32(x);
  }
}

template <typename R>
struct BPhase;
template <>
struct BPhase<double> {
  static __device__ __forceinline__ Phase<double> at(const double2* E, const float*, long long off) {
    return Phase<double>{E + off};
  }
};
template <>
struct BPhase<float> {
  static __device__ __forceinline__ Phase<float> at(const double2*, const float* p32, long long off) {
    return Phase<float>{p32 + off};
  }
};

// x = 0, r = p = b; |b|^2; state init with thresh = tol2[s] |b|^2 (inactive
// systems are marked done).
template <typename R>
__global__ void kb_init(const BSys* __restrict__ sys, const int* __restrict__ bsys, BState* bst,
                        const double* __restrict__ tol2, const V2<R>* __restrict__ b, V2<R>* __restrict__ x,
                        V2<R>* __restrict__ r, V2<R>* __restrict__ p, int maxit, double* partials,
                        unsigned* tickets) {
  BLOCK_SYS();
  double acc[1] = {0.0};
  for (int k = lb * blockDim.x + threadIdx.x; k < g.N; k += stride) {
    const long long i = S_.off + k;
    Cx<R> bk = ld<R>(b, i);
    st(x, i, Cx<R>{(R)0, (R)0});
    st(r, i, bk);
    st(p, i, bk);
    acc[0] += (double)norm2(bk);
  }
  double tot[1];
  if (group_sum<1>(acc, partials, S_.block0, S_.nblocks, tickets + s_, tot) && threadIdx.x == 0) {
    CGScal& c = bst[s_].cg;
    c.rr = c.bb = tot[0];
    c.thresh = tol2[s_] * tot[0];
    c.sigma = S_.sigma;
    c.iter = 0;
    c.maxit = min(maxit, S_.maxit);
    c.alpha = c.beta = c.pAp = 0.0;
    bst[s_].alpha32 = bst[s_].beta32 = 0.f;
    c.done = (!bst[s_].active || tot[0] <= c.thresh) ? CG_CONVERGED : CG_RUNNING;
    if (!isfinite(tot[0])) c.done = CG_BREAKDOWN;
  }
}

// p_new = r + beta p_old (beta = 0 on a system's first iteration), evaluated
// at every stencil point it reads; u = M^dagger p_new; per-system <p, A p>.
template <typename R>
__device__ __forceinline__ void pmdag_body(int vb, const BSys* __restrict__ sys, const int* __restrict__ bsys,
                                           BState* bst, const double2* __restrict__ E,
                                           const float* __restrict__ p32, const V2<R>* __restrict__ r,
                                           const V2<R>* __restrict__ pold, V2<R>* __restrict__ pnew,
                                           V2<R>* __restrict__ u, double* partials, unsigned* tickets,
                                           unsigned* ndone) {
  VBLOCK_SYS_CG(vb, false);
  if (skip) return;
  const Phase<R> ph = BPhase<R>::at(E, p32, S_.off);
  const R dm = sc.dm, sigma = sc.sigma, beta = sc.coef, dk = geo_dk(g, R(0));
  const V2<R>* rs = r + S_.off;
  const V2<R>* pos = pold + S_.off;
  V2<R>* pns = pnew + S_.off;
  V2<R>* us = u + S_.off;
  auto P = [&](int k) {
    const Cx<R> a = ld<R>(rs, k), bb = ld<R>(pos, k);
    return Cx<R>{fma(beta, bb.re, a.re), fma(beta, bb.im, a.im)};
  };
  R loc = 0;
  for (int q = lb * blockDim.x + threadIdx.x; q < g.H; q += stride) {
    const Nbr nb = neighbours(g, q);
    const Cx<R> ea = ph(nb.tp);
    const Cx<R> za = cneg_if(Cx<R>{ea.re - dm, -ea.im}, nb.wrap_tp);
    const Cx<R> eb = ph(g.H + nb.tm);
    const Cx<R> zb = cneg_if(Cx<R>{dm - eb.re, -eb.im}, nb.wrap_tm);
    const PairOut<R> o = mdag_pair_ld<R>(g, za, zb, dk, nb, P);
    const Cx<R> pa = P(q), pb = P(g.H + q);
    st(pns, q, pa);
    st(pns, g.H + q, pb);
    st(us, q, o.a);
    st(us, g.H + q, o.b);
    loc += norm2(o.a) + norm2(o.b);
    if (sigma != (R)0) loc += sigma * (norm2(pa) + norm2(pb));
  }
  const double bt = block_total(loc);
  double tot;
  if (group_finish(bt, partials, S_.block0, S_.nblocks, tickets + s_, &tot, vb) && threadIdx.x == 0) {
    CGScal& c = bst[s_].cg;
    c.pAp = tot;
    if (!(tot > 0.0) || !isfinite(tot)) {
      c.alpha = 0.0;
      c.done = CG_BREAKDOWN;
      atomicAdd(ndone, 1u);
    } else {
      c.alpha = c.rr / tot;
    }
    bst[s_].alpha32 = (float)c.alpha;
  }
}

template <typename R>
__global__ void __launch_bounds__(512) kb_cg_pmdag(const BSys* __restrict__ sys, const int* __restrict__ bsys,
                                                   BState* bst, const double2* __restrict__ E,
                                                   const float* __restrict__ p32, const V2<R>* __restrict__ r,
                                                   const V2<R>* __restrict__ pold, V2<R>* __restrict__ pnew,
                                                   V2<R>* __restrict__ u, double* partials, unsigned* tickets,
                                                   unsigned* ndone) {
  pmdag_body<R>(blockIdx.x, sys, bsys, bst, E, p32, r, pold, pnew, u, partials, tickets, ndone);
}

template <typename R>
__device__ __forceinline__ void m_body(int vb, const BSys* __restrict__ sys, const int* __restrict__ bsys,
                                       BState* bst, const double2* __restrict__ E,
                                       const float* __restrict__ p32, const V2<R>* __restrict__ u,
                                       const V2<R>* __restrict__ p, V2<R>* __restrict__ x,
                                       V2<R>* __restrict__ r, double* partials, unsigned* tickets,
                                       unsigned* ndone) {
  VBLOCK_SYS_CG(vb, true);
  if (skip) return;
  const Phase<R> ph = BPhase<R>::at(E, p32, S_.off);
  const R dm = sc.dm, sigma = sc.sigma, alpha = sc.coef;
  const V2<R>* us = u + S_.off;
  R loc = 0;
  for (int q = lb * blockDim.x + threadIdx.x; q < g.H; q += stride) {
    Nbr nb = neighbours(g, q);
    PairOut<R> o = m_pair<R>(g, ph, dm, us, nb);
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const long long k = S_.off + (h ? g.H + q : q);
      Cx<R> Ap = h ? o.b : o.a;
      Cx<R> pk = ld<R>(p, k), xk = ld<R>(x, k), rk = ld<R>(r, k);
      Ap.re = fma(sigma, pk.re, Ap.re);
      Ap.im = fma(sigma, pk.im, Ap.im);
      xk.re = fma(alpha, pk.re, xk.re);
      xk.im = fma(alpha, pk.im, xk.im);
      rk.re = fma(-alpha, Ap.re, rk.re);
      rk.im = fma(-alpha, Ap.im, rk.im);
      st(x, k, xk);
      st(r, k, rk);
      loc += norm2(rk);
    }
  }
  const double bt = block_total(loc);
  double tot;
  if (group_finish(bt, partials, S_.block0, S_.nblocks, tickets + s_, &tot, vb) && threadIdx.x == 0) {
    CGScal& c = bst[s_].cg;
    const double rr = tot;
    c.beta = rr / c.rr;
    bst[s_].beta32 = (float)c.beta;
    c.rr = rr;
    c.iter += 1;
    if (!isfinite(rr))
      c.done = CG_BREAKDOWN;
    else if (rr <= c.thresh)
      c.done = CG_CONVERGED;
    else if (c.iter >= c.maxit)
      c.done = CG_MAXIT;
    if (c.done) atomicAdd(ndone, 1u);
  }
}

template <typename R>
__global__ void __launch_bounds__(512) kb_cg_m(const BSys* __restrict__ sys, const int* __restrict__ bsys,
                                               BState* bst, const double2* __restrict__ E,
                                               const float* __restrict__ p32, const V2<R>* __restrict__ u,
                                               const V2<R>* __restrict__ p, V2<R>* __restrict__ x,
                                               V2<R>* __restrict__ r, double* partials, unsigned* tickets,
                                               unsigned* ndone) {
  m_body<R>(blockIdx.x, sys, bsys, bst, E, p32, u, p, x, r, partials, tickets, ndone);
}

// The batched CG as ONE persistent cooperative launch: the grid's blocks take
// the plan's virtual blocks (one group per system) in turn, and the two halves
// of an iteration -- the same bodies as kb_cg_pmdag and kb_cg_m -- are
// separated by grid barriers instead of kernel boundaries. Every 8 iterations
// the blocks read the count of finished systems between two barriers (no body
// runs there, so all blocks read the same count) and leave together once every
// running system is done. Barrier waits are bounded: a wait that gives up sets
// gb->err and every block leaves.
template <typename R>
__global__ void __launch_bounds__(512) kb_cg_persist(const BSys* __restrict__ sys, const int* __restrict__ bsys,
                                                     int nvb, BState* bst, const double2* __restrict__ E,
                                                     const float* __restrict__ p32, V2<R>* __restrict__ x,
                                                     V2<R>* __restrict__ r, V2<R>* __restrict__ p,
                                                     V2<R>* __restrict__ q, V2<R>* __restrict__ u, double* partials,
                                                     unsigned* tickets, unsigned* ndone, unsigned target,
                                                     int max_iters, GridBar* gb, long long limit,
                                                     unsigned expect) {
  for (int it = 0; it < max_iters; ++it) {
    V2<R>* pold = (it & 1) ? q : p;
    V2<R>* pnew = (it & 1) ? p : q;
    for (int vb = blockIdx.x; vb < nvb; vb += gridDim.x)
      pmdag_body<R>(vb, sys, bsys, bst, E, p32, r, pold, pnew, u, partials, tickets, ndone);
    if (!grid_barrier(gb, expect, limit)) return;
    for (int vb = blockIdx.x; vb < nvb; vb += gridDim.x)
      m_body<R>(vb, sys, bsys, bst, E, p32, u, pnew, x, r, partials, tickets, ndone);
    if (!grid_barrier(gb, expect, limit)) return;
    if ((it & 7) == 7) {
      const unsigned d = __ldcg(ndone);
      if (!grid_barrier(gb, expect, limit)) return;
      if (d >= target) return;
    }
  }
}

// Condition of the batched device-side loop: continue while fewer than
// `target` systems have finished and the trip count is below trips[1].
__global__ void kb_loop_continue(cudaGraphConditionalHandle h, const unsigned* ndone, unsigned target,
                                 unsigned* trips) {
  if (threadIdx.x == 0) {
    const unsigned t = trips[0] + 1u;
    trips[0] = t;
    cudaGraphSetConditional(h, (*ndone < target && t < trips[1]) ? 1u : 0u);
  }
}

// FP64 u = M^dagger x for every system (plain)
__global__ void __launch_bounds__(512) kb_mdag64(const BSys* __restrict__ sys, const int* __restrict__ bsys,
                                                 const double2* __restrict__ E, const double2* __restrict__ x,
                                                 double2* __restrict__ u) {
  BLOCK_SYS();
  const Phase<double> ph{E + S_.off};
  for (int q = lb * blockDim.x + threadIdx.x; q < g.H; q += stride) {
    Nbr nb = neighbours(g, q);
    PairOut<double> o = mdag_pair<double>(g, ph, S_.dm, x + S_.off, nb);
    st(u + S_.off, q, o.a);
    st(u + S_.off, g.H + q, o.b);
  }
}

// FP64 r = b - (M u + sigma x), per-system |r|^2, |b|^2 into rrbb[2 s]; the
// FP32 copy r32 = r (the right-hand side of the next inner solve).
__global__ void __launch_bounds__(512) kb_resid64(const BSys* __restrict__ sys, const int* __restrict__ bsys,
                                                  const double2* __restrict__ E, const double2* __restrict__ u,
                                                  const double2* __restrict__ x, const double2* __restrict__ b,
                                                  double2* __restrict__ r, float2* __restrict__ r32,
                                                  double* rrbb, double* partials, unsigned* tickets) {
  BLOCK_SYS();
  const Phase<double> ph{E + S_.off};
  double acc[2] = {0.0, 0.0};
  for (int q = lb * blockDim.x + threadIdx.x; q < g.H; q += stride) {
    Nbr nb = neighbours(g, q);
    PairOut<double> o = m_pair<double>(g, ph, S_.dm, u + S_.off, nb);
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const long long k = S_.off + (h ? g.H + q : q);
      Cx<double> Ax = h ? o.b : o.a;
      double2 xk = x[k], bk = b[k];
      double2 rk = make_double2(bk.x - fma(S_.sigma, xk.x, Ax.re), bk.y - fma(S_.sigma, xk.y, Ax.im));
      r[k] = rk;
      if (r32) r32[k] = make_float2((float)rk.x, (float)rk.y);
      acc[0] = fma(rk.x, rk.x, fma(rk.y, rk.y, acc[0]));
      acc[1] = fma(bk.x, bk.x, fma(bk.y, bk.y, acc[1]));
    }
  }
  double tot[2];
  if (group_sum<2>(acc, partials, S_.block0, S_.nblocks, tickets + s_, tot) && threadIdx.x == 0) {
    rrbb[2 * s_] = tot[0];
    rrbb[2 * s_ + 1] = tot[1];
  }
}

// x += (double) e for active systems
__global__ void __launch_bounds__(512) kb_xadd(const BSys* __restrict__ sys, const int* __restrict__ bsys,
                                               const BState* bst, const float2* __restrict__ e,
                                               double2* __restrict__ x) {
  BLOCK_SYS();
  if (!bst[s_].active) return;
  for (int k = lb * blockDim.x + threadIdx.x; k < g.N; k += stride) {
    const long long i = S_.off + k;
    float2 ev = e[i];
    double2 xv = x[i];
    x[i] = make_double2(xv.x + (double)ev.x, xv.y + (double)ev.y);
  }
}

// ---------------------------------------------------------------------------

struct BatchWs {
  long long Ntot = 0;
  int nsys = 0;
  int blocks = 0;
  int threads = 256;
  std::vector<BSys> hsys;
  std::vector<int> hbsys;
  BSys* sys = nullptr;
  int* bsys = nullptr;
  BState* st = nullptr;
  BState* st_host = nullptr;
  double* tol2 = nullptr;
  double* rrbb = nullptr;
  double* rrbb_host = nullptr;
  unsigned* tickets = nullptr;
  unsigned* ndone = nullptr;
  unsigned* ndone_host = nullptr;
  double* partials = nullptr;
  double2 *E = nullptr, *x = nullptr, *b = nullptr, *r = nullptr, *p = nullptr, *q = nullptr, *u = nullptr;
  float *phi32 = nullptr;
  float2 *r32 = nullptr, *e32 = nullptr, *p32v = nullptr, *q32v = nullptr, *u32 = nullptr, *rr32 = nullptr;
  int nalloc = 0;  // pool slots taken by this call
  std::vector<void*> allocs;
};

// Device buffers come from the context's pool: the i-th request of a call
// takes slot i, reallocated only when it is too small for this batch.
static hmc_status bmalloc(hmc_ctx* c, BatchWs& w, void** p, size_t bytes) {
  if (bytes < 16) bytes = 16;
  const int slot = w.nalloc++;
  if (slot >= hmc_ctx::kBatchSlots) return fail(c, HMC_ERR_NOMEM, "batched workspace: too many buffers");
  if (c->bpool_bytes[slot] < bytes) {
    if (c->bpool[slot]) guarded_free(c->bpool[slot]);
    c->bpool[slot] = nullptr;
    c->bpool_bytes[slot] = 0;
    void* p = nullptr;
    if (guarded_alloc(c, bytes, &p) != HMC_OK) return fail(c, HMC_ERR_NOMEM, "batched workspace allocation failed");
    c->bpool[slot] = p;
    c->bpool_bytes[slot] = bytes;
  }
  *p = c->bpool[slot];
  return HMC_OK;
}

// Pinned host mirrors, also pooled (slot 0: states, 1: residual norms, 2: count).
static hmc_status bmalloc_host(hmc_ctx* c, int slot, void** p, size_t bytes) {
  if (c->bpool_host_bytes[slot] < bytes) {
    if (c->bpool_host[slot]) cudaFreeHost(c->bpool_host[slot]);
    c->bpool_host[slot] = nullptr;
    c->bpool_host_bytes[slot] = 0;
    HMC_CUDA(c, cudaMallocHost(&c->bpool_host[slot], bytes));
    c->bpool_host_bytes[slot] = bytes;
  }
  *p = c->bpool_host[slot];
  return HMC_OK;
}

static void bfree(BatchWs& w) {
  // pooled buffers stay with the context
  w.allocs.clear();
  w.st_host = nullptr;
  w.rrbb_host = nullptr;
  w.ndone_host = nullptr;
}

// Build the block table for `threads` threads per block and `ipt` cell-times
// per thread; returns the total block count.
static int plan_blocks(BatchWs& w, int threads, int ipt) {
  int b = 0;
  w.hbsys.clear();
  for (int s = 0; s < w.nsys; ++s) {
    BSys& S = w.hsys[s];
    const long long work = std::max(S.g.H, 1);
    int nb = (int)((work + (long long)threads * ipt - 1) / ((long long)threads * ipt));
    nb = std::max(nb, 1);
    S.block0 = b;
    S.nblocks = nb;
    for (int i = 0; i < nb; ++i) w.hbsys.push_back(s);
    b += nb;
  }
  w.blocks = b;
  w.threads = threads;
  return b;
}

// Kernel sequence of one CG iteration for all systems, in precision R.
// (iteration i reads the direction from p when i is even and from q when odd,
// and writes the new one into the other buffer)
template <typename R>
static void cg_iteration(const BatchWs& w, cudaStream_t s, V2<R>* x, V2<R>* r, V2<R>* p, V2<R>* q, V2<R>* u,
                         int i) {
  const dim3 G(w.blocks), T(w.threads);
  V2<R>* pold = (i & 1) ? q : p;
  V2<R>* pnew = (i & 1) ? p : q;
  kb_cg_pmdag<R><<<G, T, 0, s>>>(w.sys, w.bsys, w.st, w.E, w.phi32, r, pold, pnew, u, w.partials, w.tickets,
                                  w.ndone);
  kb_cg_m<R><<<G, T, 0, s>>>(w.sys, w.bsys, w.st, w.E, w.phi32, u, pnew, x, r, w.partials, w.tickets, w.ndone);
}

// Tuned (threads, cell-times per thread) per precision and size bucket.
struct TuneKey {
  int prec, bucket;
  bool operator<(const TuneKey& o) const { return prec != o.prec ? prec < o.prec : bucket < o.bucket; }
};
static std::map<TuneKey, std::pair<int, int>> g_tuned;

template <typename R>
static hmc_status upload_plan(hmc_ctx* c, BatchWs& w, cudaStream_t s) {
  HMC_CUDA(c, cudaMemcpyAsync(w.sys, w.hsys.data(), sizeof(BSys) * w.nsys, cudaMemcpyHostToDevice, s));
  HMC_CUDA(c, cudaMemcpyAsync(w.bsys, w.hbsys.data(), sizeof(int) * w.blocks, cudaMemcpyHostToDevice, s));
  return HMC_OK;
}

// Time a few CG iterations of each candidate block shape on this batch and
// keep the fastest for the (precision, size) bucket.
template <typename R>
static hmc_status autotune(hmc_ctx* c, BatchWs& w, cudaStream_t s, V2<R>* x, V2<R>* r, V2<R>* p,
                           V2<R>* q, V2<R>* u, const V2<R>* b, int* threads, int* ipt) {
  const int bucket = (int)std::log2((double)std::max<long long>(w.Ntot, 2));
  TuneKey key{(int)sizeof(R), bucket};
  auto it = g_tuned.find(key);
  if (it != g_tuned.end()) {
    *threads = it->second.first;
    *ipt = it->second.second;
    return HMC_OK;
  }
  const int cand[][2] = {{128, 1}, {128, 2}, {256, 1}, {256, 2}, {256, 4}, {512, 1}, {512, 2}};
  cudaEvent_t e0, e1;
  HMC_CUDA(c, cudaEventCreate(&e0));
  HMC_CUDA(c, cudaEventCreate(&e1));
  float best = 1e30f;
  int bt = 256, bi = 2;
  for (auto& cd : cand) {
    plan_blocks(w, cd[0], cd[1]);
    HMC_TRY(upload_plan<R>(c, w, s));
    HMC_CUDA(c, cudaMemsetAsync(w.tickets, 0, sizeof(unsigned) * w.nsys, s));
    kb_init<R><<<w.blocks, w.threads, 0, s>>>(w.sys, w.bsys, w.st, w.tol2, b, x, r, p, 1 << 30,
                                               w.partials, w.tickets);
    cg_iteration<R>(w, s, x, r, p, q, u, 0);
    HMC_CUDA(c, cudaEventRecord(e0, s));
    for (int i = 1; i < 4; ++i) cg_iteration<R>(w, s, x, r, p, q, u, i);
    HMC_CUDA(c, cudaEventRecord(e1, s));
    HMC_CUDA(c, cudaEventSynchronize(e1));
    HMC_CUDA(c, cudaGetLastError());
    float ms = 0.f;
    cudaEventElapsedTime(&ms, e0, e1);
    if (ms < best) {
      best = ms;
      bt = cd[0];
      bi = cd[1];
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  g_tuned[key] = {bt, bi};
  *threads = bt;
  *ipt = bi;
  return HMC_OK;
}

template <typename R>
static hmc_status batched_cg_loop(hmc_ctx* c, BatchWs& w, cudaStream_t s, V2<R>* x, V2<R>* r, V2<R>* p, V2<R>* q,
                                  V2<R>* u, int maxit, int pre_done, int chunk, int kid, double bytes_iter,
                                  long long* iters_launched);

// Resident blocks of the persistent batched kernel at `threads` per block.
template <typename R>
static int persist_capacity(hmc_ctx* c, int threads) {
  int occ = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kb_cg_persist<R>, threads, 0) != cudaSuccess) {
    cudaGetLastError();
    return 0;
  }
  return occ * c->nsm;
}

// The FP32 CG of all active systems as one persistent cooperative launch (the
// states left by kb_init; see kb_cg_persist). *ran is false when the launch
// does not fit (no resident block), and the caller takes the graph loop.
template <typename R>
static hmc_status batched_cg_persist(hmc_ctx* c, BatchWs& w, cudaStream_t s, V2<R>* x, V2<R>* r, V2<R>* p,
                                     V2<R>* q, V2<R>* u, int maxit, int pre_done, bool* ran) {
  *ran = false;
  const int cap = persist_capacity<R>(c, w.threads);
  if (cap < 1) return HMC_OK;
  int grid = std::min(w.blocks, cap);
  HMC_CUDA(c, cudaMemsetAsync(c->gbar, 0, sizeof(GridBar), s));
  const BSys* sys = w.sys;
  const int* bsys = w.bsys;
  int nvb = w.blocks;
  BState* bst = w.st;
  const double2* E = w.E;
  const float* p32 = w.phi32;
  double* partials = w.partials;
  unsigned* tickets = w.tickets;
  unsigned* ndone = w.ndone;
  unsigned target = (unsigned)(w.nsys - pre_done);
  int max_iters = maxit + 1;
  GridBar* gb = c->gbar;
  long long limit = c->bar_limit > 0 ? c->bar_limit : 2000000000LL;  // about one second of SM clock
  unsigned expect = (unsigned)grid + (unsigned)c->bar_extra;
  void* args[] = {&sys, &bsys, &nvb, &bst, &E, &p32, &x, &r, &p, &q, &u, &partials, &tickets, &ndone,
                  &target, &max_iters, &gb, &limit, &expect};
  const int kid = sizeof(R) == 8 ? K_BATCH_CG64 : K_BATCH_CG32;
  cudaEvent_t a = nullptr;
  prof_begin(c, kid, &a);
  const cudaError_t e = cudaLaunchCooperativeKernel((const void*)kb_cg_persist<R>, dim3(grid), dim3(w.threads),
                                                    args, 0, s);
  prof_end(c, kid, a);
  if (e != cudaSuccess) return cuda_fail(c, e, "persistent batched CG launch");
  GridBar gh{};
  HMC_CUDA(c, cudaMemcpyAsync(w.st_host, w.st, sizeof(BState) * w.nsys, cudaMemcpyDeviceToHost, s));
  HMC_CUDA(c, cudaMemcpyAsync(&gh, c->gbar, sizeof(GridBar), cudaMemcpyDeviceToHost, s));
  HMC_CUDA(c, cudaStreamSynchronize(s));
  if (gh.err) return fail(c, HMC_ERR_TIMEOUT, "persistent batched CG: a grid barrier wait gave up");
  double bytes = 0.0;
  for (int i = 0; i < w.nsys; ++i) bytes += (double)w.st_host[i].cg.iter * w.hsys[i].g.N * (sizeof(R) == 8 ? 192.0 : 88.0);
  c->prof.bytes[kid] += bytes;
  *ran = true;
  return HMC_OK;
}

// Run CG on all active systems in precision R until every system is done,
// replaying a captured graph of `chunk` iterations, or (FP32, when chosen) as
// one persistent launch.
template <typename R>
static hmc_status batched_cg(hmc_ctx* c, BatchWs& w, cudaStream_t s, const V2<R>* b, V2<R>* x, V2<R>* r,
                             V2<R>* p, V2<R>* q, V2<R>* u, int maxit, int nactive, long long* iters_launched) {
  HMC_CUDA(c, cudaMemsetAsync(w.tickets, 0, sizeof(unsigned) * w.nsys, s));
  HMC_CUDA(c, cudaMemsetAsync(w.ndone, 0, sizeof(unsigned), s));
  kb_init<R><<<w.blocks, w.threads, 0, s>>>(w.sys, w.bsys, w.st, w.tol2, b, x, r, p, maxit, w.partials,
                                             w.tickets);
  HMC_CUDA(c, cudaGetLastError());
  // systems already done at init (inactive, or converged at start) never pass
  // through kb_cg_m: count them from the states
  HMC_CUDA(c, cudaMemcpyAsync(w.st_host, w.st, sizeof(BState) * w.nsys, cudaMemcpyDeviceToHost, s));
  HMC_CUDA(c, cudaStreamSynchronize(s));
  int pre_done = 0;
  for (int i = 0; i < w.nsys; ++i) pre_done += w.st_host[i].cg.done != CG_RUNNING;
  if (pre_done == w.nsys) return HMC_OK;
  const int chunk = 8;
  const int kid = sizeof(R) == 8 ? K_BATCH_CG64 : K_BATCH_CG32;
  const double bytes_iter = sizeof(R) == 8 ? 192.0 : 88.0;
  // FP32: the persistent launch when pinned, or by timing -- the first solve of
  // the context takes the graph loop, the second the persistent launch, and
  // the one with the shorter time per iteration is kept
  if constexpr (sizeof(R) == 4) {
    int v = c->batch_variant ? c->batch_variant : c->batch_choice;
    const bool probe = (c->batch_variant == 0 && c->batch_choice == 0);
    if (probe) v = (c->batch_us[0] > 0.f) ? 2 : 1;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if (probe) {
      HMC_CUDA(c, cudaEventCreate(&e0));
      HMC_CUDA(c, cudaEventCreate(&e1));
      HMC_CUDA(c, cudaEventRecord(e0, s));
    }
    bool done = false;
    if (v == 2) {
      HMC_TRY(batched_cg_persist<R>(c, w, s, x, r, p, q, u, maxit, pre_done, &done));
      if (!done) v = 1;
    }
    if (!done) {
      HMC_TRY(batched_cg_loop<R>(c, w, s, x, r, p, q, u, maxit, pre_done, chunk, kid, bytes_iter,
                                 iters_launched));
    }
    if (probe) {
      HMC_CUDA(c, cudaEventRecord(e1, s));
      HMC_CUDA(c, cudaEventSynchronize(e1));
      float ms = 0.f;
      cudaEventElapsedTime(&ms, e0, e1);
      cudaEventDestroy(e0);
      cudaEventDestroy(e1);
      HMC_CUDA(c, cudaMemcpyAsync(w.st_host, w.st, sizeof(BState) * w.nsys, cudaMemcpyDeviceToHost, s));
      HMC_CUDA(c, cudaStreamSynchronize(s));
      int iters = 1;
      for (int i = 0; i < w.nsys; ++i) iters = std::max(iters, w.st_host[i].cg.iter);
      c->batch_us[v == 2 ? 1 : 0] = 1e3f * ms / iters;
      if (c->batch_us[0] > 0.f && c->batch_us[1] > 0.f) c->batch_choice = c->batch_us[1] < c->batch_us[0] ? 2 : 1;
      if (v == 1 && c->batch_us[0] > 0.f && persist_capacity<R>(c, w.threads) < 1) c->batch_choice = 1;
    }
    (void)nactive;
    return HMC_OK;
  }
  return batched_cg_loop<R>(c, w, s, x, r, p, q, u, maxit, pre_done, chunk, kid, bytes_iter, iters_launched);
}

// The graph-loop form of batched_cg after kb_init.
template <typename R>
static hmc_status batched_cg_loop(hmc_ctx* c, BatchWs& w, cudaStream_t s, V2<R>* x, V2<R>* r, V2<R>* p, V2<R>* q,
                                  V2<R>* u, int maxit, int pre_done, int chunk, int kid, double bytes_iter,
                                  long long* iters_launched) {
  // One graph launch for the whole batched solve: a device-side while loop
  // repeats the captured chunk until every running system is done (counted
  // in ndone) or the trip bound maxit / chunk + 2 is reached.
  if (c->use_loop_graphs && !c->prof.timing) {
    const unsigned target = (unsigned)(w.nsys - pre_done);
    cudaGraphExec_t lexec = nullptr;
    const hmc_status cs = capture_loop_graph(c, [&](cudaGraphConditionalHandle h) -> hmc_status {
      for (int i = 0; i < chunk; ++i) cg_iteration<R>(w, c->stream, x, r, p, q, u, i);
      kb_loop_continue<<<1, 32, 0, c->stream>>>(h, w.ndone, target, c->loop_trips);
      const cudaError_t e2 = cudaGetLastError();
      return e2 == cudaSuccess ? HMC_OK : cuda_fail(c, e2, "batched loop condition");
    }, &lexec);
    if (cs == HMC_OK) {
      c->loop_trips_host[0] = 0u;
      c->loop_trips_host[1] = (unsigned)(maxit / chunk + 2);
      cudaError_t e = cudaMemcpyAsync(c->loop_trips, c->loop_trips_host, 2 * sizeof(unsigned),
                                      cudaMemcpyHostToDevice, s);
      if (e == cudaSuccess) e = cudaGraphLaunch(lexec, s);
      if (e == cudaSuccess) e = cudaMemcpyAsync(w.st_host, w.st, sizeof(BState) * w.nsys, cudaMemcpyDeviceToHost, s);
      if (e == cudaSuccess)
        e = cudaMemcpyAsync(c->loop_trips_host, c->loop_trips, sizeof(unsigned), cudaMemcpyDeviceToHost, s);
      if (e == cudaSuccess) e = cudaStreamSynchronize(s);
      cudaGraphExecDestroy(lexec);
      if (e != cudaSuccess) return cuda_fail(c, e, "batched loop graph");
      const long long launched = (long long)c->loop_trips_host[0] * chunk;
      double bytes = 0.0;
      for (int i = 0; i < w.nsys; ++i) bytes += (double)w.st_host[i].cg.iter * w.hsys[i].g.N * bytes_iter;
      c->prof.bytes[kid] += bytes;
      c->prof.launches[kid] += 2 * launched;
      *iters_launched += launched;
      return HMC_OK;
    }
    c->err.clear();  // fall back to the chunked loop below
  }
  cudaGraph_t graph;
  cudaGraphExec_t exec;
  HMC_CUDA(c, cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal));
  for (int i = 0; i < chunk; ++i) cg_iteration<R>(w, s, x, r, p, q, u, i);  // even chunk: p holds the newest
  HMC_CUDA(c, cudaStreamEndCapture(s, &graph));
  cudaError_t e = cudaGraphInstantiate(&exec, graph, 0);
  if (e != cudaSuccess) {
    cudaGraphDestroy(graph);
    return cuda_fail(c, e, "cudaGraphInstantiate");
  }
  hmc_status status = HMC_OK;
  long long launched = 0;
  std::vector<char> running(w.nsys);
  for (int i = 0; i < w.nsys; ++i) running[i] = w.st_host[i].cg.done == CG_RUNNING;
  // the host reads the states after 1, 1, 2, 4, 4, ... chunks
  int per_check = 1, checks = 0;
  for (;;) {
    double act = 0.0;
    for (int i = 0; i < w.nsys; ++i) act += running[i] ? (double)w.hsys[i].g.N : 0.0;
    for (int k = 0; k < per_check && e == cudaSuccess; ++k) {
      c->prof.bytes[kid] += act * bytes_iter * chunk;
      cudaEvent_t a = nullptr;
      prof_begin(c, kid, &a);
      e = cudaGraphLaunch(exec, s);
      prof_end(c, kid, a);
      c->prof.launches[kid] += 2 * chunk - 1;
      launched += chunk;
    }
    if (e != cudaSuccess) {
      status = cuda_fail(c, e, "cudaGraphLaunch");
      break;
    }
    if (++checks >= 2 && per_check < 4) per_check *= 2;
    e = cudaMemcpyAsync(w.st_host, w.st, sizeof(BState) * w.nsys, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) {
      status = cuda_fail(c, e, "batched CG check");
      break;
    }
    int ndone = 0;
    for (int i = 0; i < w.nsys; ++i) {
      running[i] = w.st_host[i].cg.done == CG_RUNNING;
      ndone += !running[i];
    }
    if (ndone >= w.nsys) break;
    if (launched > (long long)maxit + chunk) break;  // every system stops at maxit on the device
  }
  cudaGraphExecDestroy(exec);
  cudaGraphDestroy(graph);
  *iters_launched += launched;
  return status;
}

}  // namespace hmc

using namespace hmc;

extern "C" hmc_status hmc_solve_batched(hmc_ctx* c, int nsys, const hmc_system* sys, int mixed,
                                        hmc_solve_info* infos) {
  if (!c) return HMC_ERR_INVALID;
  HMC_TRACE("hmc_solve_batched");
  if (nsys < 1 || !sys) return fail(c, HMC_ERR_INVALID, "nsys must be >= 1 and sys non-NULL");
  if (mixed != 0 && mixed != 1) return fail(c, HMC_ERR_INVALID, "mixed must be 0 or 1");
  BatchWs w;
  w.nsys = nsys;
  w.hsys.resize(nsys);
  long long off = 0;
  int maxit = 1;
  for (int s = 0; s < nsys; ++s) {
    const hmc_system& y = sys[s];
    const hmc_lattice& L = y.lat;
    if (bad_lattice(&L)) return fail(c, HMC_ERR_INVALID, "bad lattice in batched system");
    const long long N = lattice_sites(&L);
    if (!y.phi || !y.b || !y.x || ((uintptr_t)y.b) % 16 || ((uintptr_t)y.x) % 16 || ((uintptr_t)y.phi) % 8)
      return fail(c, HMC_ERR_INVALID, "batched system has a NULL or misaligned pointer");
    if (!(y.sigma >= 0.0) || !(y.tol > 0.0) || y.maxit < 1 || !std::isfinite(y.ms))
      return fail(c, HMC_ERR_INVALID, "batched system has bad sigma, tol, maxit or mass");
    const double delta = L.beta / L.nt;
    if (1.0 - delta * y.ms == 0.0) return fail(c, HMC_ERR_INVALID, "1 - delta*m_s == 0 in batched system");
    BSys& S = w.hsys[s];
    S.g = make_geo(L.n, L.m, L.nt, delta, L.kappa);
    S.off = off;
    S.dm = delta * y.ms;
    S.sigma = y.sigma;
    S.dm32 = (float)S.dm;
    S.sigma32 = (float)S.sigma;
    S.phi = y.phi;
    S.maxit = y.maxit;
    off += N;
    maxit = std::max(maxit, y.maxit);
  }
  w.Ntot = off;
  if (infos) std::memset(infos, 0, sizeof(hmc_solve_info) * nsys);

  // the work runs on a private non-default stream (graph capture needs one),
  // ordered after and before the context's stream by events
  cudaStream_t s;
  HMC_CUDA(c, cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking));
  cudaEvent_t ev_in, ev_out;
  HMC_CUDA(c, cudaEventCreateWithFlags(&ev_in, cudaEventDisableTiming));
  HMC_CUDA(c, cudaEventCreateWithFlags(&ev_out, cudaEventDisableTiming));
  HMC_CUDA(c, cudaEventRecord(ev_in, c->stream));
  HMC_CUDA(c, cudaStreamWaitEvent(s, ev_in, 0));
  cudaStream_t saved = c->stream;
  c->stream = s;

  auto body = [&]() -> hmc_status {
    const size_t Nt = (size_t)w.Ntot;
    // block tables sized for the smallest block shape (most blocks)
    plan_blocks(w, 128, 1);
    const int max_blocks = w.blocks;
    w.hbsys.reserve(max_blocks);
    HMC_TRY(bmalloc(c, w, (void**)&w.sys, sizeof(BSys) * nsys));
    HMC_TRY(bmalloc(c, w, (void**)&w.bsys, sizeof(int) * max_blocks));
    HMC_TRY(bmalloc(c, w, (void**)&w.st, sizeof(BState) * nsys));
    HMC_TRY(bmalloc(c, w, (void**)&w.tol2, sizeof(double) * nsys));
    HMC_TRY(bmalloc(c, w, (void**)&w.rrbb, sizeof(double) * 2 * nsys));
    HMC_TRY(bmalloc(c, w, (void**)&w.tickets, sizeof(unsigned) * nsys));
    HMC_TRY(bmalloc(c, w, (void**)&w.ndone, sizeof(unsigned)));
    HMC_TRY(bmalloc(c, w, (void**)&w.partials, sizeof(double) * 2 * max_blocks));  // K <= 2 values
    HMC_TRY(bmalloc(c, w, (void**)&w.E, sizeof(double2) * Nt));
    HMC_TRY(bmalloc(c, w, (void**)&w.phi32, sizeof(float) * Nt));
    HMC_TRY(bmalloc(c, w, (void**)&w.x, sizeof(double2) * Nt));
    HMC_TRY(bmalloc(c, w, (void**)&w.b, sizeof(double2) * Nt));
    HMC_TRY(bmalloc(c, w, (void**)&w.r, sizeof(double2) * Nt));
    if (!mixed) {
      HMC_TRY(bmalloc(c, w, (void**)&w.p, sizeof(double2) * Nt));
      HMC_TRY(bmalloc(c, w, (void**)&w.q, sizeof(double2) * Nt));
      HMC_TRY(bmalloc(c, w, (void**)&w.u, sizeof(double2) * Nt));
    } else {
      HMC_TRY(bmalloc(c, w, (void**)&w.u, sizeof(double2) * Nt));
      HMC_TRY(bmalloc(c, w, (void**)&w.r32, sizeof(float2) * Nt));
      HMC_TRY(bmalloc(c, w, (void**)&w.e32, sizeof(float2) * Nt));
      HMC_TRY(bmalloc(c, w, (void**)&w.p32v, sizeof(float2) * Nt));
      HMC_TRY(bmalloc(c, w, (void**)&w.q32v, sizeof(float2) * Nt));
      HMC_TRY(bmalloc(c, w, (void**)&w.u32, sizeof(float2) * Nt));
      HMC_TRY(bmalloc(c, w, (void**)&w.rr32, sizeof(float2) * Nt));
    }
    HMC_TRY(bmalloc_host(c, 0, (void**)&w.st_host, sizeof(BState) * nsys));
    HMC_TRY(bmalloc_host(c, 1, (void**)&w.rrbb_host, sizeof(double) * 2 * nsys));
    HMC_TRY(bmalloc_host(c, 2, (void**)&w.ndone_host, sizeof(unsigned)));
    HMC_CUDA(c, cudaMemsetAsync(w.tickets, 0, sizeof(unsigned) * nsys, s));
    // gather b, phases
    for (int i = 0; i < nsys; ++i)
      HMC_CUDA(c, cudaMemcpyAsync(w.b + w.hsys[i].off, sys[i].b, sizeof(double2) * w.hsys[i].g.N,
                                  cudaMemcpyDeviceToDevice, s));
    plan_blocks(w, 256, 2);
    HMC_TRY(upload_plan<double>(c, w, s));
    kb_phase<<<w.blocks, w.threads, 0, s>>>(w.sys, w.bsys, w.E, w.phi32);
    HMC_CUDA(c, cudaGetLastError());
    c->prof.launches[K_BATCH_MISC]++;

    std::vector<double> tol2(nsys);
    std::vector<BState> init(nsys);
    for (int i = 0; i < nsys; ++i) {
      std::memset(&init[i], 0, sizeof(BState));
      init[i].active = 1;
    }
    HMC_CUDA(c, cudaMemcpyAsync(w.st, init.data(), sizeof(BState) * nsys, cudaMemcpyHostToDevice, s));
    std::vector<int> iters(nsys, 0), outer(nsys, 0), inner(nsys, 0), status(nsys, HMC_OK);
    std::vector<double> rel(nsys, 0.0);
    long long launched = 0;
    int threads = 256, ipt = 2;

    if (!mixed) {
      for (int i = 0; i < nsys; ++i) tol2[i] = sys[i].tol * sys[i].tol;
      HMC_CUDA(c, cudaMemcpyAsync(w.tol2, tol2.data(), sizeof(double) * nsys, cudaMemcpyHostToDevice, s));
      HMC_TRY(autotune<double>(c, w, s, w.x, w.r, w.p, w.q, w.u, w.b, &threads, &ipt));
      plan_blocks(w, threads, ipt);
      HMC_TRY(upload_plan<double>(c, w, s));
      HMC_CUDA(c, cudaMemcpyAsync(w.st, init.data(), sizeof(BState) * nsys, cudaMemcpyHostToDevice, s));
      HMC_TRY(batched_cg<double>(c, w, s, w.b, w.x, w.r, w.p, w.q, w.u, maxit, nsys, &launched));
      HMC_CUDA(c, cudaMemcpyAsync(w.st_host, w.st, sizeof(BState) * nsys, cudaMemcpyDeviceToHost, s));
      HMC_CUDA(c, cudaStreamSynchronize(s));
      for (int i = 0; i < nsys; ++i) {
        iters[i] = w.st_host[i].cg.iter;
        if (w.st_host[i].cg.done == CG_MAXIT || w.st_host[i].cg.iter > sys[i].maxit) status[i] = HMC_ERR_NOT_CONVERGED;
        if (w.st_host[i].cg.done == CG_BREAKDOWN) status[i] = HMC_ERR_NAN;
      }
    } else {
      // defect correction: x = 0, r = b; loop: solve A e = r in FP32, x += e,
      // r = b - A x in FP64
      HMC_CUDA(c, cudaMemsetAsync(w.x, 0, sizeof(double2) * Nt, s));
      std::vector<double> bnorm(nsys, 0.0), rnorm(nsys, 0.0);
      std::vector<int> done(nsys, 0);
      bool tuned = false;
      const int max_outer = 50;
      for (int it = 0; it <= max_outer; ++it) {
        // r = b - A x (FP64), r32 = r
        kb_mdag64<<<w.blocks, w.threads, 0, s>>>(w.sys, w.bsys, w.E, w.x, w.u);
        kb_resid64<<<w.blocks, w.threads, 0, s>>>(w.sys, w.bsys, w.E, w.u, w.x, w.b, w.r, w.r32, w.rrbb,
                                                  w.partials, w.tickets);
        HMC_CUDA(c, cudaGetLastError());
        c->prof.launches[K_BATCH_RESID] += 2;
        HMC_CUDA(c, cudaMemcpyAsync(w.rrbb_host, w.rrbb, sizeof(double) * 2 * nsys, cudaMemcpyDeviceToHost, s));
        HMC_CUDA(c, cudaStreamSynchronize(s));
        int nact = 0;
        for (int i = 0; i < nsys; ++i) {
          bnorm[i] = std::sqrt(w.rrbb_host[2 * i + 1]);
          rnorm[i] = std::sqrt(w.rrbb_host[2 * i]);
          rel[i] = bnorm[i] > 0 ? rnorm[i] / bnorm[i] : 0.0;
          if (!std::isfinite(rnorm[i])) {
            status[i] = HMC_ERR_NAN;
            done[i] = 1;
          }
          if (!done[i] && rnorm[i] <= sys[i].tol * bnorm[i]) done[i] = 1;
          if (!done[i] && outer[i] >= max_outer) {
            status[i] = HMC_ERR_NOT_CONVERGED;
            done[i] = 1;
          }
          init[i].active = done[i] ? 0 : 1;
          // inner tolerance: what is left to gain, with margin, floored at FP32 reach
          const double need = bnorm[i] > 0 ? sys[i].tol * bnorm[i] / std::max(rnorm[i], 1e-300) : 1.0;
          const double t = std::max(0.5 * need, 1e-6);
          tol2[i] = t * t;
          nact += init[i].active;
        }
        if (nact == 0) break;
        HMC_CUDA(c, cudaMemcpyAsync(w.tol2, tol2.data(), sizeof(double) * nsys, cudaMemcpyHostToDevice, s));
        HMC_CUDA(c, cudaMemcpyAsync(w.st, init.data(), sizeof(BState) * nsys, cudaMemcpyHostToDevice, s));
        if (!tuned) {
          // r32 now holds the first right-hand sides: tune the FP32 block shape on them
          HMC_TRY(autotune<float>(c, w, s, w.e32, w.rr32, w.p32v, w.q32v, w.u32, w.r32, &threads, &ipt));
          plan_blocks(w, threads, ipt);
          HMC_TRY(upload_plan<float>(c, w, s));
          HMC_CUDA(c, cudaMemcpyAsync(w.st, init.data(), sizeof(BState) * nsys, cudaMemcpyHostToDevice, s));
          tuned = true;
        }
        HMC_TRY(batched_cg<float>(c, w, s, w.r32, w.e32, w.rr32, w.p32v, w.q32v, w.u32, 2000, nact, &launched));
        HMC_CUDA(c, cudaMemcpyAsync(w.st_host, w.st, sizeof(BState) * nsys, cudaMemcpyDeviceToHost, s));
        HMC_CUDA(c, cudaStreamSynchronize(s));
        for (int i = 0; i < nsys; ++i) {
          if (!init[i].active) continue;
          inner[i] += w.st_host[i].cg.iter;
          outer[i] += 1;
        }
        kb_xadd<<<w.blocks, w.threads, 0, s>>>(w.sys, w.bsys, w.st, w.e32, w.x);
        HMC_CUDA(c, cudaGetLastError());
        c->prof.launches[K_BATCH_MISC]++;
      }
      for (int i = 0; i < nsys; ++i) iters[i] = outer[i];
    }
    // true residuals in FP64 (also the report for the FP64 path), scatter x
    kb_mdag64<<<w.blocks, w.threads, 0, s>>>(w.sys, w.bsys, w.E, w.x, w.u);
    kb_resid64<<<w.blocks, w.threads, 0, s>>>(w.sys, w.bsys, w.E, w.u, w.x, w.b, w.r, nullptr, w.rrbb,
                                              w.partials, w.tickets);
    HMC_CUDA(c, cudaGetLastError());
    c->prof.launches[K_BATCH_RESID] += 2;
    HMC_CUDA(c, cudaMemcpyAsync(w.rrbb_host, w.rrbb, sizeof(double) * 2 * nsys, cudaMemcpyDeviceToHost, s));
    for (int i = 0; i < nsys; ++i)
      HMC_CUDA(c, cudaMemcpyAsync(sys[i].x, w.x + w.hsys[i].off, sizeof(double2) * w.hsys[i].g.N,
                                  cudaMemcpyDeviceToDevice, s));
    HMC_CUDA(c, cudaStreamSynchronize(s));
    hmc_status worst = HMC_OK;
    for (int i = 0; i < nsys; ++i) {
      const double bb = w.rrbb_host[2 * i + 1];
      rel[i] = bb > 0 ? std::sqrt(w.rrbb_host[2 * i] / bb) : 0.0;
      if (status[i] == HMC_OK && !(rel[i] <= sys[i].tol * (mixed ? 1.0 : 1.0 + 1e-6)) && mixed)
        status[i] = HMC_ERR_NOT_CONVERGED;
      if (status[i] != HMC_OK && worst == HMC_OK) worst = (hmc_status)status[i];
      if (infos) {
        infos[i].iters = mixed ? inner[i] : iters[i];
        infos[i].iters_outer = mixed ? outer[i] : 0;
        infos[i].iters_inner = mixed ? inner[i] : 0;
        infos[i].status = status[i];
        infos[i].true_rel_res = rel[i];
        infos[i].applies64 = mixed ? outer[i] + 1 : iters[i];
        infos[i].applies32 = mixed ? inner[i] : 0;
        const double N = (double)w.hsys[i].g.N;
        infos[i].bytes = (long long)(N * (192.0 * infos[i].applies64 + 96.0 * infos[i].applies32));
      }
    }
    if (worst != HMC_OK) return fail(c, worst, "a batched system did not converge");
    return HMC_OK;
  };
  hmc_status st = body();
  cudaStreamSynchronize(s);
  c->stream = saved;
  cudaEventRecord(ev_out, s);
  cudaStreamWaitEvent(saved, ev_out, 0);
  cudaEventDestroy(ev_in);
  cudaEventDestroy(ev_out);
  bfree(w);
  cudaStreamDestroy(s);
  return st;
}
