// The three alternative designs of the FP32 CG iteration (the grid-stride
// pair in kernels.cu is the fourth): shared-memory tiled kernels, marching
// kernels, and the persistent cooperative kernel. The autotuner times them
// against the pair (solvers.cu); hmc_set_cg_variant pins one. All of them run
// the single-precision CG of Section 3 on the operator of Eq. ferm_op.
#include "kernels.h"
#include "launch.cuh"
#include "operator.cuh"

namespace hmc {

// ---------------------------------------------------------------------------
// Tiled variants of the FP32 CG pair. A block owns TC consecutive cells
// [c0, c0 + TC) of the time slices [t0, t0 + TT) and marches through its slices.
// For every slice it stages, in shared memory, the window of cells
// (c0 - n - 1 + k) mod V, k < W = TC + 2(n + 1), on both sublattices: that window
// holds every spatial neighbour of the tile, the wrapped ones included, as long
// as W <= V (smaller lattices use the grid-stride kernels). Every input element
// is then read about W / TC times instead of once per neighbour visit, and the
// time neighbour behind the march comes from a register.
template <int TC>
struct TileWin {
  static constexpr int kMaxN = 256;  // widest lattice the window is sized for
  float2 a[TC + 2 * (kMaxN + 1)];
  float2 b[TC + 2 * (kMaxN + 1)];
};

__device__ __forceinline__ int win_index(int nc, int c0, int n, int V) {
  int k = nc - (c0 - n - 1);
  if (k < 0) k += V;
  if (k >= V) k -= V;
  return k;
}

// kernel A, tiled: p_new = r + beta p_old staged per slice; u = M^dagger p_new
template <int TC>
__global__ void __launch_bounds__(TC) k_cg32_pmdag_tiled(Geo g, Phase<float> ph, int TT,
                                                        const float2* __restrict__ r,
                                                        const float2* __restrict__ pold,
                                                        float2* __restrict__ pnew,
                                                        float2* __restrict__ u, CGScal* sc,
                                                        const float2* __restrict__ partB, int GB,
                                                        float2* __restrict__ partA) {
  __shared__ TileWin<TC> win;
  __shared__ float s_beta;
  __shared__ int s_exit, s_done;
  pdl_wait();
  if (threadIdx.x == 0) s_exit = sc->done;
  __syncthreads();
  if (s_exit) return;
  const int first = sc->first;
  const float2 rr_pair = first ? make_float2(0.f, 0.f) : ff_sum_partials(partB, GB);
  if (threadIdx.x == 0) {
    float b;
    s_done = cg32_scalars_first(sc, first, rr_pair, blockIdx.x == 0 && blockIdx.y == 0, &b);
    s_beta = b;
  }
  __syncthreads();
  if (s_done) return;
  const float dm = sc->dm32, sigma = sc->sigma32, beta = s_beta, dk = g.dkf;
  const int n = g.n, V = g.V, H = g.H, nt = g.nt;
  const int c0 = blockIdx.x * TC;
  const int c = c0 + threadIdx.x;
  const bool own = c < V;
  const int W = TC + 2 * (n + 1);
  const int t0 = blockIdx.y * TT;
  const int t1 = min(t0 + TT, nt);
  // cell coordinates and the window slots of the four spatial partners
  int kim1 = 0, kjm1 = 0, kip1 = 0, kjp1 = 0, kself = 0;
  if (own) {
    const int j = (int)fdiv((uint32_t)c, g.fn);
    const int i = c - j * n;
    kself = c - c0 + n + 1;
    kim1 = win_index(c - 1 + (i == 0 ? n : 0), c0, n, V);
    kjm1 = win_index(c - n + (j == 0 ? V : 0), c0, n, V);
    kip1 = win_index(c + 1 - (i == n - 1 ? n : 0), c0, n, V);
    kjp1 = win_index(c + n - (j == g.m - 1 ? V : 0), c0, n, V);
  }
  auto P = [&](int k) {
    float2 a = r[k], b = pold[k];
    return Cx<float>{fmaf(beta, b.x, a.x), fmaf(beta, b.y, a.y)};
  };
  // B at t0 - 1 (the time partner of the B row at t0), carried afterwards
  Cx<float> pb_prev{0.f, 0.f};
  if (own) pb_prev = P(H + (t0 == 0 ? (nt - 1) * V : (t0 - 1) * V) + c);
  float loc = 0.f;
  for (int t = t0; t < t1; ++t) {
    const int base = t * V;
    for (int k = threadIdx.x; k < W; k += TC) {
      int cell = c0 - n - 1 + k;
      if (cell < 0) cell += V;
      if (cell >= V) cell -= V;
      Cx<float> va = P(base + cell), vb = P(H + base + cell);
      win.a[k] = make_float2(va.re, va.im);
      win.b[k] = make_float2(vb.re, vb.im);
    }
    __syncthreads();
    if (own) {
      const int q = base + c;
      const bool wrap_tp = (t == nt - 1), wrap_tm = (t == 0);
      const int qtp = wrap_tp ? c : base + V + c;
      const int qtm = wrap_tm ? (nt - 1) * V + c : base - V + c;
      float2 s;
      s = win.a[kself];
      Cx<float> pa{s.x, s.y};
      s = win.b[kself];
      Cx<float> pb{s.x, s.y};
      st(pnew, q, pa);
      st(pnew, H + q, pb);
      // A row: partner (x, t+1)
      Cx<float> ea = ph(qtp);
      Cx<float> za = cneg_if(Cx<float>{ea.re - dm, -ea.im}, wrap_tp);
      Cx<float> ta = cfma(za, P(qtp), Cx<float>{-pa.re, -pa.im});
      s = win.b[kim1];
      Cx<float> b1{s.x, s.y};
      s = win.b[kjm1];
      Cx<float> b2{s.x, s.y};
      Cx<float> oa = hopsum(ta, dk, pb, b1, b2);
      // B row: partner (x, t-1), carried from the previous slice
      Cx<float> eb = ph(H + qtm);
      Cx<float> zb = cneg_if(Cx<float>{dm - eb.re, -eb.im}, wrap_tm);
      Cx<float> tb = cfma(zb, pb_prev, pb);
      s = win.a[kip1];
      Cx<float> a1{s.x, s.y};
      s = win.a[kjp1];
      Cx<float> a2{s.x, s.y};
      Cx<float> ob = hopsum(tb, dk, pa, a1, a2);
      st(u, q, oa);
      st(u, H + q, ob);
      loc += norm2(oa) + norm2(ob);
      if (sigma != 0.f) loc += sigma * (norm2(pa) + norm2(pb));
      pb_prev = pb;
    }
    __syncthreads();
  }
  pdl_trigger();
  float2 v = ff_block_sum(make_float2(loc, 0.f));
  if (threadIdx.x == 0) partA[blockIdx.y * gridDim.x + blockIdx.x] = v;
}

// kernel B, tiled: u staged per slice; A p = M u + sigma p; x, r updates
template <int TC>
__global__ void __launch_bounds__(TC) k_cg32_m_tiled(Geo g, Phase<float> ph, int TT,
                                                    const float2* __restrict__ u,
                                                    const float2* __restrict__ p,
                                                    float2* __restrict__ x, float2* __restrict__ r,
                                                    CGScal* sc, const float2* __restrict__ partA, int GA,
                                                    float2* __restrict__ partB) {
  __shared__ TileWin<TC> win;
  __shared__ float s_alpha;
  __shared__ int s_exit, s_bad;
  pdl_wait();
  if (threadIdx.x == 0) s_exit = sc->done;
  __syncthreads();
  if (s_exit) return;
  const float2 pAp_pair = ff_sum_partials(partA, GA);
  if (threadIdx.x == 0) {
    float a;
    s_bad = cg32_scalars_second(sc, pAp_pair, blockIdx.x == 0 && blockIdx.y == 0, &a);
    s_alpha = a;
  }
  __syncthreads();
  if (s_bad) return;
  const float dm = sc->dm32, sigma = sc->sigma32, alpha = s_alpha, dk = g.dkf;
  const int n = g.n, V = g.V, H = g.H, nt = g.nt;
  const int c0 = blockIdx.x * TC;
  const int c = c0 + threadIdx.x;
  const bool own = c < V;
  const int W = TC + 2 * (n + 1);
  const int t0 = blockIdx.y * TT;
  const int t1 = min(t0 + TT, nt);
  int kim1 = 0, kjm1 = 0, kip1 = 0, kjp1 = 0, kself = 0;
  if (own) {
    const int j = (int)fdiv((uint32_t)c, g.fn);
    const int i = c - j * n;
    kself = c - c0 + n + 1;
    kim1 = win_index(c - 1 + (i == 0 ? n : 0), c0, n, V);
    kjm1 = win_index(c - n + (j == 0 ? V : 0), c0, n, V);
    kip1 = win_index(c + 1 - (i == n - 1 ? n : 0), c0, n, V);
    kjp1 = win_index(c + n - (j == g.m - 1 ? V : 0), c0, n, V);
  }
  // A at t0 - 1 (the time partner of the A row at t0), carried afterwards
  Cx<float> ua_prev{0.f, 0.f};
  if (own) {
    float2 v = u[(t0 == 0 ? (nt - 1) * V : (t0 - 1) * V) + c];
    ua_prev = Cx<float>{v.x, v.y};
  }
  float loc = 0.f;
  for (int t = t0; t < t1; ++t) {
    const int base = t * V;
    for (int k = threadIdx.x; k < W; k += TC) {
      int cell = c0 - n - 1 + k;
      if (cell < 0) cell += V;
      if (cell >= V) cell -= V;
      win.a[k] = u[base + cell];
      win.b[k] = u[H + base + cell];
    }
    __syncthreads();
    if (own) {
      const int q = base + c;
      const bool wrap_tp = (t == nt - 1), wrap_tm = (t == 0);
      const int qtp = wrap_tp ? c : base + V + c;
      float2 s;
      s = win.a[kself];
      Cx<float> ua{s.x, s.y};
      s = win.b[kself];
      Cx<float> ub{s.x, s.y};
      // A row: (e^{i phi_A(t)} - dm) u_A(t-1)
      Cx<float> ea = ph(q);
      Cx<float> za = cneg_if(Cx<float>{ea.re - dm, ea.im}, wrap_tm);
      Cx<float> ta = cfma(za, ua_prev, Cx<float>{-ua.re, -ua.im});
      s = win.b[kim1];
      Cx<float> b1{s.x, s.y};
      s = win.b[kjm1];
      Cx<float> b2{s.x, s.y};
      Cx<float> oa = hopsum(ta, dk, ub, b1, b2);
      // B row: -(e^{-i phi_B(t)} - dm) u_B(t+1)
      Cx<float> eb = ph(H + q);
      Cx<float> zb = cneg_if(Cx<float>{dm - eb.re, eb.im}, wrap_tp);
      float2 nb = u[H + qtp];
      Cx<float> tb = cfma(zb, Cx<float>{nb.x, nb.y}, ub);
      s = win.a[kip1];
      Cx<float> a1{s.x, s.y};
      s = win.a[kjp1];
      Cx<float> a2{s.x, s.y};
      Cx<float> ob = hopsum(tb, dk, ua, a1, a2);
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        const int k = h ? H + q : q;
        Cx<float> Ap = h ? ob : oa;
        float2 pk = p[k], xk = x[k], rk = r[k];
        Ap.re = fmaf(sigma, pk.x, Ap.re);
        Ap.im = fmaf(sigma, pk.y, Ap.im);
        xk.x = fmaf(alpha, pk.x, xk.x);
        xk.y = fmaf(alpha, pk.y, xk.y);
        rk.x = fmaf(-alpha, Ap.re, rk.x);
        rk.y = fmaf(-alpha, Ap.im, rk.y);
        x[k] = xk;
        r[k] = rk;
        loc = fmaf(rk.x, rk.x, fmaf(rk.y, rk.y, loc));
      }
      ua_prev = ua;
    }
    __syncthreads();
  }
  pdl_trigger();
  float2 v = ff_block_sum(make_float2(loc, 0.f));
  if (threadIdx.x == 0) partB[blockIdx.y * gridDim.x + blockIdx.x] = v;
}

// ---------------------------------------------------------------------------
// Marching variants of the FP32 CG pair. A block owns blockDim.x consecutive
// cells [c0, c0 + blockDim.x) of the time slices [t0, t0 + TT); each thread
// keeps one cell and walks up in t. The time partners then come from
// registers (the value one slice ahead is loaded once and becomes the next
// slice's own value; the one behind is the previous slice's), and the spatial
// partners at the same slice, which neighbouring threads of the block load,
// come from L1. No shared memory and no barrier inside the march.
__global__ void __launch_bounds__(kMaxThreads) k_cg32_pmdag_march(Geo g, Phase<float> ph, int TT,
                                                               const float2* __restrict__ r,
                                                               const float2* __restrict__ pold,
                                                               float2* __restrict__ pnew,
                                                               float2* __restrict__ u, CGScal* sc,
                                                               const float2* __restrict__ partB, int GB,
                                                               float2* __restrict__ partA) {
  __shared__ float s_beta;
  __shared__ int s_exit, s_done;
  pdl_wait();
  if (threadIdx.x == 0) s_exit = sc->done;
  __syncthreads();
  if (s_exit) return;
  const int first = sc->first;
  const float2 rr_pair = first ? make_float2(0.f, 0.f) : ff_sum_partials(partB, GB);
  if (threadIdx.x == 0) {
    float b;
    s_done = cg32_scalars_first(sc, first, rr_pair, blockIdx.x == 0 && blockIdx.y == 0, &b);
    s_beta = b;
  }
  __syncthreads();
  if (s_done) return;
  const float dm = sc->dm32, sigma = sc->sigma32, beta = s_beta, dk = g.dkf;
  const int n = g.n, V = g.V, H = g.H, nt = g.nt;
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  const int t0 = blockIdx.y * TT;
  const int t1 = min(t0 + TT, nt);
  float loc = 0.f;
  if (c < V) {
    const int j = (int)fdiv((uint32_t)c, g.fn);
    const int i = c - j * n;
    const int cim1 = c - 1 + (i == 0 ? n : 0), cjm1 = c - n + (j == 0 ? V : 0);
    const int cip1 = c + 1 - (i == n - 1 ? n : 0), cjp1 = c + n - (j == g.m - 1 ? V : 0);
    auto P = [&](int k) {
      float2 a = r[k], b = pold[k];
      return Cx<float>{fmaf(beta, b.x, a.x), fmaf(beta, b.y, a.y)};
    };
    Cx<float> pb_prev = P(H + (t0 == 0 ? (nt - 1) * V : (t0 - 1) * V) + c);  // B at t0 - 1
    Cx<float> pa = P(t0 * V + c);                                             // A at t0
    for (int t = t0; t < t1; ++t) {
      const int base = t * V, q = base + c;
      const bool wrap_tp = (t == nt - 1), wrap_tm = (t == 0);
      const int qtp = wrap_tp ? c : q + V;
      const int qtm = wrap_tm ? (nt - 1) * V + c : q - V;
      const Cx<float> pb = P(H + q);
      const Cx<float> pa_next = P(qtp);
      // A row: partner (x, t+1)
      Cx<float> ea = ph(qtp);
      Cx<float> za = cneg_if(Cx<float>{ea.re - dm, -ea.im}, wrap_tp);
      Cx<float> ta = cfma(za, pa_next, Cx<float>{-pa.re, -pa.im});
      Cx<float> oa = hopsum(ta, dk, pb, P(H + base + cim1), P(H + base + cjm1));
      // B row: partner (x, t-1), carried
      Cx<float> eb = ph(H + qtm);
      Cx<float> zb = cneg_if(Cx<float>{dm - eb.re, -eb.im}, wrap_tm);
      Cx<float> tb = cfma(zb, pb_prev, pb);
      Cx<float> ob = hopsum(tb, dk, pa, P(base + cip1), P(base + cjp1));
      st(pnew, q, pa);
      st(pnew, H + q, pb);
      st(u, q, oa);
      st(u, H + q, ob);
      loc += norm2(oa) + norm2(ob);
      if (sigma != 0.f) loc += sigma * (norm2(pa) + norm2(pb));
      pb_prev = pb;
      pa = pa_next;
    }
  }
  pdl_trigger();
  float2 v = ff_block_sum(make_float2(loc, 0.f));
  if (threadIdx.x == 0) partA[blockIdx.y * gridDim.x + blockIdx.x] = v;
}

__global__ void __launch_bounds__(kMaxThreads) k_cg32_m_march(Geo g, Phase<float> ph, int TT,
                                                           const float2* __restrict__ u,
                                                           const float2* __restrict__ p,
                                                           float2* __restrict__ x, float2* __restrict__ r,
                                                           CGScal* sc, const float2* __restrict__ partA, int GA,
                                                           float2* __restrict__ partB) {
  __shared__ float s_alpha;
  __shared__ int s_exit, s_bad;
  pdl_wait();
  if (threadIdx.x == 0) s_exit = sc->done;
  __syncthreads();
  if (s_exit) return;
  const float2 pAp_pair = ff_sum_partials(partA, GA);
  if (threadIdx.x == 0) {
    float a;
    s_bad = cg32_scalars_second(sc, pAp_pair, blockIdx.x == 0 && blockIdx.y == 0, &a);
    s_alpha = a;
  }
  __syncthreads();
  if (s_bad) return;
  const float dm = sc->dm32, sigma = sc->sigma32, alpha = s_alpha, dk = g.dkf;
  const int n = g.n, V = g.V, H = g.H, nt = g.nt;
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  const int t0 = blockIdx.y * TT;
  const int t1 = min(t0 + TT, nt);
  float loc = 0.f;
  if (c < V) {
    const int j = (int)fdiv((uint32_t)c, g.fn);
    const int i = c - j * n;
    const int cim1 = c - 1 + (i == 0 ? n : 0), cjm1 = c - n + (j == 0 ? V : 0);
    const int cip1 = c + 1 - (i == n - 1 ? n : 0), cjp1 = c + n - (j == g.m - 1 ? V : 0);
    auto U = [&](int k) {
      float2 v = u[k];
      return Cx<float>{v.x, v.y};
    };
    Cx<float> ua_prev = U((t0 == 0 ? (nt - 1) * V : (t0 - 1) * V) + c);  // A at t0 - 1
    Cx<float> ub = U(H + t0 * V + c);                                    // B at t0
    for (int t = t0; t < t1; ++t) {
      const int base = t * V, q = base + c;
      const bool wrap_tp = (t == nt - 1), wrap_tm = (t == 0);
      const int qtp = wrap_tp ? c : q + V;
      const Cx<float> ua = U(q);
      const Cx<float> ub_next = U(H + qtp);
      // A row: (e^{i phi_A(t)} - dm) u_A(t-1), carried
      Cx<float> ea = ph(q);
      Cx<float> za = cneg_if(Cx<float>{ea.re - dm, ea.im}, wrap_tm);
      Cx<float> ta = cfma(za, ua_prev, Cx<float>{-ua.re, -ua.im});
      Cx<float> oa = hopsum(ta, dk, ub, U(H + base + cim1), U(H + base + cjm1));
      // B row: -(e^{-i phi_B(t)} - dm) u_B(t+1)
      Cx<float> eb = ph(H + q);
      Cx<float> zb = cneg_if(Cx<float>{dm - eb.re, eb.im}, wrap_tp);
      Cx<float> tb = cfma(zb, ub_next, ub);
      Cx<float> ob = hopsum(tb, dk, ua, U(base + cip1), U(base + cjp1));
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        const int k = h ? H + q : q;
        Cx<float> Ap = h ? ob : oa;
        float2 pk = p[k], xk = x[k], rk = r[k];
        Ap.re = fmaf(sigma, pk.x, Ap.re);
        Ap.im = fmaf(sigma, pk.y, Ap.im);
        xk.x = fmaf(alpha, pk.x, xk.x);
        xk.y = fmaf(alpha, pk.y, xk.y);
        rk.x = fmaf(-alpha, Ap.re, rk.x);
        rk.y = fmaf(-alpha, Ap.im, rk.y);
        x[k] = xk;
        r[k] = rk;
        loc = fmaf(rk.x, rk.x, fmaf(rk.y, rk.y, loc));
      }
      ua_prev = ua;
      ub = ub_next;
    }
  }
  pdl_trigger();
  float2 v = ff_block_sum(make_float2(loc, 0.f));
  if (threadIdx.x == 0) partB[blockIdx.y * gridDim.x + blockIdx.x] = v;
}

// ---------------------------------------------------------------------------
// Persistent FP32 CG: the whole solve in one cooperative launch. Every block
// is resident for the duration and owns the cell-times [q0, q0 + ipb); it
// keeps x, and its own entries of r and p, in shared memory across
// iterations, so x never travels to memory until the end and the updates of
// the second half-iteration read no vector but u. An iteration is the same CG
// step as the two-kernel pair (p = r + beta p, u = M^dagger p, pAp, alpha,
// A p = M u + sigma p, x and r updates, |r|^2), with the kernel boundaries
// replaced by grid barriers and the block partials summed by every block in
// the same fixed order. The barrier waits are bounded: a wait that gives up
// marks the solve CG_TIMEOUT and every block leaves.
constexpr int kPersistThreads = 256;

__global__ void __launch_bounds__(kPersistThreads, 4)
    k_cg32_persist(Geo g, Phase<float> ph, float2* __restrict__ x, float2* __restrict__ r,
                   float2* __restrict__ p0, float2* __restrict__ p1, float2* __restrict__ u, CGScal* sc,
                   float2* __restrict__ partA, float2* __restrict__ partB, GridBar* gb, long long limit,
                   int ipb, unsigned expect) {
  extern __shared__ float4 s_state[];
  float4* sx = s_state;         // x at the block's cell-times: (A.re, A.im, B.re, B.im)
  float4* sp = s_state + ipb;   // p
  float4* sr = sp + ipb;        // r
  __shared__ float s_a;
  __shared__ int s_stop;
  const int H = g.H;
  const int q0 = blockIdx.x * ipb;
  const int nloc = max(0, min(ipb, H - q0));
  for (int k = threadIdx.x; k < nloc; k += blockDim.x) {
    const int q = q0 + k;
    const float2 xa = x[q], xb = x[H + q], pa = p0[q], pb = p0[H + q], ra = r[q], rb = r[H + q];
    sx[k] = make_float4(xa.x, xa.y, xb.x, xb.y);
    sp[k] = make_float4(pa.x, pa.y, pb.x, pb.y);
    sr[k] = make_float4(ra.x, ra.y, rb.x, rb.y);
  }
  const float dm = sc->dm32, sigma = sc->sigma32, dk = g.dkf;
  // scalars, held by thread 0 in FP32 (the FP64 pipe is slow on this GPU and
  // the rest of the block waits for them); the partial sums stay float-float
  float rr = sc->rr32, rr_prev = 1.f, pAp = 0.f, alpha = 0.f, beta = 0.f;
  int iter = sc->iter, done = sc->done;
  const int maxit = sc->maxit;
  const float thresh = sc->thresh32;
  float2* pold = p0;
  float2* pnew = p1;
  bool first = true;
  __syncthreads();
  for (;;) {
    // convergence and limit checks (the same decision in every block)
    if (threadIdx.x == 0) {
      if (!done) {
        if (!isfinite(rr))
          done = CG_BREAKDOWN;
        else if (rr <= thresh)
          done = CG_CONVERGED;
        else if (iter >= maxit)
          done = CG_MAXIT;
      }
      beta = first ? 0.f : rr / rr_prev;
      s_a = beta;
      s_stop = done;
    }
    __syncthreads();
    if (s_stop) break;
    const float fb = s_a;
    // first half: p = r + beta p, u = M^dagger p, partial of |u|^2 + sigma |p|^2
    float loc = 0.f;
    for (int k = threadIdx.x; k < nloc; k += blockDim.x) {
      const int q = q0 + k;
      const Nbr nb = neighbours(g, q);
      const float4 ro = sr[k], po = sp[k];
      const Cx<float> pa{fmaf(fb, po.x, ro.x), fmaf(fb, po.y, ro.y)};
      const Cx<float> pb{fmaf(fb, po.z, ro.z), fmaf(fb, po.w, ro.w)};
      // r and p were written by other blocks during this launch: loads skip
      // L1 (not coherent across SMs) and read L2
      auto P = [&](int kk) {
        const float2 a = __ldcg(r + kk), bb = __ldcg(pold + kk);
        return Cx<float>{fmaf(fb, bb.x, a.x), fmaf(fb, bb.y, a.y)};
      };
      Cx<float> ea = ph(nb.tp);
      Cx<float> za = cneg_if(Cx<float>{ea.re - dm, -ea.im}, nb.wrap_tp);
      Cx<float> ta = cfma(za, P(nb.tp), Cx<float>{-pa.re, -pa.im});
      Cx<float> oa = hopsum(ta, dk, pb, P(H + nb.im1), P(H + nb.jm1));
      Cx<float> eb = ph(H + nb.tm);
      Cx<float> zb = cneg_if(Cx<float>{dm - eb.re, -eb.im}, nb.wrap_tm);
      Cx<float> tb = cfma(zb, P(H + nb.tm), pb);
      Cx<float> ob = hopsum(tb, dk, pa, P(nb.ip1), P(nb.jp1));
      sp[k] = make_float4(pa.re, pa.im, pb.re, pb.im);
      st(pnew, q, pa);
      st(pnew, H + q, pb);
      st(u, q, oa);
      st(u, H + q, ob);
      loc += norm2(oa) + norm2(ob);
      if (sigma != 0.f) loc += sigma * (norm2(pa) + norm2(pb));
    }
    {
      const float2 v = ff_block_sum(make_float2(loc, 0.f));
      if (threadIdx.x == 0) partA[blockIdx.x] = v;
    }
    if (!grid_barrier(gb, expect, limit)) {
      done = CG_TIMEOUT;
      break;
    }
    {
      const float2 tot = ff_sum_partials(partA, gridDim.x);
      if (threadIdx.x == 0) {
        pAp = tot.x + tot.y;
        const bool bad = !(pAp > 0.f) || !isfinite(pAp);
        alpha = bad ? 0.f : rr / pAp;
        if (bad) done = CG_BREAKDOWN;
        s_a = alpha;
        s_stop = bad;
      }
      __syncthreads();
      if (s_stop) break;
    }
    const float fa = s_a;
    // second half: A p = M u + sigma p, x += alpha p, r -= alpha A p, partial of |r|^2
    loc = 0.f;
    for (int k = threadIdx.x; k < nloc; k += blockDim.x) {
      const int q = q0 + k;
      const PairOut<float> o = m_pair_ld<float>(g, ph, dm, neighbours(g, q), [&](int kk) {
        const float2 v = __ldcg(u + kk);
        return Cx<float>{v.x, v.y};
      });
      const float4 po = sp[k];
      float4 xo = sx[k], ro = sr[k];
      const float apar = fmaf(sigma, po.x, o.a.re), apai = fmaf(sigma, po.y, o.a.im);
      const float apbr = fmaf(sigma, po.z, o.b.re), apbi = fmaf(sigma, po.w, o.b.im);
      xo.x = fmaf(fa, po.x, xo.x);
      xo.y = fmaf(fa, po.y, xo.y);
      xo.z = fmaf(fa, po.z, xo.z);
      xo.w = fmaf(fa, po.w, xo.w);
      ro.x = fmaf(-fa, apar, ro.x);
      ro.y = fmaf(-fa, apai, ro.y);
      ro.z = fmaf(-fa, apbr, ro.z);
      ro.w = fmaf(-fa, apbi, ro.w);
      sx[k] = xo;
      sr[k] = ro;
      r[q] = make_float2(ro.x, ro.y);
      r[H + q] = make_float2(ro.z, ro.w);
      loc = fmaf(ro.x, ro.x, fmaf(ro.y, ro.y, fmaf(ro.z, ro.z, fmaf(ro.w, ro.w, loc))));
    }
    {
      const float2 v = ff_block_sum(make_float2(loc, 0.f));
      if (threadIdx.x == 0) partB[blockIdx.x] = v;
    }
    if (!grid_barrier(gb, expect, limit)) {
      done = CG_TIMEOUT;
      break;
    }
    {
      const float2 tot = ff_sum_partials(partB, gridDim.x);
      if (threadIdx.x == 0) {
        rr_prev = rr;
        rr = tot.x + tot.y;
        ++iter;
      }
    }
    first = false;
    float2* t = pold;
    pold = pnew;
    pnew = t;
  }
  // x back to memory; block 0 records the state for the host
  for (int k = threadIdx.x; k < nloc; k += blockDim.x) {
    const int q = q0 + k;
    const float4 xo = sx[k];
    x[q] = make_float2(xo.x, xo.y);
    x[H + q] = make_float2(xo.z, xo.w);
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    sc->rr = rr;
    sc->rr_cur = rr;
    sc->rr32 = sc->rr_cur32 = rr;
    sc->pAp = pAp;
    sc->alpha = alpha;
    sc->beta = beta;
    sc->iter = iter;
    sc->first = 0;
    sc->done = done ? done : CG_MAXIT;
  }
}

// Launch plan of the persistent kernel: 4, 3, 2 or 1 resident blocks of
// kPersistThreads per SM, each with the 48 bytes of shared state of ipb
// cell-times; false when the lattice's state does not fit on chip.
static bool persist_plan(const hmc_ctx* c, const Geo& g, int* blocks, int* ipb, size_t* smem) {
  int dev_smem = 0;
  cudaDeviceGetAttribute(&dev_smem, cudaDevAttrMaxSharedMemoryPerBlockOptin, c->device);
  for (int per_sm = 4; per_sm >= 1; --per_sm) {
    const int nb = per_sm * c->nsm;
    const int ib = (g.H + nb - 1) / nb;
    const size_t sm = (size_t)ib * 3 * sizeof(float4);
    if ((long long)nb > cg32_part_capacity(c) || sm > (size_t)dev_smem) continue;
    if (cudaFuncSetAttribute((const void*)k_cg32_persist, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)sm) != cudaSuccess) {
      cudaGetLastError();
      continue;
    }
    int occ = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_cg32_persist, kPersistThreads, sm) != cudaSuccess) {
      cudaGetLastError();
      continue;
    }
    if (occ < per_sm) continue;
    *blocks = nb;
    *ipb = ib;
    *smem = sm;
    return true;
  }
  return false;
}

bool cg32_persist_ok(const hmc_ctx* c, const Geo& g) {
  int b, i;
  size_t s;
  return persist_plan(c, g, &b, &i, &s);
}

hmc_status cg32_persist_launch(hmc_ctx* c, const Geo& g, float2* x, float2* r, float2* p0, float2* p1,
                               float2* u, CGScal* sc) {
  int blocks = 0, ipb = 0;
  size_t smem = 0;
  if (!persist_plan(c, g, &blocks, &ipb, &smem))
    return fail(c, HMC_ERR_INVALID, "persistent CG state does not fit on chip");
  HMC_CUDA(c, cudaMemsetAsync(c->gbar, 0, sizeof(GridBar), c->stream));
  Phase<float> ph = phase_of<float>(c);
  float2* pa = (float2*)c->partA;
  float2* pb = (float2*)c->partB;
  GridBar* gb = c->gbar;
  // about one second of SM clock per barrier wait before giving up
  long long limit = c->bar_limit > 0 ? c->bar_limit : 2000000000LL;
  unsigned expect = (unsigned)blocks + (unsigned)c->bar_extra;  // arrivals a barrier waits for
  Geo gg = g;
  void* args[] = {&gg, &ph, &x, &r, &p0, &p1, &u, &sc, &pa, &pb, &gb, &limit, &ipb, &expect};
  cudaError_t le = cudaSuccess;
  HMC_TRY(launch_b(c, K_CG_PERSIST32, 0.0, [&] {
    le = cudaLaunchCooperativeKernel((const void*)k_cg32_persist, dim3(blocks), dim3(kPersistThreads), args,
                                     smem, c->stream);
  }));
  if (le != cudaSuccess) return cuda_fail(c, le, "persistent CG launch");
  return HMC_OK;
}

// Tiled variants are usable when the shared-memory window holds the tile's
// spatial neighbourhood and the grid's reduction partials fit their buffers.
bool cg32_march_ok(const hmc_ctx* c, const Geo& g, int threads, int tt) {
  if (tt < 1 || threads < 32 || threads > kMaxThreads) return false;
  const long long blocks = (long long)((g.V + threads - 1) / threads) * ((g.nt + tt - 1) / tt);
  return blocks <= cg32_part_capacity(c);
}

bool cg32_tiled_ok(const hmc_ctx* c, const Geo& g, int tc, int tt) {
  if (g.n > TileWin<256>::kMaxN || tc + 2 * (g.n + 1) > g.V || tt < 1) return false;
  const long long blocks = (long long)((g.V + tc - 1) / tc) * ((g.nt + tt - 1) / tt);
  return blocks <= cg32_part_capacity(c);
}


// Launch of the tiled (sh.tiled == 1) or marching (sh.tiled == 2) kernels of
// the pair, inside the caller's instrumented launch.
void cg32_alt_pmdag(hmc_ctx* c, const Geo& g, const Shape& sh, const float2* r, const float2* pold, float2* pnew,
                    float2* u, CGScal* sc, int GB) {
  const dim3 grid((g.V + sh.threads - 1) / sh.threads, (g.nt + sh.tt - 1) / sh.tt);
  const float2* pb = (const float2*)c->partB;
  float2* pa = (float2*)c->partA;
  if (sh.tiled == 2) {
    launch_pdl(c, k_cg32_pmdag_march, grid, sh.threads, c->stream, g, phase_of<float>(c), sh.tt, r, pold, pnew, u,
               sc, pb, GB, pa);
    return;
  }
  switch (sh.threads) {
    case 256: launch_pdl(c, k_cg32_pmdag_tiled<256>, grid, 256, c->stream, g, phase_of<float>(c), sh.tt, r, pold, pnew, u, sc, pb, GB, pa); break;
    case 512: launch_pdl(c, k_cg32_pmdag_tiled<512>, grid, 512, c->stream, g, phase_of<float>(c), sh.tt, r, pold, pnew, u, sc, pb, GB, pa); break;
    default: launch_pdl(c, k_cg32_pmdag_tiled<1024>, grid, 1024, c->stream, g, phase_of<float>(c), sh.tt, r, pold, pnew, u, sc, pb, GB, pa); break;
  }
}

void cg32_alt_m(hmc_ctx* c, const Geo& g, const Shape& sh, const float2* u, const float2* p, float2* x, float2* r,
                CGScal* sc, int GA) {
  const dim3 grid((g.V + sh.threads - 1) / sh.threads, (g.nt + sh.tt - 1) / sh.tt);
  const float2* pa = (const float2*)c->partA;
  float2* pb = (float2*)c->partB;
  if (sh.tiled == 2) {
    launch_pdl(c, k_cg32_m_march, grid, sh.threads, c->stream, g, phase_of<float>(c), sh.tt, u, p, x, r, sc, pa, GA,
               pb);
    return;
  }
  switch (sh.threads) {
    case 256: launch_pdl(c, k_cg32_m_tiled<256>, grid, 256, c->stream, g, phase_of<float>(c), sh.tt, u, p, x, r, sc, pa, GA, pb); break;
    case 512: launch_pdl(c, k_cg32_m_tiled<512>, grid, 512, c->stream, g, phase_of<float>(c), sh.tt, u, p, x, r, sc, pa, GA, pb); break;
    default: launch_pdl(c, k_cg32_m_tiled<1024>, grid, 1024, c->stream, g, phase_of<float>(c), sh.tt, u, p, x, r, sc, pa, GA, pb); break;
  }
}

}  // namespace hmc
