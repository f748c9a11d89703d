// The libhmc kernels: operator applications, fused CG iterations, residuals,
// FGMRES vector operations and the pseudofermion force.
#include "kernels.h"
#include "operator.cuh"

namespace hmc {

// Algorithmic HBM bytes per lattice site of each kernel (reads + writes of the
// arrays it must touch, each once), used to report achieved bandwidth.
const char* const kKernelNames[K_COUNT] = {
    "phase_table",    "apply_Mdag_f64", "apply_M_f64",   "apply_Mdag_f32", "apply_M_f32",
    "cg_Mdag_f64",    "cg_M_update_f64", "cg_p_f64",     "cg_pMdag_f32",    "cg_M_update_f32",
    "cg_p_f32",       "residual_f64",   "residual_f32",  "cg_init0",       "convert",
    "norm2",          "gmres_mdot",     "gmres_gs_update", "gmres_scale",  "gmres_x_update",
    "force",          "axpy",           "md_update",     "batch_cg_graph_f64", "batch_cg_graph_f32",
    "batch_init",     "batch_residual", "batch_misc",   "cg_persist_f32"};

const double kKernelBytesPerSite[K_COUNT] = {
    8 + 16 + 4,          // phase: phi in, E and phi32 out
    16 + 16 + 16,        // M^dagger f64: in, E, out
    16 + 16 + 16,        // M f64
    8 + 4 + 8,           // M^dagger f32: in, phi32, out
    8 + 4 + 8,           // M f32
    16 + 16 + 16,        // cg M^dagger f64: p, E, u
    16 + 16 + 16 + 32 + 32,  // cg M f64: u, E, p, x rw, r rw
    16 + 32,             // p = r + beta p
    8 + 8 + 4 + 8 + 8,   // cg M^dagger f32 with the p update: r, p_old, phi32, p_new, u
    8 + 4 + 8 + 16 + 16, // cg M f32
    8 + 16,              // p f32
    16 + 16 + 16 + 16 + 16,  // residual f64: u, E, x, b, r
    8 + 4 + 8 + 8 + 8,   // residual f32
    16 + 16 * 3,         // init0 (f64 sizes)
    16 + 8,              // convert
    16,                  // norm2
    0,                   // mdot (depends on the basis size)
    0,                   // gs update
    16 + 16 + 8,         // scale
    0,                   // x update
    16 + 16 + 16 + 16 + 16,  // force: eta, E, xi, chi, grad rw
    24,                  // axpy
    24,                  // md update
    192, 96, 16 * 4, 16 * 5, 0,
    0};  // persistent CG: 56 B per site and iteration, counted after the solve

// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(kThreads) k_phase(int N, const double* __restrict__ phi,
                                                    double2* __restrict__ E,
                                                    float* __restrict__ phi32) {
  for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < N; k += gridDim.x * blockDim.x) {
    double s, co;
    double x = phi[k];
    sincos(x, &s, &co);
    E[k] = make_double2(co, s);
    phi32[k] = (float)x;
  }
}

template <typename R>
Phase<R> phase_of(hmc_ctx* c);
template <>
Phase<double> phase_of<double>(hmc_ctx* c) {
  return Phase<double>{(const double2*)c->ws[WS_E]};
}
template <>
Phase<float> phase_of<float>(hmc_ctx* c) {
  return Phase<float>{(const float*)c->ws[WS_PHI32]};
}

template <typename R>
__global__ void __launch_bounds__(kThreads) k_mdag(Geo g, Phase<R> ph, R dm,
                                                   const V2<R>* __restrict__ p,
                                                   V2<R>* __restrict__ out) {
  for (int q = blockIdx.x * blockDim.x + threadIdx.x; q < g.H; q += gridDim.x * blockDim.x) {
    Nbr nb = neighbours(g, q);
    PairOut<R> o = mdag_pair<R>(g, ph, dm, p, nb);
    st(out, q, o.a);
    st(out, g.H + q, o.b);
  }
}

template <typename R>
__global__ void __launch_bounds__(kThreads) k_m(Geo g, Phase<R> ph, R dm, const V2<R>* __restrict__ u,
                                                const V2<R>* __restrict__ y, R sigma,
                                                V2<R>* __restrict__ out) {
  for (int q = blockIdx.x * blockDim.x + threadIdx.x; q < g.H; q += gridDim.x * blockDim.x) {
    Nbr nb = neighbours(g, q);
    PairOut<R> o = m_pair<R>(g, ph, dm, u, nb);
    if (y != nullptr) {
      Cx<R> ya = ld<R>(y, q), yb = ld<R>(y, g.H + q);
      o.a.re = fma(sigma, ya.re, o.a.re);
      o.a.im = fma(sigma, ya.im, o.a.im);
      o.b.re = fma(sigma, yb.re, o.b.re);
      o.b.im = fma(sigma, yb.im, o.b.im);
    }
    st(out, q, o.a);
    st(out, g.H + q, o.b);
  }
}

// u = M^dagger p; pAp = |u|^2 + sigma |p|^2 = <p, (M M^dagger + sigma) p>; alpha = rr / pAp.
template <typename R>
__global__ void __launch_bounds__(kMaxThreads) k_cg_mdag(Geo g, Phase<R> ph,
                                                      const V2<R>* __restrict__ p,
                                                      V2<R>* __restrict__ u, CGScal* sc,
                                                      double* partials, unsigned* ticket) {
  pdl_wait();
  if (sc->done) return;
  const R dm = (R)sc->dm;
  const R sigma = (R)sc->sigma;
  double acc[1] = {0.0};
  for (int q = blockIdx.x * blockDim.x + threadIdx.x; q < g.H; q += gridDim.x * blockDim.x) {
    Nbr nb = neighbours(g, q);
    PairOut<R> o = mdag_pair<R>(g, ph, dm, p, nb);
    st(u, q, o.a);
    st(u, g.H + q, o.b);
    R loc = norm2(o.a) + norm2(o.b);
    if (sigma != (R)0) loc += sigma * (norm2(ld<R>(p, q)) + norm2(ld<R>(p, g.H + q)));
    acc[0] += (double)loc;
  }
  pdl_trigger();
  double tot[1];
  if (grid_sum<1>(acc, partials, ticket, tot) && threadIdx.x == 0) {
    double pAp = tot[0];
    sc->pAp = pAp;
    if (!(pAp > 0.0) || !isfinite(pAp)) {
      sc->alpha = 0.0;
      sc->done = CG_BREAKDOWN;
    } else {
      sc->alpha = sc->rr / pAp;
    }
  }
}

// A p = M u + sigma p;  x += alpha p;  r -= alpha A p;  beta = |r_new|^2 / |r|^2.
template <typename R>
__global__ void __launch_bounds__(kMaxThreads) k_cg_m(Geo g, Phase<R> ph,
                                                   const V2<R>* __restrict__ u,
                                                   const V2<R>* __restrict__ p, V2<R>* __restrict__ x,
                                                   V2<R>* __restrict__ r, CGScal* sc,
                                                   double* partials, unsigned* ticket) {
  pdl_wait();
  if (sc->done) return;
  const R dm = (R)sc->dm;
  const R sigma = (R)sc->sigma;
  const R alpha = (R)sc->alpha;
  double acc[1] = {0.0};
  for (int q = blockIdx.x * blockDim.x + threadIdx.x; q < g.H; q += gridDim.x * blockDim.x) {
    Nbr nb = neighbours(g, q);
    PairOut<R> o = m_pair<R>(g, ph, dm, u, nb);
    R loc = 0;
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const int k = h ? g.H + q : q;
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
    acc[0] += (double)loc;
  }
  pdl_trigger();
  double tot[1];
  if (grid_sum<1>(acc, partials, ticket, tot) && threadIdx.x == 0) {
    double rr = tot[0];
    sc->beta = rr / sc->rr;
    sc->rr = rr;
    sc->iter += 1;
    if (!isfinite(rr))
      sc->done = CG_BREAKDOWN;
    else if (rr <= sc->thresh)
      sc->done = CG_CONVERGED;
    else if (sc->iter >= sc->maxit)
      sc->done = CG_MAXIT;
  }
}

template <typename R>
__global__ void __launch_bounds__(kMaxThreads) k_cg_p(int N, const V2<R>* __restrict__ r,
                                                   V2<R>* __restrict__ p, const CGScal* sc) {
  pdl_wait();
  if (sc->done) return;
  pdl_trigger();
  const R beta = (R)sc->beta;
  for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < N; k += gridDim.x * blockDim.x) {
    Cx<R> rk = ld<R>(r, k), pk = ld<R>(p, k);
    pk.re = fma(beta, pk.re, rk.re);
    pk.im = fma(beta, pk.im, rk.im);
    st(p, k, pk);
  }
}

// FP32 CG, two kernels per iteration, no atomics and no last-block tail: a
// kernel only writes one reduction partial per block; every block of the next
// kernel sums those partials itself in the same fixed order (so all blocks hold
// identical scalars) after pdl_wait() has made them visible.
//
// Kernel A (iteration i): rr_i = sum of B's partials; convergence and limit
// checks; beta = rr_i / rr_{i-1} (0 on the first iteration); then
//   p_new = r + beta p_old, u = M^dagger p_new,
//   partial of pAp = |u|^2 + sigma |p_new|^2.
// Kernel B: pAp = sum of A's partials, alpha = rr_i / pAp; then
//   A p = M u + sigma p_new;  x += alpha p_new;  r -= alpha A p;  partial of |r|^2.
// Block 0 records the scalars in sc for the host.
//
// The scalars of a kernel are known only after its block has summed the
// previous kernel's partials. So that the stencil loads of a thread's first
// item are in flight during that reduction, each kernel evaluates its first
// item's stencil before the reduction: kernel B computes M u (which does not
// depend on alpha), kernel A computes M^dagger r and M^dagger p_old separately
// and forms M^dagger p_new = M^dagger r + beta M^dagger p_old once beta is
// known (linearity; both stencils are evaluated afresh from the stored vectors
// every iteration, so no recurrence error builds up). Later items use the
// direct form.
__device__ __forceinline__ void cg32_time_factors(const Phase<float>& ph, const Nbr& nb, int H, float dm,
                                                  Cx<float>& za, Cx<float>& zb) {
  Cx<float> ea = ph(nb.tp);
  za = cneg_if(Cx<float>{ea.re - dm, -ea.im}, nb.wrap_tp);
  Cx<float> eb = ph(H + nb.tm);
  zb = cneg_if(Cx<float>{dm - eb.re, -eb.im}, nb.wrap_tm);
}

__global__ void __launch_bounds__(kMaxThreads) k_cg32_pmdag(Geo g, Phase<float> ph,
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
  const float dm = sc->dm32, sigma = sc->sigma32, dk = g.dkf;
  const int H = g.H;
  const int stride = gridDim.x * blockDim.x;
  int q = blockIdx.x * blockDim.x + threadIdx.x;
  // first item: both stencils, before beta is known
  const bool have0 = q < H;
  Nbr nb0;
  PairOut<float> mr{}, mp{};
  float2 r0a{}, r0b{}, p0a{}, p0b{};
  if (have0) {
    nb0 = neighbours(g, q);
    Cx<float> za, zb;
    cg32_time_factors(ph, nb0, H, dm, za, zb);
    mr = mdag_pair_ld<float>(g, za, zb, dk, nb0, [&](int k) { float2 v = r[k]; return Cx<float>{v.x, v.y}; });
    r0a = r[nb0.q];
    r0b = r[H + nb0.q];
    if (!first) {
      mp = mdag_pair_ld<float>(g, za, zb, dk, nb0, [&](int k) { float2 v = pold[k]; return Cx<float>{v.x, v.y}; });
      p0a = pold[nb0.q];
      p0b = pold[H + nb0.q];
    }
  }
  // |r|^2: from the init kernel on the first iteration, else from B's partials;
  // the scalars are formed once per block by thread 0
  const float2 rr_pair = first ? make_float2(0.f, 0.f) : ff_sum_partials(partB, GB);
  if (threadIdx.x == 0) {
    const double rr = first ? sc->rr_cur : ff_to_double(rr_pair);
    int done = CG_RUNNING;
    if (!isfinite(rr))
      done = CG_BREAKDOWN;
    else if (rr <= sc->thresh)
      done = CG_CONVERGED;
    else if (sc->iter >= sc->maxit)
      done = CG_MAXIT;
    const double beta = first ? 0.0 : rr / sc->rr;
    s_beta = (float)beta;
    s_done = done;
    if (blockIdx.x == 0) {
      sc->rr_cur = rr;
      sc->beta = beta;
      if (done) {
        sc->rr = rr;
        sc->done = done;
      }
    }
  }
  __syncthreads();
  if (s_done) return;
  const float beta = s_beta;
  float loc = 0.f;
  if (have0) {
    Cx<float> pa{fmaf(beta, p0a.x, r0a.x), fmaf(beta, p0a.y, r0a.y)};
    Cx<float> pb{fmaf(beta, p0b.x, r0b.x), fmaf(beta, p0b.y, r0b.y)};
    Cx<float> oa{fmaf(beta, mp.a.re, mr.a.re), fmaf(beta, mp.a.im, mr.a.im)};
    Cx<float> ob{fmaf(beta, mp.b.re, mr.b.re), fmaf(beta, mp.b.im, mr.b.im)};
    st(pnew, nb0.q, pa);
    st(pnew, H + nb0.q, pb);
    st(u, nb0.q, oa);
    st(u, H + nb0.q, ob);
    loc += norm2(oa) + norm2(ob);
    if (sigma != 0.f) loc += sigma * (norm2(pa) + norm2(pb));
  }
  for (q += stride; q < H; q += stride) {
    Nbr nb = neighbours(g, q);
    auto P = [&](int k) {
      float2 a = r[k], b = pold[k];
      return Cx<float>{fmaf(beta, b.x, a.x), fmaf(beta, b.y, a.y)};
    };
    Cx<float> za, zb;
    cg32_time_factors(ph, nb, H, dm, za, zb);
    PairOut<float> o = mdag_pair_ld<float>(g, za, zb, dk, nb, P);
    Cx<float> pa = P(nb.q), pb = P(H + nb.q);
    st(pnew, nb.q, pa);
    st(pnew, H + nb.q, pb);
    st(u, nb.q, o.a);
    st(u, H + nb.q, o.b);
    loc += norm2(o.a) + norm2(o.b);
    if (sigma != 0.f) loc += sigma * (norm2(pa) + norm2(pb));
  }
  pdl_trigger();
  ff_write_partial(loc, partA);
}

__global__ void __launch_bounds__(kMaxThreads) k_cg32_m(Geo g, Phase<float> ph,
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
  const float dm = sc->dm32, sigma = sc->sigma32;
  const int H = g.H;
  const int stride = gridDim.x * blockDim.x;
  int q = blockIdx.x * blockDim.x + threadIdx.x;
  // first item: M u before alpha is known
  const bool have0 = q < H;
  PairOut<float> o0{};
  if (have0) o0 = m_pair<float>(g, ph, dm, u, neighbours(g, q));
  const float2 pAp_pair = ff_sum_partials(partA, GA);
  if (threadIdx.x == 0) {
    const double pAp = ff_to_double(pAp_pair);
    const double rr = sc->rr_cur;
    const bool bad = !(pAp > 0.0) || !isfinite(pAp);
    s_bad = bad;
    s_alpha = bad ? 0.f : (float)(rr / pAp);
    if (blockIdx.x == 0) {
      sc->pAp = pAp;
      sc->rr = rr;
      sc->first = 0;
      if (bad) {
        sc->alpha = 0.0;
        sc->done = CG_BREAKDOWN;
      } else {
        sc->alpha = rr / pAp;
        sc->iter += 1;
      }
    }
  }
  __syncthreads();
  if (s_bad) return;
  const float alpha = s_alpha;
  float loc = 0.f;
  auto update = [&](int qq, const PairOut<float>& o) {
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const int k = h ? H + qq : qq;
      Cx<float> Ap = h ? o.b : o.a;
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
  };
  if (have0) update(q, o0);
  for (q += stride; q < H; q += stride) update(q, m_pair<float>(g, ph, dm, u, neighbours(g, q)));
  pdl_trigger();
  ff_write_partial(loc, partB);
}

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
    const double rr = first ? sc->rr_cur : ff_to_double(rr_pair);
    int done = CG_RUNNING;
    if (!isfinite(rr))
      done = CG_BREAKDOWN;
    else if (rr <= sc->thresh)
      done = CG_CONVERGED;
    else if (sc->iter >= sc->maxit)
      done = CG_MAXIT;
    const double beta = first ? 0.0 : rr / sc->rr;
    s_beta = (float)beta;
    s_done = done;
    if (blockIdx.x == 0 && blockIdx.y == 0) {
      sc->rr_cur = rr;
      sc->beta = beta;
      if (done) {
        sc->rr = rr;
        sc->done = done;
      }
    }
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
    const double pAp = ff_to_double(pAp_pair);
    const double rr = sc->rr_cur;
    const bool bad = !(pAp > 0.0) || !isfinite(pAp);
    s_bad = bad;
    s_alpha = bad ? 0.f : (float)(rr / pAp);
    if (blockIdx.x == 0 && blockIdx.y == 0) {
      sc->pAp = pAp;
      sc->rr = rr;
      sc->first = 0;
      if (bad) {
        sc->alpha = 0.0;
        sc->done = CG_BREAKDOWN;
      } else {
        sc->alpha = rr / pAp;
        sc->iter += 1;
      }
    }
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
    const double rr = first ? sc->rr_cur : ff_to_double(rr_pair);
    int done = CG_RUNNING;
    if (!isfinite(rr))
      done = CG_BREAKDOWN;
    else if (rr <= sc->thresh)
      done = CG_CONVERGED;
    else if (sc->iter >= sc->maxit)
      done = CG_MAXIT;
    const double beta = first ? 0.0 : rr / sc->rr;
    s_beta = (float)beta;
    s_done = done;
    if (blockIdx.x == 0 && blockIdx.y == 0) {
      sc->rr_cur = rr;
      sc->beta = beta;
      if (done) {
        sc->rr = rr;
        sc->done = done;
      }
    }
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
    const double pAp = ff_to_double(pAp_pair);
    const double rr = sc->rr_cur;
    const bool bad = !(pAp > 0.0) || !isfinite(pAp);
    s_bad = bad;
    s_alpha = bad ? 0.f : (float)(rr / pAp);
    if (blockIdx.x == 0 && blockIdx.y == 0) {
      sc->pAp = pAp;
      sc->rr = rr;
      sc->first = 0;
      if (bad) {
        sc->alpha = 0.0;
        sc->done = CG_BREAKDOWN;
      } else {
        sc->alpha = rr / pAp;
        sc->iter += 1;
      }
    }
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
__device__ __forceinline__ bool grid_barrier(GridBar* gb, unsigned nblocks, long long limit) {
  __shared__ int s_ok;
  __syncthreads();
  if (threadIdx.x == 0) {
    volatile unsigned* vgen = &gb->gen;
    volatile int* verr = &gb->err;
    int ok = (*verr == 0);
    if (ok) {
      const unsigned my = *vgen;
      __threadfence();
      if (atomicAdd(&gb->count, 1u) == nblocks - 1u) {
        atomicExch(&gb->count, 0u);
        __threadfence();
        atomicAdd(&gb->gen, 1u);
      } else {
        const long long t0 = clock64();
        while (*vgen == my) {
          if (*verr) {
            ok = 0;
            break;
          }
          if (clock64() - t0 > limit) {
            atomicExch(&gb->err, 1);
            ok = 0;
            break;
          }
          __nanosleep(64);
        }
      }
      __threadfence();
    }
    s_ok = ok;
  }
  __syncthreads();
  return s_ok != 0;
}

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
  // scalars, held by thread 0 in FP64 and handed to the block as floats
  double rr = sc->rr, rr_prev = 1.0, pAp = 0.0, alpha = 0.0, beta = 0.0;
  int iter = sc->iter, done = sc->done;
  const int maxit = sc->maxit;
  const double thresh = sc->thresh;
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
      beta = first ? 0.0 : rr / rr_prev;
      s_a = (float)beta;
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
        pAp = ff_to_double(tot);
        const bool bad = !(pAp > 0.0) || !isfinite(pAp);
        alpha = bad ? 0.0 : rr / pAp;
        if (bad) done = CG_BREAKDOWN;
        s_a = (float)alpha;
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
        rr = ff_to_double(tot);
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

template <typename R>
__global__ void __launch_bounds__(kThreads) k_resid(Geo g, Phase<R> ph, R dm,
                                                    const V2<R>* __restrict__ u,
                                                    const V2<R>* __restrict__ x,
                                                    const V2<R>* __restrict__ b, R sigma,
                                                    V2<R>* __restrict__ r, V2<R>* __restrict__ p,
                                                    CGScal* init, double tol2, int maxit,
                                                    double dsigma, double ddm, double* out2,
                                                    double* partials, unsigned* ticket) {
  double acc[2] = {0.0, 0.0};
  for (int q = blockIdx.x * blockDim.x + threadIdx.x; q < g.H; q += gridDim.x * blockDim.x) {
    Nbr nb = neighbours(g, q);
    PairOut<R> o = m_pair<R>(g, ph, dm, u, nb);
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const int k = h ? g.H + q : q;
      Cx<R> Ax = h ? o.b : o.a;
      Cx<R> xk = ld<R>(x, k), bk = ld<R>(b, k);
      Cx<R> rk;
      rk.re = bk.re - fma(sigma, xk.re, Ax.re);
      rk.im = bk.im - fma(sigma, xk.im, Ax.im);
      st(r, k, rk);
      if (p != nullptr) st(p, k, rk);
      acc[0] += (double)norm2(rk);
      acc[1] += (double)norm2(bk);
    }
  }
  double tot[2];
  if (grid_sum<2>(acc, partials, ticket, tot) && threadIdx.x == 0) {
    if (out2 != nullptr) {
      out2[0] = tot[0];
      out2[1] = tot[1];
    }
    if (init != nullptr) {
      init->rr = tot[0];
      init->bb = tot[1];
      init->thresh = tol2 * tot[1];
      init->sigma = dsigma;
      init->dm = ddm;
      init->sigma32 = (float)dsigma;
      init->dm32 = (float)ddm;
      init->iter = 0;
      init->maxit = maxit;
      init->alpha = init->beta = init->pAp = 0.0;
      init->done = (tot[0] <= init->thresh) ? CG_CONVERGED : CG_RUNNING;
      if (!isfinite(tot[0])) init->done = CG_BREAKDOWN;
      init->first = 1;
      init->rr_cur = tot[0];
    }
  }
}

template <typename R>
__global__ void __launch_bounds__(kThreads) k_init0(int N, const V2<R>* __restrict__ b,
                                                    V2<R>* __restrict__ x, V2<R>* __restrict__ r,
                                                    V2<R>* __restrict__ p, CGScal* sc, double tol2,
                                                    int maxit, double sigma, double ddm,
                                                    double* partials, unsigned* ticket) {
  double acc[1] = {0.0};
  for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < N; k += gridDim.x * blockDim.x) {
    Cx<R> bk = ld<R>(b, k);
    st(x, k, Cx<R>{(R)0, (R)0});
    st(r, k, bk);
    st(p, k, bk);
    acc[0] += (double)norm2(bk);
  }
  double tot[1];
  if (grid_sum<1>(acc, partials, ticket, tot) && threadIdx.x == 0) {
    sc->rr = tot[0];
    sc->bb = tot[0];
    sc->thresh = tol2 * tot[0];
    sc->sigma = sigma;
    sc->dm = ddm;
    sc->sigma32 = (float)sigma;
    sc->dm32 = (float)ddm;
    sc->iter = 0;
    sc->maxit = maxit;
    sc->alpha = sc->beta = sc->pAp = 0.0;
    sc->done = (tot[0] <= sc->thresh) ? CG_CONVERGED : CG_RUNNING;
    if (!isfinite(tot[0])) sc->done = CG_BREAKDOWN;
    sc->first = 1;
    sc->rr_cur = tot[0];
  }
}

__global__ void __launch_bounds__(kThreads) k_to32(int N, const double2* __restrict__ in,
                                                   float2* __restrict__ out) {
  for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < N; k += gridDim.x * blockDim.x) {
    double2 v = in[k];
    out[k] = make_float2((float)v.x, (float)v.y);
  }
}
__global__ void __launch_bounds__(kThreads) k_to64(int N, const float2* __restrict__ in,
                                                   double2* __restrict__ out) {
  for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < N; k += gridDim.x * blockDim.x) {
    float2 v = in[k];
    out[k] = make_double2((double)v.x, (double)v.y);
  }
}

__global__ void __launch_bounds__(kThreads) k_norm2(int N, const double2* __restrict__ v, double* out,
                                                    double* partials, unsigned* ticket) {
  double acc[1] = {0.0};
  for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < N; k += gridDim.x * blockDim.x) {
    double2 a = v[k];
    acc[0] = fma(a.x, a.x, fma(a.y, a.y, acc[0]));
  }
  double tot[1];
  if (grid_sum<1>(acc, partials, ticket, tot) && threadIdx.x == 0) *out = tot[0];
}

__global__ void __launch_bounds__(kThreads) k_redot(int N, const double2* __restrict__ u,
                                                    const double2* __restrict__ v, double* out,
                                                    double* partials, unsigned* ticket) {
  double acc[1] = {0.0};
  for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < N; k += gridDim.x * blockDim.x) {
    double2 a = u[k], b = v[k];
    acc[0] = fma(a.x, b.x, fma(a.y, b.y, acc[0]));
  }
  double tot[1];
  if (grid_sum<1>(acc, partials, ticket, tot) && threadIdx.x == 0) *out = tot[0];
}

// h[i] = V_i^H w for the NV basis vectors (NV a compile-time constant, so the
// basis pointers stay in the parameter bank and every loop unrolls).
template <int NV>
__global__ void __launch_bounds__(kThreads) k_mdot(int N, VecList V, const double2* __restrict__ w,
                                                   double* hout, double* partials, unsigned* ticket) {
  double acc[2 * NV];
#pragma unroll
  for (int i = 0; i < 2 * NV; ++i) acc[i] = 0.0;
  for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < N; k += gridDim.x * blockDim.x) {
    double2 wk = w[k];
#pragma unroll
    for (int i = 0; i < NV; ++i) {
      double2 vk = V.v[i][k];
      // conj(v) w
      acc[2 * i] = fma(vk.x, wk.x, fma(vk.y, wk.y, acc[2 * i]));
      acc[2 * i + 1] = fma(vk.x, wk.y, fma(-vk.y, wk.x, acc[2 * i + 1]));
    }
  }
  double tot[2 * NV];
  if (grid_sum<2 * NV>(acc, partials, ticket, tot) && threadIdx.x == 0) {
#pragma unroll
    for (int i = 0; i < 2 * NV; ++i) hout[i] = tot[i];
  }
}

// w -= sum_i h[i] V_i over the NV basis vectors, then |w|^2.
template <int NV>
__global__ void __launch_bounds__(kThreads) k_gsupd(int N, VecList V, const double* h,
                                                    double2* __restrict__ w, double* ww,
                                                    double* partials, unsigned* ticket) {
  __shared__ double hs[2 * NV];
  if (threadIdx.x < 2 * NV) hs[threadIdx.x] = h[threadIdx.x];
  __syncthreads();
  double acc[1] = {0.0};
  for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < N; k += gridDim.x * blockDim.x) {
    double2 wk = w[k];
#pragma unroll
    for (int i = 0; i < NV; ++i) {
      double2 vk = V.v[i][k];
      const double hr = hs[2 * i], hi = hs[2 * i + 1];
      // w -= h v
      wk.x = fma(-hr, vk.x, fma(hi, vk.y, wk.x));
      wk.y = fma(-hr, vk.y, fma(-hi, vk.x, wk.y));
    }
    w[k] = wk;
    acc[0] = fma(wk.x, wk.x, fma(wk.y, wk.y, acc[0]));
  }
  double tot[1];
  if (grid_sum<1>(acc, partials, ticket, tot) && threadIdx.x == 0) *ww = tot[0];
}

__global__ void __launch_bounds__(kThreads) k_scale(int N, double s, const double2* __restrict__ w,
                                                    double2* __restrict__ v, float2* __restrict__ v32) {
  for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < N; k += gridDim.x * blockDim.x) {
    double2 a = w[k];
    a.x *= s;
    a.y *= s;
    v[k] = a;
    if (v32 != nullptr) v32[k] = make_float2((float)a.x, (float)a.y);
  }
}

__global__ void __launch_bounds__(kThreads) k_xupd(int N, VecList Z, CoefList y, int nz,
                                                   double2* __restrict__ x) {
  for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < N; k += gridDim.x * blockDim.x) {
    double2 xk = x[k];
    for (int i = 0; i < nz; ++i) {
      double2 z = Z.v[i][k];
      xk.x = fma(y.re[i], z.x, fma(-y.im[i], z.y, xk.x));
      xk.y = fma(y.re[i], z.y, fma(y.im[i], z.x, xk.y));
    }
    x[k] = xk;
  }
}

__global__ void __launch_bounds__(kThreads) k_axpy_real(int N, double a, const double* __restrict__ x,
                                                        double* __restrict__ y) {
  for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < N; k += gridDim.x * blockDim.x)
    y[k] = fma(a, x[k], y[k]);
}

__global__ void __launch_bounds__(kThreads) k_axpby_c(int N, double a, const double2* __restrict__ x,
                                                      double b, double2* __restrict__ y) {
  for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < N; k += gridDim.x * blockDim.x) {
    double2 xv = x[k], yv = y[k];
    y[k] = make_double2(fma(a, xv.x, b * yv.x), fma(a, xv.y, b * yv.y));
  }
}

// Force of one term at the cell-time q. dM/dphi in row k is i s e^{+i phi} (A)
// or i s e^{-i phi} (B), s = -1 on the wrapping hop; its column is the time
// partner (t-1 for A, t+1 for B). With c = conj(eta_k) dM_k w_tp:
//   -2 Re(c) = 2 s Im(conj(eta) e^{+-i phi} w_tp).
__global__ void __launch_bounds__(kThreads) k_force(Geo g, Phase<double> ph,
                                                    const double2* __restrict__ eta,
                                                    const double2* __restrict__ xi,
                                                    const double2* __restrict__ chi,
                                                    double* __restrict__ grad) {
  for (int q = blockIdx.x * blockDim.x + threadIdx.x; q < g.H; q += gridDim.x * blockDim.x) {
    Nbr nb = neighbours(g, q);
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const int k = h ? g.H + q : q;
      const int kp = h ? g.H + nb.tp : nb.tm;
      const bool wrap = h ? nb.wrap_tp : nb.wrap_tm;
      Cx<double> e = ph(k);
      if (h) e.im = -e.im;  // B rows: e^{-i phi}
      double2 wv = xi[kp];
      if (chi != nullptr) {
        double2 cv = chi[kp];
        wv.x -= cv.x;
        wv.y -= cv.y;
      }
      double2 et = eta[k];
      // c0 = e * w ;  Im(conj(eta) c0) = et.x * c0.im - et.y * c0.re
      double c0r = e.re * wv.x - e.im * wv.y;
      double c0i = e.re * wv.y + e.im * wv.x;
      double im = et.x * c0i - et.y * c0r;
      double val = 2.0 * (wrap ? -im : im);
      grad[k] += val;
    }
  }
}

__global__ void __launch_bounds__(kThreads) k_gauss_grad(int N, const double* __restrict__ phi,
                                                         double inv_dU, int accumulate,
                                                         double* __restrict__ grad) {
  for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < N; k += gridDim.x * blockDim.x) {
    double v = phi[k] * inv_dU;
    grad[k] = accumulate ? grad[k] + v : v;
  }
}

__global__ void __launch_bounds__(kThreads) k_half_sq(int N, const double* __restrict__ a, double sa,
                                                      const double* __restrict__ b, double* out,
                                                      double* partials, unsigned* ticket) {
  double acc[2] = {0.0, 0.0};
  for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < N; k += gridDim.x * blockDim.x) {
    double x = a[k];
    acc[0] = fma(x, x, acc[0]);
    if (b != nullptr) {
      double y = b[k];
      acc[1] = fma(y, y, acc[1]);
    }
  }
  double tot[2];
  if (grid_sum<2>(acc, partials, ticket, tot) && threadIdx.x == 0) {
    out[0] = 0.5 * sa * tot[0];
    out[1] = 0.5 * tot[1];
  }
}

// ---------------------------------------------------------------------------
// Launchers
#define GRID(work) grid_for(c, (work)), kThreads, 0, c->stream
// Launch with the programmatic-serialization attribute (see pdl_wait).
// Programmatic launches are used only between consecutive kernels of a
// captured iteration chunk: the first kernel of a capture (no kernel before it
// in the graph) and every launch outside a capture are ordinary launches.
template <typename... KA, typename... A>
static void launch_pdl(hmc_ctx* c, void (*k)(KA...), dim3 grid, int threads, cudaStream_t s, A... args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = grid;
  cfg.blockDim = dim3(threads);
  cfg.dynamicSmemBytes = 0;
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  const bool pdl = c->capturing && c->pdl_armed;
  cfg.attrs = pdl ? attr : nullptr;
  cfg.numAttrs = pdl ? 1 : 0;
  (void)cudaLaunchKernelEx(&cfg, k, ((KA)args)...);  // errors surface through cudaGetLastError
  if (c->capturing) c->pdl_armed = true;
}
#define PDL(id, work) dim3(shape_grid(c, (id), (work))), c->shape[(id)].threads, c->stream

// tuned launch shape of a CG kernel
#define SHAPE(id, work) shape_grid(c, (id), (work)), c->shape[(id)].threads, 0, c->stream

hmc_status k_phase_launch(hmc_ctx* c, const double* phi) {
  const int N = c->geo.N;
  return launch(c, K_PHASE, [&] {
    k_phase<<<GRID(N)>>>(N, phi, (double2*)c->ws[WS_E], (float*)c->ws[WS_PHI32]);
  });
}

template <typename R>
hmc_status mdag_launch(hmc_ctx* c, const Geo& g, R dm, const V2<R>* p, V2<R>* out) {
  return launch(c, sizeof(R) == 8 ? K_MDAG64 : K_MDAG32,
                [&] { k_mdag<R><<<GRID(g.H)>>>(g, phase_of<R>(c), dm, p, out); });
}
template <typename R>
hmc_status m_launch(hmc_ctx* c, const Geo& g, R dm, const V2<R>* u, const V2<R>* y, R sigma,
                    V2<R>* out) {
  return launch(c, sizeof(R) == 8 ? K_M64 : K_M32,
                [&] { k_m<R><<<GRID(g.H)>>>(g, phase_of<R>(c), dm, u, y, sigma, out); });
}
template <typename R>
hmc_status cg_mdag_launch(hmc_ctx* c, const Geo& g, const V2<R>* p, V2<R>* u, CGScal* sc,
                          unsigned* ticket) {
  return launch(c, sizeof(R) == 8 ? K_CG_MDAG64 : K_CG_MDAG32, [&] {
    launch_pdl(c, k_cg_mdag<R>, PDL(sizeof(R) == 8 ? K_CG_MDAG64 : K_CG_MDAG32, g.H), g, phase_of<R>(c), p,
               u, sc, c->partials, ticket);
  });
}
template <typename R>
hmc_status cg_m_launch(hmc_ctx* c, const Geo& g, const V2<R>* u, const V2<R>* p, V2<R>* x,
                       V2<R>* r, CGScal* sc, unsigned* ticket) {
  return launch(c, sizeof(R) == 8 ? K_CG_M64 : K_CG_M32, [&] {
    launch_pdl(c, k_cg_m<R>, PDL(sizeof(R) == 8 ? K_CG_M64 : K_CG_M32, g.H), g, phase_of<R>(c), u, p, x, r,
               sc, c->partials, ticket);
  });
}
template <typename R>
hmc_status cg_p_launch(hmc_ctx* c, int N, const V2<R>* r, V2<R>* p, const CGScal* sc) {
  return launch(c, sizeof(R) == 8 ? K_CG_P64 : K_CG_P32,
                [&] { launch_pdl(c, k_cg_p<R>, PDL(sizeof(R) == 8 ? K_CG_P64 : K_CG_P32, N), N, r, p, sc); });
}
template <typename R>
hmc_status resid_launch(hmc_ctx* c, const Geo& g, R dm, const V2<R>* u, const V2<R>* x,
                        const V2<R>* b, double sigma, V2<R>* r, V2<R>* p, CGScal* init,
                        double tol2, int maxit, double* out2, unsigned* ticket, double ddm) {
  return launch(c, sizeof(R) == 8 ? K_RESID64 : K_RESID32, [&] {
    k_resid<R><<<GRID(g.H)>>>(g, phase_of<R>(c), dm, u, x, b, (R)sigma, r, p, init, tol2, maxit,
                              sigma, ddm, out2, c->partials, ticket);
  });
}
template <typename R>
hmc_status init0_launch(hmc_ctx* c, int N, const V2<R>* b, V2<R>* x, V2<R>* r, V2<R>* p, CGScal* sc,
                        double tol2, int maxit, double sigma, unsigned* ticket, double ddm) {
  return launch(c, K_INIT0, [&] {
    k_init0<R><<<GRID(N)>>>(N, b, x, r, p, sc, tol2, maxit, sigma, ddm, c->partials, ticket);
  });
}

#define INST(R)                                                                                   \
  template hmc_status mdag_launch<R>(hmc_ctx*, const Geo&, R, const V2<R>*, V2<R>*);             \
  template hmc_status m_launch<R>(hmc_ctx*, const Geo&, R, const V2<R>*, const V2<R>*, R,        \
                                  V2<R>*);                                                        \
  template hmc_status cg_mdag_launch<R>(hmc_ctx*, const Geo&, const V2<R>*, V2<R>*, CGScal*,     \
                                        unsigned*);                                               \
  template hmc_status cg_m_launch<R>(hmc_ctx*, const Geo&, const V2<R>*, const V2<R>*,           \
                                     V2<R>*, V2<R>*, CGScal*, unsigned*);                         \
  template hmc_status cg_p_launch<R>(hmc_ctx*, int, const V2<R>*, V2<R>*, const CGScal*);        \
  template hmc_status resid_launch<R>(hmc_ctx*, const Geo&, R, const V2<R>*, const V2<R>*,       \
                                      const V2<R>*, double, V2<R>*, V2<R>*, CGScal*, double, int, \
                                      double*, unsigned*, double);                                \
  template hmc_status init0_launch<R>(hmc_ctx*, int, const V2<R>*, V2<R>*, V2<R>*, V2<R>*,       \
                                      CGScal*, double, int, double, unsigned*, double);
INST(float)
INST(double)
#undef INST

// Condition of the device-side CG loop: continue while the solve runs and the
// trip count is below its bound (trips[1], so the loop ends even if the done
// flag were never set).
__global__ void k_loop_continue(cudaGraphConditionalHandle h, const CGScal* sc, unsigned* trips) {
  if (threadIdx.x == 0) {
    const unsigned t = trips[0] + 1u;
    trips[0] = t;
    cudaGraphSetConditional(h, (sc->done == CG_RUNNING && t < trips[1]) ? 1u : 0u);
  }
}

hmc_status loop_continue_launch(hmc_ctx* c, cudaGraphConditionalHandle h, const CGScal* sc) {
  k_loop_continue<<<1, 32, 0, c->stream>>>(h, sc, c->loop_trips);
  const cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? HMC_OK : cuda_fail(c, e, "loop condition");
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

hmc_status cg32_pmdag_launch(hmc_ctx* c, const Geo& g, const float2* r, const float2* pold,
                             float2* pnew, float2* u, CGScal* sc, unsigned* ticket) {
  (void)ticket;
  const int GB = shape_grid(c, K_CG_M32, g.H);
  const Shape& sh = c->shape[K_CG_MDAG32];
  if (sh.tiled == 1 && !cg32_tiled_ok(c, g, sh.threads, sh.tt)) return fail(c, HMC_ERR_INVALID, "tiled CG shape does not fit");
  if (sh.tiled == 2 && !cg32_march_ok(c, g, sh.threads, sh.tt)) return fail(c, HMC_ERR_INVALID, "CG shape does not fit");
  return launch_b(c, K_CG_MDAG32, 36.0 * g.N, [&] {
    if (sh.tiled == 2) {
      const dim3 grid((g.V + sh.threads - 1) / sh.threads, (g.nt + sh.tt - 1) / sh.tt);
      launch_pdl(c, k_cg32_pmdag_march, grid, sh.threads, c->stream, g, phase_of<float>(c), sh.tt, r, pold, pnew,
                 u, sc, (const float2*)c->partB, GB, (float2*)c->partA);
    } else if (sh.tiled) {
      const dim3 grid((g.V + sh.threads - 1) / sh.threads, (g.nt + sh.tt - 1) / sh.tt);
      const float2* pb = (const float2*)c->partB;
      float2* pa = (float2*)c->partA;
      switch (sh.threads) {
        case 256: launch_pdl(c, k_cg32_pmdag_tiled<256>, grid, 256, c->stream, g, phase_of<float>(c), sh.tt, r, pold, pnew, u, sc, pb, GB, pa); break;
        case 512: launch_pdl(c, k_cg32_pmdag_tiled<512>, grid, 512, c->stream, g, phase_of<float>(c), sh.tt, r, pold, pnew, u, sc, pb, GB, pa); break;
        default: launch_pdl(c, k_cg32_pmdag_tiled<1024>, grid, 1024, c->stream, g, phase_of<float>(c), sh.tt, r, pold, pnew, u, sc, pb, GB, pa); break;
      }
    } else {
      launch_pdl(c, k_cg32_pmdag, dim3(shape_grid(c, K_CG_MDAG32, g.H)), sh.threads, c->stream, g,
                 phase_of<float>(c), r, pold, pnew, u, sc, (const float2*)c->partB, GB, (float2*)c->partA);
    }
  });
}
hmc_status cg32_m_launch(hmc_ctx* c, const Geo& g, const float2* u, const float2* p, float2* x,
                         float2* r, CGScal* sc, unsigned* ticket) {
  (void)ticket;
  const int GA = shape_grid(c, K_CG_MDAG32, g.H);
  const Shape& sh = c->shape[K_CG_M32];
  if (sh.tiled == 1 && !cg32_tiled_ok(c, g, sh.threads, sh.tt)) return fail(c, HMC_ERR_INVALID, "tiled CG shape does not fit");
  if (sh.tiled == 2 && !cg32_march_ok(c, g, sh.threads, sh.tt)) return fail(c, HMC_ERR_INVALID, "CG shape does not fit");
  return launch_b(c, K_CG_M32, 52.0 * g.N, [&] {
    if (sh.tiled == 2) {
      const dim3 grid((g.V + sh.threads - 1) / sh.threads, (g.nt + sh.tt - 1) / sh.tt);
      launch_pdl(c, k_cg32_m_march, grid, sh.threads, c->stream, g, phase_of<float>(c), sh.tt, u, p, x, r, sc,
                 (const float2*)c->partA, GA, (float2*)c->partB);
    } else if (sh.tiled) {
      const dim3 grid((g.V + sh.threads - 1) / sh.threads, (g.nt + sh.tt - 1) / sh.tt);
      const float2* pa = (const float2*)c->partA;
      float2* pb = (float2*)c->partB;
      switch (sh.threads) {
        case 256: launch_pdl(c, k_cg32_m_tiled<256>, grid, 256, c->stream, g, phase_of<float>(c), sh.tt, u, p, x, r, sc, pa, GA, pb); break;
        case 512: launch_pdl(c, k_cg32_m_tiled<512>, grid, 512, c->stream, g, phase_of<float>(c), sh.tt, u, p, x, r, sc, pa, GA, pb); break;
        default: launch_pdl(c, k_cg32_m_tiled<1024>, grid, 1024, c->stream, g, phase_of<float>(c), sh.tt, u, p, x, r, sc, pa, GA, pb); break;
      }
    } else {
      launch_pdl(c, k_cg32_m, dim3(shape_grid(c, K_CG_M32, g.H)), sh.threads, c->stream, g, phase_of<float>(c),
                 u, p, x, r, sc, (const float2*)c->partA, GA, (float2*)c->partB);
    }
  });
}

int cg_kernel_occupancy(int id, int threads) {
  int nb = 0;
  const void* f = nullptr;
  switch (id) {
    case K_CG_MDAG64: f = (const void*)k_cg_mdag<double>; break;
    case K_CG_M64: f = (const void*)k_cg_m<double>; break;
    case K_CG_P64: f = (const void*)k_cg_p<double>; break;
    case K_CG_MDAG32: f = (const void*)k_cg32_pmdag; break;
    case K_CG_M32: f = (const void*)k_cg32_m; break;
    default: return 1;
  }
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, f, threads, 0) != cudaSuccess) {
    cudaGetLastError();
    return 1;
  }
  return nb > 0 ? nb : 1;
}

hmc_status to32_launch(hmc_ctx* c, int N, const double2* in, float2* out) {
  return launch(c, K_CONVERT, [&] { k_to32<<<GRID(N)>>>(N, in, out); });
}
hmc_status to64_launch(hmc_ctx* c, int N, const float2* in, double2* out) {
  return launch(c, K_CONVERT, [&] { k_to64<<<GRID(N)>>>(N, in, out); });
}
hmc_status norm2_launch(hmc_ctx* c, int N, const double2* v, double* out, unsigned* ticket) {
  return launch(c, K_NORM, [&] { k_norm2<<<GRID(N)>>>(N, v, out, c->partials, ticket); });
}
hmc_status redot_launch(hmc_ctx* c, int N, const double2* u, const double2* v, double* out,
                        unsigned* ticket) {
  return launch(c, K_NORM, [&] { k_redot<<<GRID(N)>>>(N, u, v, out, c->partials, ticket); });
}
#define NV_CASES(X) X(1) X(2) X(3) X(4) X(5) X(6) X(7) X(8) X(9) X(10) X(11) X(12) X(13) X(14) X(15) X(16)

hmc_status mdot_launch(hmc_ctx* c, int N, VecList V, int nv, const double2* w, double* hout,
                       unsigned* ticket) {
  if (nv < 1 || nv > kMaxRestart) return fail(c, HMC_ERR_INVALID, "basis size out of range");
  return launch_b(c, K_MDOT, 16.0 * N * (nv + 1), [&] {
    switch (nv) {
#define X(n) \
  case n: k_mdot<n><<<GRID(N)>>>(N, V, w, hout, c->partials, ticket); break;
      NV_CASES(X)
#undef X
    }
  });
}
hmc_status gsupd_launch(hmc_ctx* c, int N, VecList V, int nv, const double* h, double2* w,
                        double* ww, unsigned* ticket) {
  if (nv < 1 || nv > kMaxRestart) return fail(c, HMC_ERR_INVALID, "basis size out of range");
  return launch_b(c, K_GSUPD, 16.0 * N * (nv + 2), [&] {
    switch (nv) {
#define X(n) \
  case n: k_gsupd<n><<<GRID(N)>>>(N, V, h, w, ww, c->partials, ticket); break;
      NV_CASES(X)
#undef X
    }
  });
}
hmc_status scale_launch(hmc_ctx* c, int N, double s, const double2* w, double2* v, float2* v32) {
  return launch(c, K_SCALE, [&] { k_scale<<<GRID(N)>>>(N, s, w, v, v32); });
}
hmc_status xupd_launch(hmc_ctx* c, int N, VecList Z, CoefList y, int nz, double2* x) {
  return launch_b(c, K_XUPD, 16.0 * N * (nz + 2), [&] { k_xupd<<<GRID(N)>>>(N, Z, y, nz, x); });
}
hmc_status axpy_real_launch(hmc_ctx* c, int N, double a, const double* x, double* y) {
  return launch(c, K_AXPY, [&] { k_axpy_real<<<GRID(N)>>>(N, a, x, y); });
}
hmc_status axpby_c_launch(hmc_ctx* c, int N, double a, const double2* x, double b, double2* y) {
  return launch(c, K_AXPY, [&] { k_axpby_c<<<GRID(N)>>>(N, a, x, b, y); });
}
hmc_status force_launch(hmc_ctx* c, const Geo& g, const double2* eta, const double2* xi,
                        const double2* chi, double* grad) {
  return launch(c, K_FORCE,
                [&] { k_force<<<GRID(g.H)>>>(g, phase_of<double>(c), eta, xi, chi, grad); });
}
hmc_status gauss_grad_launch(hmc_ctx* c, int N, const double* phi, double inv_dU, int accumulate,
                             double* grad) {
  return launch(c, K_MD, [&] { k_gauss_grad<<<GRID(N)>>>(N, phi, inv_dU, accumulate, grad); });
}
hmc_status half_sq_launch(hmc_ctx* c, int N, const double* a, double sa, const double* b, double* out,
                          unsigned* ticket) {
  return launch(c, K_NORM,
                [&] { k_half_sq<<<GRID(N)>>>(N, a, sa, b, out, c->partials, ticket); });
}

}  // namespace hmc
