// The libhmc kernels: operator applications, fused CG iterations (the
// grid-stride FP32 pair; the other FP32 designs are in cg32_designs.cu),
// residuals, FGMRES vector operations and the pseudofermion force.
// Passages: the operator of Eq. ferm_op (Section 2), CG (Section 3), the vector
// steps of Algorithm A.1 (Appendix A), the force of Eqs. p_dot, f_chi_i and
// def_xi_i, the energies of Eq. hamiltonian.
#include "kernels.h"
#include "launch.cuh"
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
    "batch_init",     "batch_residual", "batch_misc",   "cg_persist_f32", "mmdag_fused_f32",
    "mmdag_fused_f64", "cg1_fused_f32",  "cg_resident_f32"};

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
    0,                   // persistent CG: 96 B per site and iteration, counted after the solve
    8 + 4 + 8,           // fused M M^dagger f32: p, phi32, out (u stays on chip)
    16 + 16 + 16,        // fused M M^dagger f64: p, E, out
    5 * 8 + 4 + 5 * 8,   // single-reduction CG f32: r, w, s, p, x, phi32 in; r, w, s, p, x out
    0};                  // resident CG: 96 B per site and iteration, counted after the solve

// ---------------------------------------------------------------------------
// e^{i phi} for the FP64 stencils of Eq. ferm_op, and phi rounded to float.
__global__ void __launch_bounds__(kThreads) k_phase(int N, const double* __restrict__ phi,
                                                    double2* __restrict__ E,
                                                    float* __restrict__ phi32) {
  for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < N; k += gridDim.x * blockDim.x) {
    double s, co;
    double x = phi[k];
    sincos(x, &s, &co);
    E[k] = make_double2(co, s);
    phi32[k] = phi_to_f32(x);
  }
}


// out = M^dagger p (Eq. ferm_op, conjugate transpose), one cell-time per thread.
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

// out = M u (Eq. ferm_op), one cell-time per thread.
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

// FP64 CG (Section 3), first kernel of an iteration:
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

// FP64 CG (Section 3), second kernel of an iteration:
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

// p = r + beta p, the last step of a CG iteration (Section 3).
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
// The single-precision CG of Section 3 (the inner solver of Algorithm A.1) as
// a pair of kernels per iteration.
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
    float b;
    s_done = cg32_scalars_first(sc, first, rr_pair, blockIdx.x == 0, &b);
    s_beta = b;
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
    float a;
    s_bad = cg32_scalars_second(sc, pAp_pair, blockIdx.x == 0, &a);
    s_alpha = a;
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
// The same FP32 CG pair with two cells per thread (n even). A work item is the
// pair of cells (i, i+1), i even, of one row and time slice: its complex64
// values are one 16-byte float4 in each vector, and so are the values of its
// time partners and of its j-neighbours. The i-neighbour inside the pair is
// the other half of the thread's own float4; only the one across the pair
// boundary (i-1 for the A rows, i+2 for the B rows) is an 8-byte load. The
// rows of Eq. ferm_op are formed in the same order as in mdag_pair / m_pair,
// so the results equal those of the one-cell kernels.
struct Nbr2 {
  int q;         // even cell-time index of the pair's first cell (A site)
  int tm, tp;    // the pair at t-1, t+1 (wrapped)
  int jm1, jp1;  // the pair at j-1, j+1 (wrapped)
  int im1;       // the single cell (i-1, j) of the first cell
  int ip1;       // the single cell (i+2, j) beyond the second cell
  bool wrap_tm, wrap_tp;
};

__device__ __forceinline__ Nbr2 neighbours2(const Geo& g, int q2) {
  Nbr2 b;
  const int q = 2 * q2;
  b.q = q;
  const int t = (int)fdiv((uint32_t)q, g.fV);
  const int c = q - t * g.V;
  const int j = (int)fdiv((uint32_t)c, g.fn);
  const int i = c - j * g.n;
  b.wrap_tm = (t == 0);
  b.wrap_tp = (t == g.nt - 1);
  b.tm = q - g.V + (b.wrap_tm ? g.H : 0);
  b.tp = q + g.V - (b.wrap_tp ? g.H : 0);
  b.im1 = q - 1 + (i == 0 ? g.n : 0);
  b.ip1 = q + 2 - (i + 2 == g.n ? g.n : 0);
  b.jm1 = q - g.n + (j == 0 ? g.V : 0);
  b.jp1 = q + g.n - (j == g.m - 1 ? g.V : 0);
  return b;
}

__device__ __forceinline__ Cx<float> lo2(const float4& v) { return Cx<float>{v.x, v.y}; }
__device__ __forceinline__ Cx<float> hi2(const float4& v) { return Cx<float>{v.z, v.w}; }
__device__ __forceinline__ float4 cat2(Cx<float> a, Cx<float> b) { return make_float4(a.re, a.im, b.re, b.im); }
__device__ __forceinline__ float4 axpy4(float a, float4 x, float4 y) {
  return make_float4(fmaf(a, x.x, y.x), fmaf(a, x.y, y.y), fmaf(a, x.z, y.z), fmaf(a, x.w, y.w));
}
__device__ __forceinline__ float norm4(float4 v) { return v.x * v.x + v.y * v.y + v.z * v.z + v.w * v.w; }

// e^{i phi} of the two cells of the pair at k (phi as float pairs, in [-pi, pi]).
__device__ __forceinline__ void phase2(const float* phi32, int k, Cx<float>& e0, Cx<float>& e1) {
  const float2 f = *reinterpret_cast<const float2*>(phi32 + k);
  float s0, c0, s1, c1;
  __sincosf(f.x, &s0, &c0);
  __sincosf(f.y, &s1, &c1);
  e0 = Cx<float>{c0, s0};
  e1 = Cx<float>{c1, s1};
}

// Time-hop factors of M^dagger at the pair: A rows (hop to t+1, phase of A at
// t+1, conjugated), B rows (hop to t-1, phase of B at t-1).
__device__ __forceinline__ void mdag_factors2(const float* phi32, const Nbr2& nb, int H, float dm, Cx<float> (&za)[2],
                                              Cx<float> (&zb)[2]) {
  Cx<float> ea0, ea1, eb0, eb1;
  phase2(phi32, nb.tp, ea0, ea1);
  phase2(phi32, H + nb.tm, eb0, eb1);
  za[0] = cneg_if(Cx<float>{ea0.re - dm, -ea0.im}, nb.wrap_tp);
  za[1] = cneg_if(Cx<float>{ea1.re - dm, -ea1.im}, nb.wrap_tp);
  zb[0] = cneg_if(Cx<float>{dm - eb0.re, -eb0.im}, nb.wrap_tm);
  zb[1] = cneg_if(Cx<float>{dm - eb1.re, -eb1.im}, nb.wrap_tm);
}

// M^dagger of the vector returned by L4 (float4 pairs at even indices) and
// L1 (single cells), at the pair nb: the A pair into oA, the B pair into oB.
template <typename L4, typename L1>
__device__ __forceinline__ void mdag2(int H, const Cx<float> (&za)[2], const Cx<float> (&zb)[2], float dk,
                                      const Nbr2& nb, L4 ld4, L1 ld1, float4& oA, float4& oB) {
  const float4 pa = ld4(nb.q), pb = ld4(H + nb.q);
  const float4 pat = ld4(nb.tp), pbt = ld4(H + nb.tm);
  const float4 pbj = ld4(H + nb.jm1), paj = ld4(nb.jp1);
  const Cx<float> pbi = ld1(H + nb.im1), pai = ld1(nb.ip1);
  const Cx<float> a0 = hopsum(cfma(za[0], lo2(pat), Cx<float>{-pa.x, -pa.y}), dk, lo2(pb), pbi, lo2(pbj));
  const Cx<float> a1 = hopsum(cfma(za[1], hi2(pat), Cx<float>{-pa.z, -pa.w}), dk, hi2(pb), lo2(pb), hi2(pbj));
  const Cx<float> b0 = hopsum(cfma(zb[0], lo2(pbt), lo2(pb)), dk, lo2(pa), hi2(pa), lo2(paj));
  const Cx<float> b1 = hopsum(cfma(zb[1], hi2(pbt), hi2(pb)), dk, hi2(pa), pai, hi2(paj));
  oA = cat2(a0, a1);
  oB = cat2(b0, b1);
}

// M u at the pair nb (phases of the pair's own cells).
__device__ __forceinline__ void m2(const Geo& g, const float* phi32, float dm, const Nbr2& nb,
                                   const float4* __restrict__ u, float4& oA, float4& oB) {
  const int H = g.H;
  const float dk = g.dkf;
  const float2* u2 = reinterpret_cast<const float2*>(u);
  const float4 ua = u[nb.q >> 1], ub = u[(H + nb.q) >> 1];
  const float4 uat = u[nb.tm >> 1], ubt = u[(H + nb.tp) >> 1];
  const float4 ubj = u[(H + nb.jm1) >> 1], uaj = u[nb.jp1 >> 1];
  const float2 ubi2 = u2[H + nb.im1], uai2 = u2[nb.ip1];
  Cx<float> ea0, ea1, eb0, eb1;
  phase2(phi32, nb.q, ea0, ea1);
  phase2(phi32, H + nb.q, eb0, eb1);
  const Cx<float> za0 = cneg_if(Cx<float>{ea0.re - dm, ea0.im}, nb.wrap_tm);
  const Cx<float> za1 = cneg_if(Cx<float>{ea1.re - dm, ea1.im}, nb.wrap_tm);
  const Cx<float> zb0 = cneg_if(Cx<float>{dm - eb0.re, eb0.im}, nb.wrap_tp);
  const Cx<float> zb1 = cneg_if(Cx<float>{dm - eb1.re, eb1.im}, nb.wrap_tp);
  const Cx<float> a0 =
      hopsum(cfma(za0, lo2(uat), Cx<float>{-ua.x, -ua.y}), dk, lo2(ub), Cx<float>{ubi2.x, ubi2.y}, lo2(ubj));
  const Cx<float> a1 = hopsum(cfma(za1, hi2(uat), Cx<float>{-ua.z, -ua.w}), dk, hi2(ub), lo2(ub), hi2(ubj));
  const Cx<float> b0 = hopsum(cfma(zb0, lo2(ubt), lo2(ub)), dk, lo2(ua), hi2(ua), lo2(uaj));
  const Cx<float> b1 = hopsum(cfma(zb1, hi2(ubt), hi2(ub)), dk, hi2(ua), Cx<float>{uai2.x, uai2.y}, hi2(uaj));
  oA = cat2(a0, a1);
  oB = cat2(b0, b1);
}

__global__ void __launch_bounds__(kMaxThreads) k_cg32_pmdag2(Geo g, const float* __restrict__ phi32,
                                                          const float4* __restrict__ r,
                                                          const float4* __restrict__ pold,
                                                          float4* __restrict__ pnew, float4* __restrict__ u,
                                                          CGScal* sc, const float2* __restrict__ partB, int GB,
                                                          float2* __restrict__ partA) {
  __shared__ float s_beta;
  __shared__ int s_exit, s_done;
  pdl_wait();
  if (threadIdx.x == 0) s_exit = sc->done;
  __syncthreads();
  if (s_exit) return;
  const int first = sc->first;
  const float dm = sc->dm32, sigma = sc->sigma32, dk = g.dkf;
  const int H = g.H, H2 = g.H >> 1, Hh = g.H >> 1;
  const int stride = gridDim.x * blockDim.x;
  const float2* r1 = reinterpret_cast<const float2*>(r);
  const float2* po1 = reinterpret_cast<const float2*>(pold);
  int q2 = blockIdx.x * blockDim.x + threadIdx.x;
  // first item: both stencils, before beta is known
  const bool have0 = q2 < H2;
  Nbr2 nb0;
  float4 mrA{}, mrB{}, mpA{}, mpB{}, r0a{}, r0b{}, p0a{}, p0b{};
  if (have0) {
    nb0 = neighbours2(g, q2);
    Cx<float> za[2], zb[2];
    mdag_factors2(phi32, nb0, H, dm, za, zb);
    mdag2(H, za, zb, dk, nb0, [&](int k) { return r[k >> 1]; },
          [&](int k) { const float2 v = r1[k]; return Cx<float>{v.x, v.y}; }, mrA, mrB);
    r0a = r[q2];
    r0b = r[Hh + q2];
    if (!first) {
      mdag2(H, za, zb, dk, nb0, [&](int k) { return pold[k >> 1]; },
            [&](int k) { const float2 v = po1[k]; return Cx<float>{v.x, v.y}; }, mpA, mpB);
      p0a = pold[q2];
      p0b = pold[Hh + q2];
    }
  }
  const float2 rr_pair = first ? make_float2(0.f, 0.f) : ff_sum_partials(partB, GB);
  if (threadIdx.x == 0) {
    float b;
    s_done = cg32_scalars_first(sc, first, rr_pair, blockIdx.x == 0, &b);
    s_beta = b;
  }
  __syncthreads();
  if (s_done) return;
  const float beta = s_beta;
  float loc = 0.f;
  if (have0) {
    const float4 pa = axpy4(beta, p0a, r0a), pb = axpy4(beta, p0b, r0b);
    const float4 oa = axpy4(beta, mpA, mrA), ob = axpy4(beta, mpB, mrB);
    pnew[q2] = pa;
    pnew[Hh + q2] = pb;
    u[q2] = oa;
    u[Hh + q2] = ob;
    loc += norm4(oa) + norm4(ob);
    if (sigma != 0.f) loc += sigma * (norm4(pa) + norm4(pb));
  }
  for (q2 += stride; q2 < H2; q2 += stride) {
    const Nbr2 nb = neighbours2(g, q2);
    auto P4 = [&](int k) { return axpy4(beta, pold[k >> 1], r[k >> 1]); };
    auto P1 = [&](int k) {
      const float2 a = r1[k], b = po1[k];
      return Cx<float>{fmaf(beta, b.x, a.x), fmaf(beta, b.y, a.y)};
    };
    Cx<float> za[2], zb[2];
    mdag_factors2(phi32, nb, H, dm, za, zb);
    float4 oa, ob;
    mdag2(H, za, zb, dk, nb, P4, P1, oa, ob);
    const float4 pa = P4(nb.q), pb = P4(H + nb.q);
    pnew[q2] = pa;
    pnew[Hh + q2] = pb;
    u[q2] = oa;
    u[Hh + q2] = ob;
    loc += norm4(oa) + norm4(ob);
    if (sigma != 0.f) loc += sigma * (norm4(pa) + norm4(pb));
  }
  pdl_trigger();
  ff_write_partial(loc, partA);
}

__global__ void __launch_bounds__(kMaxThreads) k_cg32_m2(Geo g, const float* __restrict__ phi32,
                                                      const float4* __restrict__ u, const float4* __restrict__ p,
                                                      float4* __restrict__ x, float4* __restrict__ r, CGScal* sc,
                                                      const float2* __restrict__ partA, int GA,
                                                      float2* __restrict__ partB) {
  __shared__ float s_alpha;
  __shared__ int s_exit, s_bad;
  pdl_wait();
  if (threadIdx.x == 0) s_exit = sc->done;
  __syncthreads();
  if (s_exit) return;
  const float dm = sc->dm32, sigma = sc->sigma32;
  const int H2 = g.H >> 1, Hh = g.H >> 1;
  const int stride = gridDim.x * blockDim.x;
  int q2 = blockIdx.x * blockDim.x + threadIdx.x;
  const bool have0 = q2 < H2;
  float4 oA0{}, oB0{};
  if (have0) m2(g, phi32, dm, neighbours2(g, q2), u, oA0, oB0);
  const float2 pAp_pair = ff_sum_partials(partA, GA);
  if (threadIdx.x == 0) {
    float a;
    s_bad = cg32_scalars_second(sc, pAp_pair, blockIdx.x == 0, &a);
    s_alpha = a;
  }
  __syncthreads();
  if (s_bad) return;
  const float alpha = s_alpha;
  float loc = 0.f;
  auto update = [&](int k, float4 Ap) {
    const float4 pk = p[k];
    Ap = axpy4(sigma, pk, Ap);
    x[k] = axpy4(alpha, pk, x[k]);
    const float4 rk = axpy4(-alpha, Ap, r[k]);
    r[k] = rk;
    loc = fmaf(rk.x, rk.x, fmaf(rk.y, rk.y, loc));
    loc = fmaf(rk.z, rk.z, fmaf(rk.w, rk.w, loc));
  };
  if (have0) {
    update(q2, oA0);
    update(Hh + q2, oB0);
  }
  for (q2 += stride; q2 < H2; q2 += stride) {
    float4 oA, oB;
    m2(g, phi32, dm, neighbours2(g, q2), u, oA, oB);
    update(q2, oA);
    update(Hh + q2, oB);
  }
  pdl_trigger();
  ff_write_partial(loc, partB);
}

// True residual b - (M M^dagger + sigma) x and its norm in FP64 (Section 3;
// the restart step of Algorithm A.1).
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
      init->rr32 = init->rr_cur32 = (float)tot[0];
      init->thresh32 = (float)init->thresh;
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
    sc->rr32 = sc->rr_cur32 = (float)tot[0];
    sc->thresh32 = (float)sc->thresh;
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

// Arnoldi step of Algorithm A.1 (classical Gram-Schmidt in two passes):
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

// v_j = w / |w| (Algorithm A.1).
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

// x += sum_i y_i z_i, the update of Algorithm A.1 after the least-squares solve.
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

// The MD updates phi += c dt pi and pi -= d dt F (Sections 2, 4 and 5.2).
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

// Pseudofermion force (Eqs. p_dot, f_chi_i, def_xi_i):
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

// d/dphi of phi^2 / (2 delta U), the Gaussian term of Eq. hamiltonian.
__global__ void __launch_bounds__(kThreads) k_gauss_grad(int N, const double* __restrict__ phi,
                                                         double inv_dU, int accumulate,
                                                         double* __restrict__ grad) {
  for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < N; k += gridDim.x * blockDim.x) {
    double v = phi[k] * inv_dU;
    grad[k] = accumulate ? grad[k] + v : v;
  }
}

// Sums of squares for the kinetic and Gaussian terms of H (Eq. hamiltonian).
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

hmc_status cg32_pmdag_launch(hmc_ctx* c, const Geo& g, const float2* r, const float2* pold,
                             float2* pnew, float2* u, CGScal* sc, unsigned* ticket) {
  (void)ticket;
  const int GB = shape_grid(c, K_CG_M32, g.H);
  const Shape& sh = c->shape[K_CG_MDAG32];
  if (sh.tiled == 1 && !cg32_tiled_ok(c, g, sh.threads, sh.tt)) return fail(c, HMC_ERR_INVALID, "tiled CG shape does not fit");
  if (sh.tiled == 2 && !cg32_march_ok(c, g, sh.threads, sh.tt)) return fail(c, HMC_ERR_INVALID, "CG shape does not fit");
  return launch_b(c, K_CG_MDAG32, 36.0 * g.N, [&] {
    if (sh.tiled == 4) {
      launch_pdl(c, k_cg32_pmdag2, dim3(shape_grid(c, K_CG_MDAG32, g.H)), sh.threads, c->stream, g,
                 (const float*)c->ws[WS_PHI32], (const float4*)r, (const float4*)pold, (float4*)pnew, (float4*)u, sc,
                 (const float2*)c->partB, GB, (float2*)c->partA);
    } else if (sh.tiled) {
      cg32_alt_pmdag(c, g, sh, r, pold, pnew, u, sc, GB);
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
    if (sh.tiled == 4) {
      launch_pdl(c, k_cg32_m2, dim3(shape_grid(c, K_CG_M32, g.H)), sh.threads, c->stream, g,
                 (const float*)c->ws[WS_PHI32], (const float4*)u, (const float4*)p, (float4*)x, (float4*)r, sc,
                 (const float2*)c->partA, GA, (float2*)c->partB);
    } else if (sh.tiled) {
      cg32_alt_m(c, g, sh, u, p, x, r, sc, GA);
    } else {
      launch_pdl(c, k_cg32_m, dim3(shape_grid(c, K_CG_M32, g.H)), sh.threads, c->stream, g, phase_of<float>(c),
                 u, p, x, r, sc, (const float2*)c->partA, GA, (float2*)c->partB);
    }
  });
}

int cg_kernel_occupancy(int id, int threads, int pairs) {
  int nb = 0;
  const void* f = nullptr;
  if (pairs && id == K_CG_MDAG32) f = (const void*)k_cg32_pmdag2;
  if (pairs && id == K_CG_M32) f = (const void*)k_cg32_m2;
  if (f == nullptr) switch (id) {
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
