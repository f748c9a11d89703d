// FP32 CG with the direction p and the intermediate u = M^dagger p resident
// in shared memory for the whole solve (the inner solver of Section 3 and
// Algorithm A.1; the same CG step as the two-kernel pair). One cooperative
// launch per solve; every block owns a tile of cells -- all n cells of a row
// i, Jt rows j, Tt time slices -- and keeps p_A, p_B, u_A, u_B of the tile in
// shared memory, each array padded by the one row and the one time slice of
// neighbouring tiles its stencil reads (Eq. ferm_op: the A rows of M^dagger
// read p_B at (i, j), (i-1, j), (i, j-1) and p_A at t+1; the B rows read p_A
// at (i, j), (i+1, j), (i, j+1) and p_B at t-1; M reads u the same way with
// the time hops reversed). With all of i in the tile, the i-neighbours wrap
// inside it.
//
// Iteration (scalars held by thread 0 of every block in FP64, partials summed
// by every block in the same fixed order):
//   first half:  p = r + beta p on the tile (in place) and on the padding
//                (from r and the previous p of the neighbouring tiles, which
//                their owners publish); u = M^dagger p on the tile; the
//                tile's edge rows and slices of u published; partial of
//                |u|^2 + sigma |p|^2;                      -- grid barrier --
//   second half: alpha = |r|^2 / <p, A p>; the padding of u read from the
//                neighbours' published edges; A p = M u + sigma p, r -= alpha
//                A p on the tile (x and r stay in memory, read and written by
//                their owner only); partial of |r|^2. x += alpha p waits for
//                the next first half, where it joins the loads of r (and for
//                the exit, after the last iteration).
//                                                          -- grid barrier --
// The padding slices that lie beyond t = nt - 1 or before t = 0 hold the
// anti-periodic continuation (negated values), so the time hops carry no
// sign of their own, as in the fused M M^dagger kernel. Published p edges
// alternate between two buffers by iteration parity (a tile reads the
// previous iteration's edges while its neighbours write the current ones);
// published u edges are written before the first barrier and read after it.
// Data other blocks wrote is read with L2-only loads (L1 is not coherent
// across SMs). The barrier waits are bounded: a wait that gives up marks the
// solve CG_TIMEOUT and every block leaves.
#include <algorithm>
#include <cstdint>

#include "kernels.h"
#include "launch.cuh"
#include "operator.cuh"

namespace hmc {

// Tile of the resident kernel: J rows, T slices (nominal; the last tile in
// each direction may be smaller), the number of tiles, and the rows of the
// tile a block works on at once (threads = n x rows).
struct ResTile {
  int J = 0, T = 0, tiles_j = 0, tiles_t = 0, rows = 0;
};

constexpr int kResMaxThreads = 1024;
// at most this many tiles (one block each): the partial sums below load up to
// kResMaxTiles / 32 partials per lane of warp 0
constexpr int kResMaxTiles = 256;

// Sum of G <= kResMaxTiles float-float partials by warp 0 alone, in a fixed
// order; valid in thread 0. Every lane issues all of its loads before the
// first addition, and no block-wide barrier is needed: the other warps go on
// to the next phase's loads meanwhile.
__device__ __forceinline__ float2 ff_warp0_sum(const float2* __restrict__ part, int G) {
  constexpr int L = kResMaxTiles / 32;
  float2 w[L];
#pragma unroll
  for (int j = 0; j < L; ++j) {
    const int b = threadIdx.x + 32 * j;
    w[j] = b < G ? __ldcg(part + b) : make_float2(0.f, 0.f);
  }
  float2 v = w[0];
#pragma unroll
  for (int j = 1; j < L; ++j) v = ff_add(v, w[j]);
#pragma unroll
  for (int o = 16; o > 0; o >>= 1)
    v = ff_add(v, make_float2(__shfl_xor_sync(0xffffffffu, v.x, o), __shfl_xor_sync(0xffffffffu, v.y, o)));
  return v;
}

__global__ void __launch_bounds__(kResMaxThreads, 1)
    k_cg32_resident(Geo g, ResTile rt, Phase<float> ph, float2* __restrict__ x, float2* __restrict__ r,
                    float2* __restrict__ P0, float2* __restrict__ P1, float2* __restrict__ U, CGScal* sc,
                    float2* __restrict__ partA, float2* __restrict__ partB, GridBar* gb, long long limit,
                    unsigned expect) {
  extern __shared__ float2 s_tile[];
  __shared__ float s_a, s_ap;
  __shared__ int s_stop;
  const int n = g.n, m = g.m, nt = g.nt, H = g.H;
  const int bj = blockIdx.x % rt.tiles_j, bt = blockIdx.x / rt.tiles_j;
  const int j0 = bj * rt.J, t0 = bt * rt.T;
  const int Jt = min(rt.J, m - j0), Tt = min(rt.T, nt - t0);
  const int J1 = rt.J + 1;
  const int SZ = (rt.T + 1) * J1 * n;  // one padded array
  float2* pA = s_tile;                 // rows 0..Jt (Jt: the row above), slices 0..Tt (Tt: the slice after)
  float2* pB = pA + SZ;                // rows -1..Jt-1, slices -1..Tt-1 (stored at +1)
  float2* uA = pB + SZ;                // rows 0..Jt, slices -1..Tt-1
  float2* uB = uA + SZ;                // rows -1..Jt-1, slices 0..Tt
  auto iPA = [&](int i, int jj, int tt) { return (tt * J1 + jj) * n + i; };
  auto iPB = [&](int i, int jj, int tt) { return ((tt + 1) * J1 + jj + 1) * n + i; };
  auto iUA = [&](int i, int jj, int tt) { return ((tt + 1) * J1 + jj) * n + i; };
  auto iUB = [&](int i, int jj, int tt) { return (tt * J1 + jj + 1) * n + i; };
  // the thread's cell column i and its first row of the tile
  const int i = threadIdx.x % n, r0 = threadIdx.x / n, RS = rt.rows;
  const bool act = r0 < RS;
  const int im = i == 0 ? n - 1 : i - 1, ip = i == n - 1 ? 0 : i + 1;
  const int rows = Jt * Tt, lines = 2 * Tt + 2 * Jt;
  const int jdn = (j0 - 1 + m) % m, jup = (j0 + Jt) % m;  // the rows below and above the tile
  const bool wlo = (t0 == 0), whi = (t0 + Tt == nt);      // padding slices across the time boundary
  const int tdn = wlo ? nt - 1 : t0 - 1, tup = whi ? 0 : t0 + Tt;
  auto cell = [&](int j, int t) { return (t * m + j) * n + i; };
  // The thread's rows R = r0, r0 + RS, ... of the tile as (jj, tt), advanced
  // without division. Within a row every shared-memory index is the row's
  // base b = (tt (J + 1) + jj) n + i plus a constant (NJ: one padded slice):
  //   p_A(jj, tt) = b, p_A(tt+1) = b + NJ, p_A(jj+1) = b + n,
  //   p_B(jj, tt) = b + NJ + n, p_B(jj-1) = b + NJ, p_B(tt-1) = b + n,
  //   u_A(jj, tt) = b + NJ, u_A(tt-1) = b, u_A(jj+1) = b + NJ + n,
  //   u_B(jj, tt) = b + n, u_B(jj-1) = b, u_B(tt+1) = b + NJ + n,
  // and the i-neighbours add dim = im - i or dip = ip - i.
  const int NJ = J1 * n, dim = im - i, dip = ip - i;
  const int V = g.V, kb = (t0 * m + j0) * n + i;  // lattice index of the tile's cell (i, 0, 0)
  const int dJ = RS % max(Jt, 1), dT = RS / max(Jt, 1);
  auto for_rows = [&](auto&& f) {
    int jj = r0 % Jt, tt = r0 / Jt;
    for (int R = r0; R < rows; R += RS) {
      f(jj, tt, (tt * J1 + jj) * n + i, kb + tt * V + jj * n);
      jj += dJ;
      tt += dT;
      if (jj >= Jt) {
        jj -= Jt;
        ++tt;
      }
    }
  };
  const float dm = sc->dm32, sigma = sc->sigma32, dk = g.dkf;
  // thread 0's scalars in FP32 (the FP64 pipe is slow on this GPU and every
  // other warp of the block waits for them); the partial sums stay float-float
  float rr = sc->rr32, rr_prev = 1.f, pAp = 0.f, alpha = 0.f, beta = 0.f;
  int iter = sc->iter, done = sc->done;
  const int maxit = sc->maxit;
  const float thresh = sc->thresh32;
  bool first = true;
  for (;;) {
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
      s_ap = alpha;  // the previous iteration's alpha: x += alpha p is applied here
      s_stop = done;
    }
    __syncthreads();
    const float fap = s_ap;
    if (s_stop) {
      // the last iteration's x update, still pending
      if (act && fap != 0.f)
        for_rows([&](int, int, int b, int k) {
          const float2 pa = pA[b], pb = pB[b + NJ + n];
          float2 xa = x[k], xb = x[H + k];
          x[k] = make_float2(fmaf(fap, pa.x, xa.x), fmaf(fap, pa.y, xa.y));
          x[H + k] = make_float2(fmaf(fap, pb.x, xb.x), fmaf(fap, pb.y, xb.y));
        });
      break;
    }
    const float fb = s_a;
    float2* Pcur = (iter & 1) ? P1 : P0;        // this iteration's published p edges
    const float2* Pold = (iter & 1) ? P0 : P1;  // the previous iteration's
    // ---- first half
    // padding of p: r + beta p_old of the neighbouring tiles' edge cells
    if (act) {
      // padding lines from the last row slot down: the slots that hold one row
      // fewer of the tile (rows are dealt from slot 0) take the extra lines
      for (int l = RS - 1 - r0; l < lines; l += RS) {
        int jj, tt, j, t, k;
        float s = 1.f;
        bool isA;
        if (l < Tt) {  // p_B, the row below
          jj = -1, tt = l, j = jdn, t = t0 + l, isA = false;
        } else if (l < 2 * Tt) {  // p_A, the row above
          jj = Jt, tt = l - Tt, j = jup, t = t0 + tt, isA = true;
        } else if (l < 2 * Tt + Jt) {  // p_B, the slice before
          jj = l - 2 * Tt, tt = -1, j = j0 + jj, t = tdn, isA = false, s = wlo ? -1.f : 1.f;
        } else {  // p_A, the slice after
          jj = l - 2 * Tt - Jt, tt = Tt, j = j0 + jj, t = tup, isA = true, s = whi ? -1.f : 1.f;
        }
        k = cell(j, t) + (isA ? 0 : H);
        float2 v = __ldcg(r + k);
        if (!first) {
          const float2 po = __ldcg(Pold + k);
          v = make_float2(fmaf(fb, po.x, v.x), fmaf(fb, po.y, v.y));
        }
        v = make_float2(s * v.x, s * v.y);
        if (isA)
          pA[iPA(i, jj, tt)] = v;
        else
          pB[iPB(i, jj, tt)] = v;
      }
      // the tile's own p, in place; its edges published for the neighbours
      for_rows([&](int jj, int tt, int b, int k) {
        const float2 ra = __ldcg(r + k), rb = __ldcg(r + H + k);
        if (fap != 0.f) {  // x += alpha p with the previous iteration's p, still in place
          const float2 pa = pA[b], pb = pB[b + NJ + n];
          const float2 xa = x[k], xb = x[H + k];
          x[k] = make_float2(fmaf(fap, pa.x, xa.x), fmaf(fap, pa.y, xa.y));
          x[H + k] = make_float2(fmaf(fap, pb.x, xb.x), fmaf(fap, pb.y, xb.y));
        }
        float2& qa = pA[b];
        float2& qb = pB[b + NJ + n];
        float2 a = ra, c = rb;
        if (!first) {
          a = make_float2(fmaf(fb, qa.x, ra.x), fmaf(fb, qa.y, ra.y));
          c = make_float2(fmaf(fb, qb.x, rb.x), fmaf(fb, qb.y, rb.y));
        }
        qa = a;
        qb = c;
        if (jj == 0 || tt == 0) Pcur[k] = a;
        if (jj == Jt - 1 || tt == Tt - 1) Pcur[H + k] = c;
      });
    }
    __syncthreads();
    // u = M^dagger p on the tile
    float loc = 0.f;
    if (act) {
      for_rows([&](int jj, int tt, int b, int k) {
        const int t = t0 + tt;
        const Cx<float> pa = ld<float>(pA, b), pb = ld<float>(pB, b + NJ + n);
        // A row: time partner p_A(t+1), phase of A at t+1 conjugated
        const Cx<float> ea = ph(t + 1 == nt ? k + V - H : k + V);
        const Cx<float> ua = hopsum(cfma(Cx<float>{ea.re - dm, -ea.im}, ld<float>(pA, b + NJ), Cx<float>{-pa.re, -pa.im}),
                                    dk, pb, ld<float>(pB, b + NJ + n + dim), ld<float>(pB, b + NJ));
        // B row: time partner p_B(t-1), phase of B at t-1
        const Cx<float> eb = ph(H + (t == 0 ? k - V + H : k - V));
        const Cx<float> ub = hopsum(cfma(Cx<float>{dm - eb.re, -eb.im}, ld<float>(pB, b + n), pb), dk, pa,
                                    ld<float>(pA, b + dip), ld<float>(pA, b + n));
        uA[b + NJ] = make_float2(ua.re, ua.im);
        uB[b + n] = make_float2(ub.re, ub.im);
        // edges the neighbours' M reads: u_A of the bottom row and the last
        // slice, u_B of the top row and the first slice
        if (jj == 0 || tt == Tt - 1) U[k] = make_float2(ua.re, ua.im);
        if (jj == Jt - 1 || tt == 0) U[H + k] = make_float2(ub.re, ub.im);
        loc += norm2(ua) + norm2(ub);
        if (sigma != 0.f) loc += sigma * (norm2(pa) + norm2(pb));
      });
    }
    {
      const float2 v = ff_block_sum(make_float2(loc, 0.f));
      if (threadIdx.x == 0) partA[blockIdx.x] = v;
    }
    if (!grid_barrier(gb, expect, limit)) {
      done = CG_TIMEOUT;
      break;
    }
    // ---- second half
    if (threadIdx.x < 32) {
      const float2 tot = ff_warp0_sum(partA, gridDim.x);
      if (threadIdx.x == 0) {
        pAp = tot.x + tot.y;
        const bool bad = !(pAp > 0.f) || !isfinite(pAp);
        alpha = bad ? 0.f : rr / pAp;
        if (bad) done = CG_BREAKDOWN;
        s_a = alpha;
        s_stop = bad;
      }
    }
    // padding of u from the neighbours' published edges
    if (act) {
      for (int l = r0; l < lines; l += RS) {
        int jj, tt, j, t;
        float s = 1.f;
        bool isA;
        if (l < Tt) {  // u_B, the row below
          jj = -1, tt = l, j = jdn, t = t0 + l, isA = false;
        } else if (l < 2 * Tt) {  // u_A, the row above
          jj = Jt, tt = l - Tt, j = jup, t = t0 + tt, isA = true;
        } else if (l < 2 * Tt + Jt) {  // u_A, the slice before
          jj = l - 2 * Tt, tt = -1, j = j0 + jj, t = tdn, isA = true, s = wlo ? -1.f : 1.f;
        } else {  // u_B, the slice after
          jj = l - 2 * Tt - Jt, tt = Tt, j = j0 + jj, t = tup, isA = false, s = whi ? -1.f : 1.f;
        }
        const float2 v = __ldcg(U + cell(j, t) + (isA ? 0 : H));
        if (isA)
          uA[iUA(i, jj, tt)] = make_float2(s * v.x, s * v.y);
        else
          uB[iUB(i, jj, tt)] = make_float2(s * v.x, s * v.y);
      }
    }
    __syncthreads();
    if (s_stop) break;
    const float fa = s_a;
    loc = 0.f;
    if (act) {
      for_rows([&](int, int, int b, int k) {
        const Cx<float> ua = ld<float>(uA, b + NJ), ub = ld<float>(uB, b + n);
        // (M u)_A(t) = -u_A(t) + (e^{i phi_A(t)} - dm) u_A(t-1) - dk [u_B(i,j) + u_B(i-1,j) + u_B(i,j-1)](t)
        const Cx<float> ea = ph(k);
        Cx<float> oa = hopsum(cfma(Cx<float>{ea.re - dm, ea.im}, ld<float>(uA, b), Cx<float>{-ua.re, -ua.im}), dk, ub,
                              ld<float>(uB, b + n + dim), ld<float>(uB, b));
        // (M u)_B(t) = u_B(t) + (dm - e^{-i phi_B(t)}) u_B(t+1) - dk [u_A(i,j) + u_A(i+1,j) + u_A(i,j+1)](t)
        const Cx<float> eb = ph(H + k);
        Cx<float> ob = hopsum(cfma(Cx<float>{dm - eb.re, eb.im}, ld<float>(uB, b + NJ + n), ub), dk, ua,
                              ld<float>(uA, b + NJ + dip), ld<float>(uA, b + NJ + n));
        const float2 pa = pA[b], pb = pB[b + NJ + n];
        oa.re = fmaf(sigma, pa.x, oa.re);
        oa.im = fmaf(sigma, pa.y, oa.im);
        ob.re = fmaf(sigma, pb.x, ob.re);
        ob.im = fmaf(sigma, pb.y, ob.im);
        float2 ra = r[k], rb = r[H + k];
        ra = make_float2(fmaf(-fa, oa.re, ra.x), fmaf(-fa, oa.im, ra.y));
        rb = make_float2(fmaf(-fa, ob.re, rb.x), fmaf(-fa, ob.im, rb.y));
        r[k] = ra;
        r[H + k] = rb;
        loc = fmaf(ra.x, ra.x, fmaf(ra.y, ra.y, fmaf(rb.x, rb.x, fmaf(rb.y, rb.y, loc))));
      });
    }
    {
      const float2 v = ff_block_sum(make_float2(loc, 0.f));
      if (threadIdx.x == 0) partB[blockIdx.x] = v;
    }
    if (!grid_barrier(gb, expect, limit)) {
      done = CG_TIMEOUT;
      break;
    }
    if (threadIdx.x < 32) {
      const float2 tot = ff_warp0_sum(partB, gridDim.x);
      if (threadIdx.x == 0) {
        rr_prev = rr;
        rr = tot.x + tot.y;
      }
    }
    ++iter;  // in every thread: its parity selects the buffer of published p edges
    first = false;
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

// ---------------------------------------------------------------------------
// The same kernel with two cells per thread (n even): a thread owns the cells
// (i, i+1), i even, of a row, whose complex64 values form one 16-byte float4
// in every vector and in every shared-memory array, so each load, store and
// index computation serves two cells. The i-neighbour inside the pair is the
// thread's own other half; the one across the pair boundary is the left
// pair's second cell (A rows of M^dagger and M read B at i-1) or the right
// pair's first cell (B rows read A at i+1). The rows of Eq. ferm_op are formed
// in the same order as in the one-cell kernel.
__device__ __forceinline__ Cx<float> lo4(const float4& v) { return Cx<float>{v.x, v.y}; }
__device__ __forceinline__ Cx<float> hi4(const float4& v) { return Cx<float>{v.z, v.w}; }
__device__ __forceinline__ float4 pk4(Cx<float> a, Cx<float> b) { return make_float4(a.re, a.im, b.re, b.im); }
__device__ __forceinline__ float sq4(const float4& v) { return v.x * v.x + v.y * v.y + v.z * v.z + v.w * v.w; }
// e^{i phi} of the two cells of the pair at pair index kp
__device__ __forceinline__ void phases2(const float* __restrict__ phi32, int kp, Cx<float>& e0, Cx<float>& e1) {
  const float2 f = __ldg(reinterpret_cast<const float2*>(phi32) + kp);
  float s0, c0, s1, c1;
  __sincosf(f.x, &s0, &c0);
  __sincosf(f.y, &s1, &c1);
  e0 = Cx<float>{c0, s0};
  e1 = Cx<float>{c1, s1};
}

__global__ void __launch_bounds__(kResMaxThreads, 1)
    k_cg32_resident2(Geo g, ResTile rt, const float* __restrict__ phi32, float4* __restrict__ x,
                     float4* __restrict__ r, float4* __restrict__ P0, float4* __restrict__ P1, float4* __restrict__ U,
                     CGScal* sc, float2* __restrict__ partA, float2* __restrict__ partB, GridBar* gb, long long limit,
                     unsigned expect) {
  extern __shared__ float4 s_tile4[];
  __shared__ float s_a, s_ap;
  __shared__ int s_stop;
  // all sizes and indices in cell pairs
  const int n2 = g.n >> 1, m = g.m, nt = g.nt, H2 = g.H >> 1, V2 = g.V >> 1;
  const int bj = blockIdx.x % rt.tiles_j, bt = blockIdx.x / rt.tiles_j;
  const int j0 = bj * rt.J, t0 = bt * rt.T;
  const int Jt = min(rt.J, m - j0), Tt = min(rt.T, nt - t0);
  const int J1 = rt.J + 1;
  const int SZ = (rt.T + 1) * J1 * n2;
  float4* pA = s_tile4;  // the same padded layout as the one-cell kernel, in pairs
  float4* pB = pA + SZ;
  float4* uA = pB + SZ;
  float4* uB = uA + SZ;
  auto iPA = [&](int q, int jj, int tt) { return (tt * J1 + jj) * n2 + q; };
  auto iPB = [&](int q, int jj, int tt) { return ((tt + 1) * J1 + jj + 1) * n2 + q; };
  auto iUA = [&](int q, int jj, int tt) { return ((tt + 1) * J1 + jj) * n2 + q; };
  auto iUB = [&](int q, int jj, int tt) { return (tt * J1 + jj + 1) * n2 + q; };
  const int q = threadIdx.x % n2, r0 = threadIdx.x / n2, RS = rt.rows;
  const bool act = r0 < RS;
  const int dim = (q == 0 ? n2 - 1 : q - 1) - q, dip = (q == n2 - 1 ? 0 : q + 1) - q;
  const int rows = Jt * Tt, lines = 2 * Tt + 2 * Jt;
  const int jdn = (j0 - 1 + m) % m, jup = (j0 + Jt) % m;
  const bool wlo = (t0 == 0), whi = (t0 + Tt == nt);
  const int tdn = wlo ? nt - 1 : t0 - 1, tup = whi ? 0 : t0 + Tt;
  auto cell = [&](int j, int t) { return (t * m + j) * n2 + q; };
  const int NJ = J1 * n2, kb = (t0 * m + j0) * n2 + q;
  const int dJ = RS % max(Jt, 1), dT = RS / max(Jt, 1);
  auto for_rows = [&](auto&& f) {
    int jj = r0 % Jt, tt = r0 / Jt;
    for (int R = r0; R < rows; R += RS) {
      f(jj, tt, (tt * J1 + jj) * n2 + q, kb + tt * V2 + jj * n2);
      jj += dJ;
      tt += dT;
      if (jj >= Jt) {
        jj -= Jt;
        ++tt;
      }
    }
  };
  const float dm = sc->dm32, sigma = sc->sigma32, dk = g.dkf;
  // thread 0's scalars in FP32 (the FP64 pipe is slow on this GPU and every
  // other warp of the block waits for them); the partial sums stay float-float
  float rr = sc->rr32, rr_prev = 1.f, pAp = 0.f, alpha = 0.f, beta = 0.f;
  int iter = sc->iter, done = sc->done;
  const int maxit = sc->maxit;
  const float thresh = sc->thresh32;
  bool first = true;
  for (;;) {
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
      s_ap = alpha;  // the previous iteration's alpha: x += alpha p is applied here
      s_stop = done;
    }
    __syncthreads();
    const float fap = s_ap;
    if (s_stop) {
      // the last iteration's x update, still pending
      if (act && fap != 0.f)
        for_rows([&](int, int, int b, int k) {
          const float4 pa = pA[b], pb = pB[b + NJ + n2];
          float4 xa = x[k], xb = x[H2 + k];
          x[k] = make_float4(fmaf(fap, pa.x, xa.x), fmaf(fap, pa.y, xa.y), fmaf(fap, pa.z, xa.z), fmaf(fap, pa.w, xa.w));
          x[H2 + k] = make_float4(fmaf(fap, pb.x, xb.x), fmaf(fap, pb.y, xb.y), fmaf(fap, pb.z, xb.z), fmaf(fap, pb.w, xb.w));
        });
      break;
    }
    const float fb = s_a;
    float4* Pcur = (iter & 1) ? P1 : P0;
    const float4* Pold = (iter & 1) ? P0 : P1;
    // ---- first half: padding of p, the tile's own p
    if (act) {
      // padding lines from the last row slot down: the slots that hold one row
      // fewer of the tile (rows are dealt from slot 0) take the extra lines
      for (int l = RS - 1 - r0; l < lines; l += RS) {
        int jj, tt, j, t;
        float sg = 1.f;
        bool isA;
        if (l < Tt) {
          jj = -1, tt = l, j = jdn, t = t0 + l, isA = false;
        } else if (l < 2 * Tt) {
          jj = Jt, tt = l - Tt, j = jup, t = t0 + tt, isA = true;
        } else if (l < 2 * Tt + Jt) {
          jj = l - 2 * Tt, tt = -1, j = j0 + jj, t = tdn, isA = false, sg = wlo ? -1.f : 1.f;
        } else {
          jj = l - 2 * Tt - Jt, tt = Tt, j = j0 + jj, t = tup, isA = true, sg = whi ? -1.f : 1.f;
        }
        const int k = cell(j, t) + (isA ? 0 : H2);
        float4 v = __ldcg(r + k);
        if (!first) {
          const float4 po = __ldcg(Pold + k);
          v = make_float4(fmaf(fb, po.x, v.x), fmaf(fb, po.y, v.y), fmaf(fb, po.z, v.z), fmaf(fb, po.w, v.w));
        }
        v = make_float4(sg * v.x, sg * v.y, sg * v.z, sg * v.w);
        if (isA)
          pA[iPA(q, jj, tt)] = v;
        else
          pB[iPB(q, jj, tt)] = v;
      }
      for_rows([&](int jj, int tt, int b, int k) {
        const float4 ra = __ldcg(r + k), rb = __ldcg(r + H2 + k);
        if (fap != 0.f) {  // x += alpha p with the previous iteration's p, still in place
          const float4 pa = pA[b], pb = pB[b + NJ + n2];
          const float4 xa = x[k], xb = x[H2 + k];
          x[k] = make_float4(fmaf(fap, pa.x, xa.x), fmaf(fap, pa.y, xa.y), fmaf(fap, pa.z, xa.z), fmaf(fap, pa.w, xa.w));
          x[H2 + k] = make_float4(fmaf(fap, pb.x, xb.x), fmaf(fap, pb.y, xb.y), fmaf(fap, pb.z, xb.z), fmaf(fap, pb.w, xb.w));
        }
        float4& qa = pA[b];
        float4& qb = pB[b + NJ + n2];
        float4 a = ra, c = rb;
        if (!first) {
          const float4 oa = qa, ob = qb;
          a = make_float4(fmaf(fb, oa.x, ra.x), fmaf(fb, oa.y, ra.y), fmaf(fb, oa.z, ra.z), fmaf(fb, oa.w, ra.w));
          c = make_float4(fmaf(fb, ob.x, rb.x), fmaf(fb, ob.y, rb.y), fmaf(fb, ob.z, rb.z), fmaf(fb, ob.w, rb.w));
        }
        qa = a;
        qb = c;
        if (jj == 0 || tt == 0) Pcur[k] = a;
        if (jj == Jt - 1 || tt == Tt - 1) Pcur[H2 + k] = c;
      });
    }
    __syncthreads();
    // u = M^dagger p on the tile
    float loc = 0.f;
    if (act) {
      for_rows([&](int jj, int tt, int b, int k) {
        const int t = t0 + tt;
        const float4 pa = pA[b], pb = pB[b + NJ + n2];
        Cx<float> ea0, ea1, eb0, eb1;
        phases2(phi32, t + 1 == nt ? k + V2 - H2 : k + V2, ea0, ea1);
        phases2(phi32, H2 + (t == 0 ? k - V2 + H2 : k - V2), eb0, eb1);
        // A rows: p_A(t+1), p_B at (i, j), (i-1, j), (i, j-1)
        const float4 atp = pA[b + NJ], bdn = pB[b + NJ], bl = pB[b + NJ + n2 + dim];
        const Cx<float> ua0 = hopsum(cfma(Cx<float>{ea0.re - dm, -ea0.im}, lo4(atp), Cx<float>{-pa.x, -pa.y}), dk,
                                     lo4(pb), hi4(bl), lo4(bdn));
        const Cx<float> ua1 = hopsum(cfma(Cx<float>{ea1.re - dm, -ea1.im}, hi4(atp), Cx<float>{-pa.z, -pa.w}), dk,
                                     hi4(pb), lo4(pb), hi4(bdn));
        // B rows: p_B(t-1), p_A at (i, j), (i+1, j), (i, j+1)
        const float4 btm = pB[b + n2], aup = pA[b + n2], ar = pA[b + dip];
        const Cx<float> ub0 = hopsum(cfma(Cx<float>{dm - eb0.re, -eb0.im}, lo4(btm), lo4(pb)), dk, lo4(pa), hi4(pa),
                                     lo4(aup));
        const Cx<float> ub1 = hopsum(cfma(Cx<float>{dm - eb1.re, -eb1.im}, hi4(btm), hi4(pb)), dk, hi4(pa), lo4(ar),
                                     hi4(aup));
        const float4 ua = pk4(ua0, ua1), ub = pk4(ub0, ub1);
        uA[b + NJ] = ua;
        uB[b + n2] = ub;
        if (jj == 0 || tt == Tt - 1) U[k] = ua;
        if (jj == Jt - 1 || tt == 0) U[H2 + k] = ub;
        loc += sq4(ua) + sq4(ub);
        if (sigma != 0.f) loc += sigma * (sq4(pa) + sq4(pb));
      });
    }
    {
      const float2 v = ff_block_sum(make_float2(loc, 0.f));
      if (threadIdx.x == 0) partA[blockIdx.x] = v;
    }
    if (!grid_barrier(gb, expect, limit)) {
      done = CG_TIMEOUT;
      break;
    }
    // ---- second half
    if (threadIdx.x < 32) {
      const float2 tot = ff_warp0_sum(partA, gridDim.x);
      if (threadIdx.x == 0) {
        pAp = tot.x + tot.y;
        const bool bad = !(pAp > 0.f) || !isfinite(pAp);
        alpha = bad ? 0.f : rr / pAp;
        if (bad) done = CG_BREAKDOWN;
        s_a = alpha;
        s_stop = bad;
      }
    }
    if (act) {
      for (int l = r0; l < lines; l += RS) {
        int jj, tt, j, t;
        float sg = 1.f;
        bool isA;
        if (l < Tt) {
          jj = -1, tt = l, j = jdn, t = t0 + l, isA = false;
        } else if (l < 2 * Tt) {
          jj = Jt, tt = l - Tt, j = jup, t = t0 + tt, isA = true;
        } else if (l < 2 * Tt + Jt) {
          jj = l - 2 * Tt, tt = -1, j = j0 + jj, t = tdn, isA = true, sg = wlo ? -1.f : 1.f;
        } else {
          jj = l - 2 * Tt - Jt, tt = Tt, j = j0 + jj, t = tup, isA = false, sg = whi ? -1.f : 1.f;
        }
        const float4 v = __ldcg(U + cell(j, t) + (isA ? 0 : H2));
        const float4 w = make_float4(sg * v.x, sg * v.y, sg * v.z, sg * v.w);
        if (isA)
          uA[iUA(q, jj, tt)] = w;
        else
          uB[iUB(q, jj, tt)] = w;
      }
    }
    __syncthreads();
    if (s_stop) break;
    const float fa = s_a;
    loc = 0.f;
    if (act) {
      for_rows([&](int, int, int b, int k) {
        const float4 ua = uA[b + NJ], ub = uB[b + n2];
        Cx<float> ea0, ea1, eb0, eb1;
        phases2(phi32, k, ea0, ea1);
        phases2(phi32, H2 + k, eb0, eb1);
        // A rows: u_A(t-1), u_B at (i, j), (i-1, j), (i, j-1)
        const float4 atm = uA[b], bdn = uB[b], bl = uB[b + n2 + dim];
        Cx<float> oa0 = hopsum(cfma(Cx<float>{ea0.re - dm, ea0.im}, lo4(atm), Cx<float>{-ua.x, -ua.y}), dk, lo4(ub),
                               hi4(bl), lo4(bdn));
        Cx<float> oa1 = hopsum(cfma(Cx<float>{ea1.re - dm, ea1.im}, hi4(atm), Cx<float>{-ua.z, -ua.w}), dk, hi4(ub),
                               lo4(ub), hi4(bdn));
        // B rows: u_B(t+1), u_A at (i, j), (i+1, j), (i, j+1)
        const float4 btp = uB[b + NJ + n2], aup = uA[b + NJ + n2], ar = uA[b + NJ + dip];
        Cx<float> ob0 = hopsum(cfma(Cx<float>{dm - eb0.re, eb0.im}, lo4(btp), lo4(ub)), dk, lo4(ua), hi4(ua),
                               lo4(aup));
        Cx<float> ob1 = hopsum(cfma(Cx<float>{dm - eb1.re, eb1.im}, hi4(btp), hi4(ub)), dk, hi4(ua), lo4(ar),
                               hi4(aup));
        const float4 pa = pA[b], pb = pB[b + NJ + n2];
        const float4 apa = make_float4(fmaf(sigma, pa.x, oa0.re), fmaf(sigma, pa.y, oa0.im), fmaf(sigma, pa.z, oa1.re),
                                       fmaf(sigma, pa.w, oa1.im));
        const float4 apb = make_float4(fmaf(sigma, pb.x, ob0.re), fmaf(sigma, pb.y, ob0.im), fmaf(sigma, pb.z, ob1.re),
                                       fmaf(sigma, pb.w, ob1.im));
        float4 ra = r[k], rb = r[H2 + k];
        ra = make_float4(fmaf(-fa, apa.x, ra.x), fmaf(-fa, apa.y, ra.y), fmaf(-fa, apa.z, ra.z),
                         fmaf(-fa, apa.w, ra.w));
        rb = make_float4(fmaf(-fa, apb.x, rb.x), fmaf(-fa, apb.y, rb.y), fmaf(-fa, apb.z, rb.z),
                         fmaf(-fa, apb.w, rb.w));
        r[k] = ra;
        r[H2 + k] = rb;
        loc = fmaf(ra.x, ra.x, fmaf(ra.y, ra.y, fmaf(rb.x, rb.x, fmaf(rb.y, rb.y, loc))));
        loc = fmaf(ra.z, ra.z, fmaf(ra.w, ra.w, fmaf(rb.z, rb.z, fmaf(rb.w, rb.w, loc))));
      });
    }
    {
      const float2 v = ff_block_sum(make_float2(loc, 0.f));
      if (threadIdx.x == 0) partB[blockIdx.x] = v;
    }
    if (!grid_barrier(gb, expect, limit)) {
      done = CG_TIMEOUT;
      break;
    }
    if (threadIdx.x < 32) {
      const float2 tot = ff_warp0_sum(partB, gridDim.x);
      if (threadIdx.x == 0) {
        rr_prev = rr;
        rr = tot.x + tot.y;
      }
    }
    ++iter;
    first = false;
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

// ---------------------------------------------------------------------------
// Host side

static size_t res_smem(const Geo& g, int J, int T) { return (size_t)4 * (T + 1) * (J + 1) * g.n * sizeof(float2); }

// Tile plan: every tile of J rows and T slices resident at once (one
// cooperative launch), its padded p and u arrays within the shared memory a
// block may use, and at most kResMaxThreads threads (n, or n / 2 with two
// cells per thread, per row of the tile). Among the plans that fit, the one
// with the fewest cells per tile, then the fewest padding rows and slices per
// cell.
static bool res_plan(const hmc_ctx* c, const Geo& g, bool pairs, ResTile* out, size_t* smem_out) {
  const int per_row = pairs ? g.n / 2 : g.n;
  if (per_row < 1 || per_row > kResMaxThreads) return false;
  int dev_smem = 0;
  cudaDeviceGetAttribute(&dev_smem, cudaDevAttrMaxSharedMemoryPerBlockOptin, c->device);
  const size_t cap = (size_t)std::max(0, dev_smem - 1024);  // the kernel's static arrays
  const int rows_max = kResMaxThreads / per_row;
  bool found = false;
  long long best_cells = 0;
  double best_halo = 0.0;
  for (int J = 1; J <= g.m; ++J)
    for (int T = 1; T <= g.nt; ++T) {
      const size_t sm = res_smem(g, J, T);
      if (sm > cap) break;  // larger T only grows it
      const int tj = (g.m + J - 1) / J, tt = (g.nt + T - 1) / T;
      const long long tiles = (long long)tj * tt;
      if (tiles > c->nsm || tiles > kResMaxTiles || 2 * tiles > cg32_part_capacity(c)) continue;
      const long long cells = (long long)J * T * g.n;
      const double halo = (double)(J + T) / ((double)J * T);
      if (!found || cells < best_cells || (cells == best_cells && halo < best_halo)) {
        found = true;
        best_cells = cells;
        best_halo = halo;
        out->J = J;
        out->T = T;
        out->tiles_j = tj;
        out->tiles_t = tt;
        out->rows = std::min(rows_max, J * T);
        *smem_out = sm;
      }
    }
  return found;
}

bool cg32_resident_ok(const hmc_ctx* c, const Geo& g) {
  ResTile rt;
  size_t sm = 0;
  return res_plan(c, g, false, &rt, &sm);
}

hmc_status cg32_resident_launch(hmc_ctx* c, const Geo& g, float2* x, float2* r, float2* p0, float2* p1, float2* u,
                                CGScal* sc) {
  // two cells per thread where n is even and every vector is 16-byte aligned
  auto al16 = [](const void* v) { return ((uintptr_t)v & 15u) == 0; };
  ResTile rt;
  size_t smem = 0;
  bool pairs = !(g.n & 1) && al16(x) && al16(r) && al16(p0) && al16(p1) && al16(u) && res_plan(c, g, true, &rt, &smem);
  if (!pairs && !res_plan(c, g, false, &rt, &smem))
    return fail(c, HMC_ERR_INVALID, "resident CG tiles do not fit on chip");
  const void* kfn = pairs ? (const void*)k_cg32_resident2 : (const void*)k_cg32_resident;
  if (cudaFuncSetAttribute(kfn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess)
    return cuda_fail(c, cudaGetLastError(), "resident CG shared memory");
  // whole warps (the block reductions shuffle across all 32 lanes); threads
  // beyond n x rows hold no row
  const int threads = ((pairs ? g.n / 2 : g.n) * rt.rows + 31) / 32 * 32;
  const int blocks = rt.tiles_j * rt.tiles_t;
  int occ = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kfn, threads, smem) != cudaSuccess ||
      (long long)occ * c->nsm < blocks) {
    cudaGetLastError();
    return fail(c, HMC_ERR_INVALID, "resident CG tiles cannot all be resident");
  }
  HMC_CUDA(c, cudaMemsetAsync(c->gbar, 0, sizeof(GridBar), c->stream));
  Phase<float> ph = phase_of<float>(c);
  const float* phi32 = ph.phi;
  float2* pa = (float2*)c->partA;
  float2* pb = (float2*)c->partB;
  GridBar* gb = c->gbar;
  long long limit = c->bar_limit > 0 ? c->bar_limit : 2000000000LL;
  unsigned expect = (unsigned)blocks + (unsigned)c->bar_extra;
  Geo gg = g;
  float4 *x4 = (float4*)x, *r4 = (float4*)r, *p04 = (float4*)p0, *p14 = (float4*)p1, *u4 = (float4*)u;
  void* args1[] = {&gg, &rt, &ph, &x, &r, &p0, &p1, &u, &sc, &pa, &pb, &gb, &limit, &expect};
  void* args2[] = {&gg, &rt, (void*)&phi32, &x4, &r4, &p04, &p14, &u4, &sc, &pa, &pb, &gb, &limit, &expect};
  cudaError_t le = cudaSuccess;
  HMC_TRY(launch_b(c, K_CG_RES32, 0.0, [&] {
    le = cudaLaunchCooperativeKernel(kfn, dim3(blocks), dim3(threads), pairs ? args2 : args1, smem, c->stream);
  }));
  if (le != cudaSuccess) return cuda_fail(c, le, "resident CG launch");
  c->shape[K_CG_RES32].tiled = pairs ? 4 : 0;  // reported as the design
  return HMC_OK;
}

}  // namespace hmc
