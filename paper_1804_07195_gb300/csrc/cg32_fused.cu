// FP32 CG with ONE kernel and ONE grid-wide reduction per iteration: the
// single-reduction form of CG (Chronopoulos and Gear, J. Comput. Appl. Math.
// 25 (1989) 153) with the operator A = M M^dagger + sigma (Eq. hamiltonian)
// applied by the marching scheme of the fused M M^dagger kernel, u = M^dagger r
// kept in shared memory. It is the inner FP32 solver of Section 3 and of
// Algorithm A.1 in another order of the same operations; in exact arithmetic
// its iterates equal those of plain CG.
//
// Iteration i (scalars gamma_i = |r_i|^2, delta_i = <r_i, A r_i>, both reduced
// by the previous launch; w_i = A r_i, s_{i-1} = A p_{i-1} kept as vectors):
//   beta_i  = gamma_i / gamma_{i-1}            (0 on the first iteration)
//   alpha_i = gamma_i / (delta_i - beta_i gamma_i / alpha_{i-1})
//                                              (gamma_0 / delta_0 first)
//   p_i = r_i + beta_i p_{i-1},   s_i = w_i + beta_i s_{i-1}
//   x_{i+1} = x_i + alpha_i p_i,  r_{i+1} = r_i - alpha_i s_i
//   w_{i+1} = A r_{i+1};  partials of gamma_{i+1} and of
//   delta_{i+1} = |M^dagger r_{i+1}|^2 + sigma |r_{i+1}|^2.
// The denominator of alpha_i equals <p_i, A p_i> in exact arithmetic; a
// non-positive or non-finite one ends the solve as a breakdown.
//
// A block owns a tile of Ti x Tj cells and Tt time slices, with a ring of one
// cell, exactly as the fused M M^dagger kernel. The slices of r_i, w_i,
// s_{i-1} (and, for the tile's own cells, p_{i-1} and x_i) and of phi arrive
// by cp.async D slices ahead; as a slice lands, each thread turns its own
// cell into r_{i+1} in place (and, on the tile's own slices, writes p_i, s_i,
// x_{i+1}, r_{i+1}), so the stencil steps of the fused kernel then apply A to
// r_{i+1} and the output is w_{i+1}. The first slices' copies are issued
// before the block sums the previous launch's partials, so they are in flight
// during that reduction.
//
// Vectors read on the ring (r, w, s) belong to neighbouring tiles too, so the
// launch reads them from one buffer and writes the next iterate to another;
// p and x are read and written only by their owner, in place. The scalar
// state alternates in the same way between two slots of CGScal (a launch reads
// slot par and its block 0 writes slot par ^ 1), and the reduction partials
// between the two buffers partA / partB, so no launch writes what one of its
// own blocks may still read.
#include <algorithm>
#include <cstdint>
#include <type_traits>
#include <vector>

#include "kernels.h"
#include "launch.cuh"
#include "operator.cuh"

namespace hmc {

namespace {

template <int B>
__device__ __forceinline__ void cp_async_b(void* smem, const void* gmem) {
  const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.ca.shared.global [%0], [%1], %2;" ::"r"(s), "l"(gmem), "n"(B) : "memory");
}
__device__ __forceinline__ void cp_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_wait() {
  asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory");
}

// e^{i phi} from phi in [-pi, pi] as float (phi_to_f32): hardware sine and cosine
__device__ __forceinline__ Cx<float> phase_f(float x) {
  float s, c;
  __sincosf(x, &s, &c);
  return Cx<float>{c, s};
}

__device__ __forceinline__ Cx<float> ldc(const float2* s, int k) {
  const float2 v = s[k];
  return Cx<float>{v.x, v.y};
}
__device__ __forceinline__ void stc(float2* s, int k, Cx<float> v) { s[k] = make_float2(v.re, v.im); }

// Block sums of two float-float values in a fixed order; valid in thread 0.
__device__ __forceinline__ void ff_block_sum2(float2& a, float2& b) {
  __shared__ float4 sm[32];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    a = ff_add(a, make_float2(__shfl_xor_sync(0xffffffffu, a.x, o), __shfl_xor_sync(0xffffffffu, a.y, o)));
    b = ff_add(b, make_float2(__shfl_xor_sync(0xffffffffu, b.x, o), __shfl_xor_sync(0xffffffffu, b.y, o)));
  }
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
  if (lane == 0) sm[warp] = make_float4(a.x, a.y, b.x, b.y);
  __syncthreads();
  if (warp == 0) {
    const float4 v = lane < nw ? sm[lane] : make_float4(0.f, 0.f, 0.f, 0.f);
    a = make_float2(v.x, v.y);
    b = make_float2(v.z, v.w);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      a = ff_add(a, make_float2(__shfl_xor_sync(0xffffffffu, a.x, o), __shfl_xor_sync(0xffffffffu, a.y, o)));
      b = ff_add(b, make_float2(__shfl_xor_sync(0xffffffffu, b.x, o), __shfl_xor_sync(0xffffffffu, b.y, o)));
    }
  }
}

}  // namespace

// Operands of one launch (see the file comment).
struct CG1Args {
  const float* phi32;
  const float2* r_in;
  const float2* w_in;
  const float2* s_in;
  float2* r_out;
  float2* w_out;
  float2* s_out;
  float2* p;
  float2* x;
  CGScal* sc;
  const float2* part_in;  // [2][G]: partials of gamma, then of delta (previous launch)
  float2* part_out;       // [2][G] of this launch
  int G;                  // blocks of every launch of the solve
  int par;                // scalar slot read; slot par ^ 1 is written
  int prime;              // 1: only w_0 = A r_0 and its partials (r_0 in r_in, output in w_out)
};

constexpr int kCG1MaxThreads = 512;
// dynamic shared memory per block: the 227 KB opt-in limit less 1 KB for the
// kernel's static arrays
constexpr int kCG1MaxDynSmem = 227 * 1024 - 1024;

template <int D>
__global__ void __launch_bounds__(kCG1MaxThreads) k_cg32_fused1(Geo g, FusedShape fs, CG1Args a) {
  constexpr int S = D + 2;
  static_assert(S % 4 == 0, "the ring size must be a multiple of 4");
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int TX = fs.Ti + 2, TY = fs.Tj + 2, NT = TX * TY;
  // slot arrays [S][2][NT] (sublattice A, then B, per slot)
  float2* SR = (float2*)smem_raw;  // r_i, turned into r_{i+1} in place
  float2* SW = SR + 2 * S * NT;    // w_i
  float2* SS = SW + 2 * S * NT;    // s_{i-1}
  float2* SP = SS + 2 * S * NT;    // p_{i-1} (tile cells)
  float2* SX = SP + 2 * S * NT;    // x_i (tile cells)
  float2* UA = SX + 2 * S * NT;    // [2][NT] u_A by time parity
  float2* UB = UA + 2 * NT;        // [4][NT] u_B by time mod 4
  float* PA = (float*)(UB + 4 * NT);  // [S][NT] phi_A
  float* PB = PA + S * NT;            // [S][NT] phi_B

  __shared__ float s_ab[2];
  __shared__ int s_flag;
  const int tid = threadIdx.x;
  pdl_wait();
  CGScal* sc = a.sc;
  if (tid == 0) s_flag = sc->done;
  __syncthreads();
  if (s_flag) return;
  const int prime = a.prime;
  const int it = prime ? 0 : sc->cg1_it[a.par];
  const bool first = (it == 0);

  int b = blockIdx.x;
  const int bi = b % fs.tiles_i;
  b /= fs.tiles_i;
  const int bj = b % fs.tiles_j;
  const int bt = b / fs.tiles_j;
  const int i0 = bi * fs.Ti, j0 = bj * fs.Tj, t0 = bt * fs.Tt;
  const int wi = min(fs.Ti, g.n - i0), wj = min(fs.Tj, g.m - j0), T = min(fs.Tt, g.nt - t0);
  const int li = tid % TX, lj = tid / TX;
  int gi = (i0 - 1 + li) % g.n;
  if (gi < 0) gi += g.n;
  int gj = (j0 - 1 + lj) % g.m;
  if (gj < 0) gj += g.m;
  const int cell = gj * g.n + gi;
  const bool active = tid < NT;
  const bool in_tile = active && li >= 1 && li <= wi && lj >= 1 && lj <= wj;
  const bool need_uA = active && lj >= 1, need_uB = active && lj <= TY - 2;
  const int nim = max(tid - 1, 0), nip = min(tid + 1, NT - 1);
  const int njm = max(tid - TX, 0), njp = min(tid + TX, NT - 1);
  const float dk = g.dkf;
  const float dm = sc->dm32, sigma = sc->sigma32;
  const int V = g.V, H = g.H, nt = g.nt;
  const bool wrap_lo = (t0 == 0);
  const int rw_hi = nt - t0 + 1;
  int toff_ld = (wrap_lo ? nt - 1 : t0 - 1) * V;
  int r_ld = 0;
  // what each slice needs: r always; w, s on every box cell; p, x on the tile
  const bool ld_w = !prime, ld_s = !prime && !first;

  auto issue = [&](auto JS) {  // the next slice into slot JS
    constexpr int js = decltype(JS)::value;
    if (active && r_ld <= T + 1) {
      const int sA = (2 * js) * NT + tid, sB = sA + NT, sp = js * NT + tid;
      const int kA = cell + toff_ld, kB = kA + H;
      cp_async_b<8>(SR + sA, a.r_in + kA);
      cp_async_b<8>(SR + sB, a.r_in + kB);
      if (ld_w) {
        cp_async_b<8>(SW + sA, a.w_in + kA);
        cp_async_b<8>(SW + sB, a.w_in + kB);
      }
      if (ld_s) {
        cp_async_b<8>(SS + sA, a.s_in + kA);
        cp_async_b<8>(SS + sB, a.s_in + kB);
      }
      // p and x only for the tile's own slices (r_ld = 1 .. T)
      if (!prime && in_tile && r_ld >= 1 && r_ld <= T) {
        if (!first) {
          cp_async_b<8>(SP + sA, a.p + kA);
          cp_async_b<8>(SP + sB, a.p + kB);
        }
        cp_async_b<8>(SX + sA, a.x + kA);
        cp_async_b<8>(SX + sB, a.x + kB);
      }
      cp_async_b<4>(PA + sp, a.phi32 + kA);
      cp_async_b<4>(PB + sp, a.phi32 + kB);
    }
    cp_commit();
    ++r_ld;
    toff_ld += V;
    if (toff_ld == H) toff_ld = 0;
  };

  issue(IC<0>{});
  issue(IC<1>{});
  if constexpr (D >= 2) issue(IC<2>{});
  if constexpr (D >= 3) issue(IC<3>{});
  if constexpr (D >= 4) issue(IC<4>{});
  if constexpr (D >= 5) issue(IC<5>{});
  if constexpr (D >= 6) issue(IC<6>{});

  // scalars of this iteration from the previous launch's partials (every
  // block sums them in the same order, so all blocks agree)
  float alpha = 0.f, beta = 0.f;
  if (!prime) {
    float2 ga = make_float2(0.f, 0.f), de = make_float2(0.f, 0.f);
    for (int k = tid; k < a.G; k += blockDim.x) {
      ga = ff_add(ga, __ldcg(a.part_in + k));
      de = ff_add(de, __ldcg(a.part_in + a.G + k));
    }
    ff_block_sum2(ga, de);
    if (tid == 0) {
      const double gamma = ff_to_double(ga), delta = ff_to_double(de);
      int done = CG_RUNNING;
      double al = 0.0, be = 0.0;
      if (!isfinite(gamma)) {
        done = CG_BREAKDOWN;
      } else if (gamma <= sc->thresh) {
        done = CG_CONVERGED;
      } else if (it >= sc->maxit) {
        done = CG_MAXIT;
      } else {
        double den = delta;
        if (!first) {
          be = gamma / sc->cg1_gamma[a.par];
          den = delta - be * gamma / sc->cg1_alpha[a.par];
        }
        al = gamma / den;
        if (!(den > 0.0) || !isfinite(al) || !isfinite(be)) done = CG_BREAKDOWN;
      }
      s_ab[0] = (float)al;
      s_ab[1] = (float)be;
      s_flag = done;
      if (blockIdx.x == 0) {
        sc->rr = gamma;
        sc->rr_cur = gamma;
        if (done) {
          sc->done = done;
        } else {
          const int nx = a.par ^ 1;
          sc->cg1_gamma[nx] = gamma;
          sc->cg1_alpha[nx] = al;
          sc->cg1_it[nx] = it + 1;
          sc->alpha = al;
          sc->beta = be;
          sc->pAp = gamma / al;
          sc->iter = it + 1;
          sc->first = 0;
        }
      }
    }
    __syncthreads();
    if (s_flag) {
      cp_wait<0>();
      return;
    }
    alpha = s_ab[0];
    beta = s_ab[1];
  } else if (blockIdx.x == 0 && tid == 0) {
    sc->cg1_it[0] = 0;
  }

  // halo slices outside [0, nt) continue r, w, s anti-periodically
  auto negate_own = [&](auto JS) {
    constexpr int js = decltype(JS)::value;
    if (!active) return;
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const int sl = (2 * js + h) * NT + tid;
      SR[sl] = make_float2(-SR[sl].x, -SR[sl].y);
      if (ld_w) SW[sl] = make_float2(-SW[sl].x, -SW[sl].y);
      if (ld_s) SS[sl] = make_float2(-SS[sl].x, -SS[sl].y);
    }
  };
  // the thread's own cell of slice rl (in slot JS) becomes r_{i+1}; on the
  // tile's own slices p_i, s_i, x_{i+1}, r_{i+1} are written
  auto convert = [&](auto JS, int rl) {
    constexpr int js = decltype(JS)::value;
    if (prime || !active) return;
    const bool own = in_tile && rl >= 1 && rl <= T;
    const int toff = (t0 - 1 + rl) * V;
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const int sl = (2 * js + h) * NT + tid;
      const float2 r = SR[sl], w = SW[sl];
      float2 s = w;  // s_i = w_i + beta s_{i-1}
      if (!first) {
        const float2 so = SS[sl];
        s = make_float2(fmaf(beta, so.x, w.x), fmaf(beta, so.y, w.y));
      }
      const float2 rn = make_float2(fmaf(-alpha, s.x, r.x), fmaf(-alpha, s.y, r.y));
      SR[sl] = rn;
      if (own) {
        float2 pn = r;  // p_i = r_i + beta p_{i-1}
        if (!first) {
          const float2 po = SP[sl];
          pn = make_float2(fmaf(beta, po.x, r.x), fmaf(beta, po.y, r.y));
        }
        const float2 xo = SX[sl];
        const int k = cell + toff + h * H;
        a.p[k] = pn;
        a.x[k] = make_float2(fmaf(alpha, pn.x, xo.x), fmaf(alpha, pn.y, xo.y));
        a.s_out[k] = s;
        a.r_out[k] = rn;
      }
    }
  };

  Cx<float> pAc{}, pBc{}, pAp{}, pBp{};  // r_{i+1} at t, t-1
  Cx<float> ea_c{}, ea_p{}, eb_p{};
  Cx<float> uA_m1{}, uA_m2{}, uB_0{}, uB_m1{};
  float gam = 0.f, del = 0.f;
  int toff_out = t0 * V;

  auto step = [&](auto JJ, auto OUTC, auto UC, int k) {
    constexpr int J = decltype(JJ)::value, JN = (J + 1) % S, JL = (J + D + 1) % S;
    constexpr bool OUT = decltype(OUTC)::value, U = decltype(UC)::value;
    constexpr int KA = J & 1, KA1 = (J + 1) & 1;
    constexpr int KB1 = (J + 1) & 3, KB_1 = (J + 3) & 3;
    if constexpr (U) {
      cp_wait<D - 1>();
      if (k == 0) {
        if (wrap_lo) negate_own(IC<J>{});
        convert(IC<J>{}, 0);
      }
      if (k + 1 >= rw_hi) negate_own(IC<JN>{});
      convert(IC<JN>{}, k + 1);
    }
    __syncthreads();
    if constexpr (U) issue(IC<JL>{});
    if constexpr (OUT) {
      if (in_tile) {
        const float2* UAm = UA + KA1 * NT;
        const float2* UBm = UB + KB_1 * NT;
        // w = (M u)(t-1) + sigma r(t-1), rows of Eq. ferm_op as in the fused kernel
        Cx<float> oA = hopsum(cfma(Cx<float>{ea_p.re - dm, ea_p.im}, uA_m2, Cx<float>{-uA_m1.re, -uA_m1.im}), dk,
                              uB_m1, ldc(UBm, nim), ldc(UBm, njm));
        Cx<float> oB = hopsum(cfma(Cx<float>{dm - eb_p.re, eb_p.im}, uB_0, uB_m1), dk, uA_m1, ldc(UAm, nip),
                              ldc(UAm, njp));
        oA.re = fmaf(sigma, pAp.re, oA.re);
        oA.im = fmaf(sigma, pAp.im, oA.im);
        oB.re = fmaf(sigma, pBp.re, oB.re);
        oB.im = fmaf(sigma, pBp.im, oB.im);
        stc(a.w_out, cell + toff_out, oA);
        stc(a.w_out, cell + toff_out + H, oB);
        const float rr = norm2(pAp) + norm2(pBp);
        gam += rr;
        del += norm2(uA_m1) + norm2(uB_m1) + sigma * rr;
      }
      toff_out += V;
    }
    if constexpr (U) {
      if (k == 0 && active) {
        pAc = ldc(SR + (2 * J) * NT, tid);
        pBc = ldc(SR + (2 * J + 1) * NT, tid);
      }
      Cx<float> uA{}, uBn{}, eb_c{}, ea_n{}, pAn{}, pBn{};
      const float2* SAJ = SR + (2 * J) * NT;
      const float2* SBJ = SAJ + NT;
      const float2* SAN = SR + (2 * JN) * NT;
      const float2* SBN = SAN + NT;
      if (active) {
        pAn = ldc(SAN, tid);
        pBn = ldc(SBN, tid);
        ea_n = phase_f(PA[JN * NT + tid]);
        eb_c = phase_f(PB[J * NT + tid]);
      }
      if (need_uA) {
        uA = hopsum(cfma(Cx<float>{ea_n.re - dm, -ea_n.im}, pAn, Cx<float>{-pAc.re, -pAc.im}), dk, pBc,
                    ldc(SBJ, nim), ldc(SBJ, njm));
        stc(UA + KA * NT, tid, uA);
      }
      if (need_uB) {
        uBn = hopsum(cfma(Cx<float>{dm - eb_c.re, -eb_c.im}, pBc, pBn), dk, pAn, ldc(SAN, nip), ldc(SAN, njp));
        stc(UB + KB1 * NT, tid, uBn);
      }
      uA_m2 = uA_m1;
      uA_m1 = uA;
      uB_m1 = uB_0;
      uB_0 = uBn;
      pAp = pAc;
      pBp = pBc;
      pAc = pAn;
      pBc = pBn;
      ea_p = ea_c;
      ea_c = ea_n;
      eb_p = eb_c;
    }
  };

  step(IC<0>{}, std::false_type{}, std::true_type{}, 0);
  if (T >= 1) step(IC<1 % S>{}, std::false_type{}, std::true_type{}, 1);
  for (int k0 = 0; T >= 2; k0 += S) {
    if (k0 + 2 > T) break;
    step(IC<2 % S>{}, std::true_type{}, std::true_type{}, k0 + 2);
    if (k0 + 3 > T) break;
    step(IC<3 % S>{}, std::true_type{}, std::true_type{}, k0 + 3);
    if constexpr (S > 4) {
      if (k0 + 4 > T) break;
      step(IC<4 % S>{}, std::true_type{}, std::true_type{}, k0 + 4);
      if (k0 + 5 > T) break;
      step(IC<5 % S>{}, std::true_type{}, std::true_type{}, k0 + 5);
    }
    if constexpr (S > 6) {
      if (k0 + 6 > T) break;
      step(IC<6 % S>{}, std::true_type{}, std::true_type{}, k0 + 6);
      if (k0 + 7 > T) break;
      step(IC<7 % S>{}, std::true_type{}, std::true_type{}, k0 + 7);
    }
    if (k0 + S > T) break;
    step(IC<0>{}, std::true_type{}, std::true_type{}, k0 + S);
    if (k0 + S + 1 > T) break;
    step(IC<1>{}, std::true_type{}, std::true_type{}, k0 + S + 1);
  }
  switch ((T + 1) % 4) {
    case 0: step(IC<0>{}, std::true_type{}, std::false_type{}, T + 1); break;
    case 1: step(IC<1>{}, std::true_type{}, std::false_type{}, T + 1); break;
    case 2: step(IC<2>{}, std::true_type{}, std::false_type{}, T + 1); break;
    default: step(IC<3>{}, std::true_type{}, std::false_type{}, T + 1); break;
  }
  cp_wait<0>();
  pdl_trigger();
  float2 ga = make_float2(gam, 0.f), de = make_float2(del, 0.f);
  ff_block_sum2(ga, de);
  if (tid == 0) {
    a.part_out[blockIdx.x] = ga;
    a.part_out[a.G + blockIdx.x] = de;
  }
}

// ---------------------------------------------------------------------------
// Host side

static int cg1_threads_of(const FusedShape& fs) { return (fs.Ti + 2) * (fs.Tj + 2); }

static int cg1_smem_of(const FusedShape& fs) {
  const int NT = cg1_threads_of(fs), S = fs.D + 2;
  return (10 * S + 6) * NT * 8 + 2 * S * NT * 4;
}

bool cg1_ok(const hmc_ctx* c, const Geo& g, const FusedShape& fs) {
  if (fs.pairs || (fs.D != 2 && fs.D != 6) || fs.Ti < 1 || fs.Tj < 1 || fs.Tt < 1) return false;
  if (cg1_threads_of(fs) > kCG1MaxThreads || cg1_smem_of(fs) > kCG1MaxDynSmem) return false;
  const long long blocks = (long long)fs.tiles_i * fs.tiles_j * fs.tiles_t;
  (void)g;
  return blocks >= 1 && 2 * blocks <= cg32_part_capacity(c);
}

// One launch; the state slot par is read and par ^ 1 written (prime: w_0 = A r_0).
static void cg1_raw(hmc_ctx* c, const Geo& g, const FusedShape& fs, const CG1Args& a) {
  static unsigned long long attr_set = 0;
  const unsigned long long bit = 1ull << (c->device & 63);
  if (!(attr_set & bit)) {
    // the opt-in limit covers the kernel's static shared arrays too
    cudaFuncSetAttribute(k_cg32_fused1<2>, cudaFuncAttributeMaxDynamicSharedMemorySize, kCG1MaxDynSmem);
    cudaFuncSetAttribute(k_cg32_fused1<6>, cudaFuncAttributeMaxDynamicSharedMemorySize, kCG1MaxDynSmem);
    attr_set |= bit;
  }
  const int threads = (cg1_threads_of(fs) + 31) / 32 * 32;
  const int smem = cg1_smem_of(fs);
  const dim3 grid(fs.tiles_i * fs.tiles_j * fs.tiles_t);
  if (fs.D == 2)
    launch_pdl_smem(c, k_cg32_fused1<2>, grid, threads, smem, c->stream, g, fs, a);
  else
    launch_pdl_smem(c, k_cg32_fused1<6>, grid, threads, smem, c->stream, g, fs, a);
}

CG1Bufs cg1_bufs(hmc_ctx* c, float2* r0) {
  CG1Bufs B{};
  const size_t bytes = sizeof(float2) * (size_t)c->geo.N;
  B.r[0] = r0;
  if (ws_get(c, WS_CG1_R1, bytes, (void**)&B.r[1]) != HMC_OK) return CG1Bufs{};
  if (ws_get(c, WS_CG1_W0, bytes, (void**)&B.w[0]) != HMC_OK) return CG1Bufs{};
  if (ws_get(c, WS_CG1_W1, bytes, (void**)&B.w[1]) != HMC_OK) return CG1Bufs{};
  if (ws_get(c, WS_CG1_S0, bytes, (void**)&B.s[0]) != HMC_OK) return CG1Bufs{};
  if (ws_get(c, WS_CG1_S1, bytes, (void**)&B.s[1]) != HMC_OK) return CG1Bufs{};
  B.part[0] = (float2*)c->partA;
  B.part[1] = (float2*)c->partB;
  return B;
}

static CG1Args cg1_args(hmc_ctx* c, const FusedShape& fs, const CG1Bufs& B, float2* p, float2* x, CGScal* sc,
                        int par, int prime) {
  CG1Args a;
  a.phi32 = (const float*)c->ws[WS_PHI32];
  a.r_in = B.r[par];
  a.w_in = B.w[par];
  a.s_in = B.s[par];
  a.r_out = B.r[par ^ 1];
  a.w_out = prime ? B.w[0] : B.w[par ^ 1];
  a.s_out = B.s[par ^ 1];
  a.p = p;
  a.x = x;
  a.sc = sc;
  a.part_in = B.part[par];
  a.part_out = prime ? B.part[0] : B.part[par ^ 1];
  a.G = fs.tiles_i * fs.tiles_j * fs.tiles_t;
  a.par = par;
  a.prime = prime;
  return a;
}

hmc_status cg1_prime_launch(hmc_ctx* c, const Geo& g, const CG1Bufs& B, float2* p, float2* x, CGScal* sc) {
  const FusedShape fs = c->cg1_shape;
  if (!cg1_ok(c, g, fs)) return fail(c, HMC_ERR_INVALID, "single-reduction CG shape not tuned");
  return launch_b(c, K_CG1_32, 20.0 * g.N, [&] { cg1_raw(c, g, fs, cg1_args(c, fs, B, p, x, sc, 0, 1)); });
}

hmc_status cg1_iter_launch(hmc_ctx* c, const Geo& g, const CG1Bufs& B, float2* p, float2* x, CGScal* sc, int par) {
  const FusedShape fs = c->cg1_shape;
  if (!cg1_ok(c, g, fs)) return fail(c, HMC_ERR_INVALID, "single-reduction CG shape not tuned");
  return launch_b(c, K_CG1_32, kKernelBytesPerSite[K_CG1_32] * g.N,
                  [&] { cg1_raw(c, g, fs, cg1_args(c, fs, B, p, x, sc, par & 1, 0)); });
}

// Tile tuner of the single-reduction kernel: every candidate runs a primed
// start and a few iterations (tolerance 0, so none stops) on this solve's
// vectors; the fastest per iteration is kept. Returns false when no tile fits.
bool cg1_tune(hmc_ctx* c, const Geo& g, const CG1Bufs& B, float2* p, float2* x, CGScal* sc,
              const std::function<hmc_status()>& reinit) {
  std::vector<FusedShape> cands;
  for (int TX : {16, 32})
    for (int Tj : {4, 6, 8, 14})
      for (int Tt : {4, 8, 16})
        for (int D : {2}) {
          const FusedShape fs = make_fused_shape(g, TX - 2, Tj, Tt, D, 0);
          if (!cg1_ok(c, g, fs)) continue;
          bool dup = false;
          for (const auto& o : cands) dup = dup || (o.Ti == fs.Ti && o.Tj == fs.Tj && o.Tt == fs.Tt && o.D == fs.D);
          if (!dup) cands.push_back(fs);
        }
  if (cands.empty()) return false;
  cudaEvent_t e0, e1;
  if (cudaEventCreate(&e0) != cudaSuccess) return false;
  if (cudaEventCreate(&e1) != cudaSuccess) {
    cudaEventDestroy(e0);
    return false;
  }
  float best = 1e30f;
  FusedShape keep = cands[0];
  for (const FusedShape& fs : cands) {
    c->cg1_shape = fs;
    if (reinit() != HMC_OK) break;
    // a candidate whose launch fails is skipped, never kept
    bool ok = cg1_prime_launch(c, g, B, p, x, sc) == HMC_OK;
    for (int i = 0; ok && i < 2; ++i) ok = cg1_iter_launch(c, g, B, p, x, sc, i) == HMC_OK;
    cudaEventRecord(e0, c->stream);
    for (int i = 0; ok && i < 6; ++i) ok = cg1_iter_launch(c, g, B, p, x, sc, i) == HMC_OK;
    cudaEventRecord(e1, c->stream);
    if (cudaEventSynchronize(e1) != cudaSuccess) break;
    if (!ok) {
      cudaGetLastError();
      c->err.clear();
      continue;
    }
    float ms = 0.f;
    cudaEventElapsedTime(&ms, e0, e1);
    if (ms < best) {
      best = ms;
      keep = fs;
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  c->cg1_shape = keep;
  return best < 1e30f;
}

hmc_status set_cg1_shape(hmc_ctx* c, int Ti, int Tj, int Tt, int D) {
  const FusedShape fs = make_fused_shape(c->geo, Ti, Tj, Tt, D, 0);
  if (!cg1_ok(c, c->geo, fs)) return fail(c, HMC_ERR_INVALID, "single-reduction CG tile does not fit");
  c->cg1_shape = fs;
  c->cg1_pinned = true;
  return HMC_OK;
}

}  // namespace hmc
