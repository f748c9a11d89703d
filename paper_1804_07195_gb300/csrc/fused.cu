// The operator A = M_ms M_ms^dagger + sigma of Eq. hamiltonian (and of the
// shifted and staggered-mass forms of Section 5.1) in ONE pass over memory:
// the intermediate u = M^dagger p never leaves the chip.
//
// A block owns a tile of Ti x Tj cells and a range of Tt time slices. Its
// threads cover the tile plus a ring of one cell on every side
// ((Ti+2) x (Tj+2) threads, one cell each) and march upward in time. Step t:
//   1. the slices t and t+1 of p_A, p_B, and of the field's phase source, are
//      resident in a ring of shared-memory slots, filled D slices ahead with
//      cp.async (each thread copies its own cell);
//   2. every thread forms u_A(t) and u_B(t+1) of its cell from the staged
//      slices (M^dagger of Eq. ferm_op: the hops t -> t+1 on A, t+1 -> t on B,
//      the three honeycomb neighbours from the neighbouring threads' slots)
//      and stores them in shared memory;
//   3. the tile's threads form (M u)(t) + sigma p(t) from u_A(t-1) (kept in a
//      register), u_A(t), u_B(t), u_B(t+1) and the neighbours' u, and store it.
// The ring cells recompute u that a neighbouring tile also computes; that
// costs arithmetic, not memory traffic, since the ring's loads are served by
// L2 while the neighbouring tile reads the same slices. Per site the kernel
// moves p (read), the phase source (read) and the result (write): 20 bytes
// in FP32 (phi as float), 48 bytes in FP64 (the e^{i phi} table).
//
// A cell at box position (li, lj) is the lattice cell ((i0 - 1 + li) mod n,
// (j0 - 1 + lj) mod m): neighbouring box positions are neighbouring lattice
// cells for every n, m >= 1 (a box wider than the lattice holds some cells
// twice), so no case needs special handling.
#include <algorithm>
#include <cstdint>
#include <type_traits>
#include <vector>

#include "kernels.h"
#include "launch.cuh"
#include "operator.cuh"

namespace hmc {

namespace {

// FP64 blocks are capped lower so that the kernel keeps its state in registers
template <typename R>
constexpr int fused_max_threads() { return sizeof(R) == 4 ? 1024 : 512; }

template <int B>
__device__ __forceinline__ void cp_async_n(void* smem, const void* gmem) {
  const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
  if constexpr (B == 16) {
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(s), "l"(gmem) : "memory");
  } else {
    asm volatile("cp.async.ca.shared.global [%0], [%1], %2;" ::"r"(s), "l"(gmem), "n"(B) : "memory");
  }
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() {
  asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory");
}

// Phase sources: what is staged per site, and e^{i phi} from it.
struct PhaseF32 {  // phi in [-pi, pi] as float (phi_to_f32); hardware sine and cosine
  using T = float;
  __device__ __forceinline__ static Cx<float> eval(float x) {
    float s, c;
    __sincosf(x, &s, &c);
    return Cx<float>{c, s};
  }
};
struct PhaseE64 {  // the FP64 table e^{i phi}
  using T = double2;
  __device__ __forceinline__ static Cx<double> eval(double2 e) { return Cx<double>{e.x, e.y}; }
};

template <typename R>
struct FusedPhase;
template <>
struct FusedPhase<float> {
  using type = PhaseF32;
};
template <>
struct FusedPhase<double> {
  using type = PhaseE64;
};

template <typename R>
__device__ __forceinline__ Cx<R> ld_c(const V2<R>* s, int k) {
  const V2<R> v = s[k];
  return Cx<R>{v.x, v.y};
}
template <typename R>
__device__ __forceinline__ void st_c(V2<R>* s, int k, Cx<R> v) {
  V2<R> w;
  w.x = v.re;
  w.y = v.im;
  s[k] = w;
}

}  // namespace

// out = (M M^dagger + sigma) p over the tile of this block; see the header
// comment. ph: the phase source (phi as float for R = float, the table
// e^{i phi} for R = double), in the canonical layout.
//
// Step k of the march (time t = t0 - 1 + k) begins with the block's only
// barrier, which publishes both the slice t+1 that arrived and the u values
// that step k-1 stored. The step then forms the output at t-1 from u(t-2),
// u(t-1), u(t) (already published), and u_A(t), u_B(t+1) for the next step.
// u_A is double-buffered and u_B kept for four times, indexed by time, so no
// step writes a buffer that another thread reads in the same step.
//
// The staged slices continue p anti-periodically in time: a slice that lies
// one period before slice 0 or after slice nt - 1 is stored negated once it
// has arrived (only blocks at either end of the time range have one), so the
// time hops carry no sign of their own and u inherits the same continuation
// (u(-1) = -u(nt - 1), u(nt) = -u(0)), which is exactly the anti-periodic
// boundary of Eq. ferm_op. The steps are unrolled over the ring's slots, so
// every slot offset is a compile-time constant.
template <typename R, int D>
__global__ void __launch_bounds__(fused_max_threads<R>()) k_mmdag_fused(Geo g, FusedShape fs,
                                                                  const typename FusedPhase<R>::type::T* __restrict__ ph,
                                                                  R dm, R sigma, const V2<R>* __restrict__ p,
                                                                  V2<R>* __restrict__ out) {
  using PS = typename FusedPhase<R>::type;
  using PT = typename PS::T;
  constexpr int S = D + 2;  // the step's slot J = k mod S also gives k mod 2 and k mod 4
  static_assert(S % 4 == 0, "the ring size must be a multiple of 4");
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int TX = fs.Ti + 2, TY = fs.Tj + 2, NT = TX * TY;
  V2<R>* SA = (V2<R>*)smem_raw;  // [S][NT] p_A slices
  V2<R>* SB = SA + S * NT;       // [S][NT] p_B slices
  V2<R>* UA = SB + S * NT;       // [2][NT] u_A by time parity
  V2<R>* UB = UA + 2 * NT;       // [4][NT] u_B by time mod 4
  PT* PA = (PT*)(UB + 4 * NT);   // [S][NT] phase source, A
  PT* PB = PA + S * NT;          // [S][NT] phase source, B

  const int tid = threadIdx.x;
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
  // u_A is read only at box rows >= 1, u_B only at rows <= TY - 2 (whole
  // warps when TX is a multiple of 32)
  const bool need_uA = active && lj >= 1, need_uB = active && lj <= TY - 2;
  // neighbouring box positions (clamped: box-edge threads compute values no
  // tile thread reads)
  const int nim = max(tid - 1, 0), nip = min(tid + 1, NT - 1);
  const int njm = max(tid - TX, 0), njp = min(tid + TX, NT - 1);
  const R dk = geo_dk(g, R(0));
  const int V = g.V, H = g.H, nt = g.nt;
  const V2<R>* __restrict__ pg = p + cell;
  const PT* __restrict__ phg = ph + cell;
  V2<R>* __restrict__ og = out + cell;
  // slice r (0 <= r <= T + 1) holds time t0 - 1 + r; it lies outside [0, nt)
  // (and is negated) for r == 0 when t0 == 0 and for r >= rw_hi
  const bool wrap_lo = (t0 == 0);
  const int rw_hi = nt - t0 + 1;
  int toff_ld = (wrap_lo ? nt - 1 : t0 - 1) * V;  // time offset of the next slice to load
  int r_ld = 0;

  auto issue = [&](auto JS) {  // the next slice into slot JS
    constexpr int js = decltype(JS)::value;
    if (active && r_ld <= T + 1) {
      const int slot = js * NT + tid;
      cp_async_n<sizeof(V2<R>)>(SA + slot, pg + toff_ld);
      cp_async_n<sizeof(V2<R>)>(SB + slot, pg + H + toff_ld);
      cp_async_n<sizeof(PT)>(PA + slot, phg + toff_ld);
      cp_async_n<sizeof(PT)>(PB + slot, phg + H + toff_ld);
    }
    cp_async_commit();
    ++r_ld;
    toff_ld += V;
    if (toff_ld == H) toff_ld = 0;
  };
  auto negate_own = [&](auto JS) {
    constexpr int js = decltype(JS)::value;
    if (active) {
      V2<R>& a = SA[js * NT + tid];
      V2<R>& c = SB[js * NT + tid];
      a.x = -a.x;
      a.y = -a.y;
      c.x = -c.x;
      c.y = -c.y;
    }
  };

  issue(IC<0>{});
  issue(IC<1>{});
  if constexpr (D >= 2) issue(IC<2>{});
  if constexpr (D >= 3) issue(IC<3>{});
  if constexpr (D >= 4) issue(IC<4>{});
  if constexpr (D >= 5) issue(IC<5>{});
  if constexpr (D >= 6) issue(IC<6>{});

  // own values carried between steps (k: the current step, t its time)
  Cx<R> pAc{}, pBc{};          // p(t)
  Cx<R> pAp{}, pBp{};          // p(t-1)
  Cx<R> ea_c{}, ea_p{}, eb_p{};  // e^{i phi_A(t)}, e^{i phi_A(t-1)}, e^{i phi_B(t-1)}
  Cx<R> uA_m1{}, uA_m2{};      // u_A(t-1), u_A(t-2)
  Cx<R> uB_0{}, uB_m1{};       // u_B(t), u_B(t-1)
  int toff_out = t0 * V;  // time offset of the next output (the first, at k = 2, is time t0)

  // the output at t - 1 (OUT) and u_A(t), u_B(t+1) (U); J = k mod S
  auto step = [&](auto JJ, auto OUTC, auto UC, int k) {
    constexpr int J = decltype(JJ)::value, JN = (J + 1) % S, JL = (J + D + 1) % S;
    constexpr bool OUT = decltype(OUTC)::value, U = decltype(UC)::value;
    // u buffers by time: u_A(t) -> UA[k & 1], u_B(t+1) -> UB[(k+1) & 3]
    constexpr int KA = J & 1, KA1 = (J + 1) & 1;
    constexpr int KB1 = (J + 1) & 3, KB_1 = (J + 3) & 3;
    if constexpr (U) {
      cp_async_wait<D - 1>();
      if (k == 0 && wrap_lo) negate_own(IC<J>{});
      if (k + 1 >= rw_hi) negate_own(IC<JN>{});
    }
    __syncthreads();
    if constexpr (U) issue(IC<JL>{});
    if constexpr (OUT) {
      if (in_tile) {
        const V2<R>* UAm = UA + KA1 * NT;   // u_A(t-1)
        const V2<R>* UBm = UB + KB_1 * NT;  // u_B(t-1)
        // (M u)_A(t-1) = -u_A(t-1) + (e^{i phi_A(t-1)} - dm) u_A(t-2) - dk [u_B(i,j) + u_B(i-1,j) + u_B(i,j-1)](t-1)
        Cx<R> oA = hopsum(cfma(Cx<R>{ea_p.re - dm, ea_p.im}, uA_m2, Cx<R>{-uA_m1.re, -uA_m1.im}), dk, uB_m1,
                          ld_c<R>(UBm, nim), ld_c<R>(UBm, njm));
        // (M u)_B(t-1) = u_B(t-1) + (dm - e^{-i phi_B(t-1)}) u_B(t) - dk [u_A(i,j) + u_A(i+1,j) + u_A(i,j+1)](t-1)
        Cx<R> oB = hopsum(cfma(Cx<R>{dm - eb_p.re, eb_p.im}, uB_0, uB_m1), dk, uA_m1, ld_c<R>(UAm, nip),
                          ld_c<R>(UAm, njp));
        oA.re = fma(sigma, pAp.re, oA.re);
        oA.im = fma(sigma, pAp.im, oA.im);
        oB.re = fma(sigma, pBp.re, oB.re);
        oB.im = fma(sigma, pBp.im, oB.im);
        st(og, toff_out, oA);
        st(og, toff_out + H, oB);
      }
      toff_out += V;
    }
    if constexpr (U) {
      if (k == 0 && active) {
        pAc = ld_c<R>(SA + J * NT, tid);
        pBc = ld_c<R>(SB + J * NT, tid);
      }
      Cx<R> uA{}, uBn{}, eb_c{}, ea_n{}, pAn{}, pBn{};
      if (active) {
        pAn = ld_c<R>(SA + JN * NT, tid);
        pBn = ld_c<R>(SB + JN * NT, tid);
        ea_n = PS::eval(PA[JN * NT + tid]);
        eb_c = PS::eval(PB[J * NT + tid]);
      }
      if (need_uA) {
        // u_A(t) = -p_A(t) + (e^{-i phi_A(t+1)} - dm) p_A(t+1) - dk [p_B(i,j) + p_B(i-1,j) + p_B(i,j-1)](t)
        uA = hopsum(cfma(Cx<R>{ea_n.re - dm, -ea_n.im}, pAn, Cx<R>{-pAc.re, -pAc.im}), dk, pBc,
                    ld_c<R>(SB + J * NT, nim), ld_c<R>(SB + J * NT, njm));
        st_c<R>(UA + KA * NT, tid, uA);
      }
      if (need_uB) {
        // u_B(t+1) = p_B(t+1) + (dm - e^{i phi_B(t)}) p_B(t) - dk [p_A(i,j) + p_A(i+1,j) + p_A(i,j+1)](t+1)
        uBn = hopsum(cfma(Cx<R>{dm - eb_c.re, -eb_c.im}, pBc, pBn), dk, pAn, ld_c<R>(SA + JN * NT, nip),
                     ld_c<R>(SA + JN * NT, njp));
        st_c<R>(UB + KB1 * NT, tid, uBn);
      }
      // shift the carried values by one time step
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

  // k = 0 and 1 form u only; from k = 2 on, each step also writes the output
  // at t - 1; the output at t0 + T - 1 comes after the last u step.
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
  // the last output (time t0 + T - 1) at the step after k = T; only the
  // parities of that step's slot matter here
  switch ((T + 1) % 4) {
    case 0: step(IC<0>{}, std::true_type{}, std::false_type{}, T + 1); break;
    case 1: step(IC<1>{}, std::true_type{}, std::false_type{}, T + 1); break;
    case 2: step(IC<2>{}, std::true_type{}, std::false_type{}, T + 1); break;
    default: step(IC<3>{}, std::true_type{}, std::false_type{}, T + 1); break;
  }
  cp_async_wait<0>();
}

// ---------------------------------------------------------------------------
// FP32 with two cells per thread. A thread owns the neighbouring cells
// (2q, 2q+1) of a row, whose complex64 values form one 16-byte float4 in
// memory when n is even, so every staging copy, shared-memory access and
// store moves two cells. The i-neighbour that lies inside the pair comes from
// the thread's own registers; the one across the pair boundary from the
// neighbouring thread's slot. The box is Ti + 4 cells wide (cells i0 - 2 to
// i0 + Ti + 1, Ti even: pairs stay aligned) and Tj + 2 rows high; the cells
// i0 - 1 and i0 + Ti are the ring, the outermost two columns only feed them.
// Each step has two block barriers: one publishes the arrived slice, the
// other the u values the step formed, and the step's output follows it (no
// lag, so u_A is single-buffered and u_B double-buffered). u is kept as
// first-cell and second-cell halves, since the i-neighbours read one half
// of a pair. Eq. ferm_op rows as in k_mmdag_fused.
__device__ __forceinline__ Cx<float> lo_c(const float4& v) { return Cx<float>{v.x, v.y}; }
__device__ __forceinline__ Cx<float> hi_c(const float4& v) { return Cx<float>{v.z, v.w}; }
__device__ __forceinline__ float4 pack4(Cx<float> a, Cx<float> b) { return make_float4(a.re, a.im, b.re, b.im); }

// Packed FP32 pair arithmetic (add.rn.f32x2, fma.rn.f32x2; sm_100 and
// later): each lane is rounded as the scalar instruction would round it, so
// a sum formed this way equals the scalar one bit for bit.
__device__ __forceinline__ unsigned long long pk2(Cx<float> v) {
  unsigned long long r;
  asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(v.re), "f"(v.im));
  return r;
}
__device__ __forceinline__ Cx<float> upk2(unsigned long long v) {
  Cx<float> r;
  asm("mov.b64 {%0, %1}, %2;" : "=f"(r.re), "=f"(r.im) : "l"(v));
  return r;
}
__device__ __forceinline__ unsigned long long add_x2(unsigned long long a, unsigned long long b) {
  unsigned long long r;
  asm("add.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(a), "l"(b));
  return r;
}
__device__ __forceinline__ unsigned long long fma_x2(unsigned long long a, unsigned long long b,
                                                     unsigned long long c) {
  unsigned long long r;
  asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(r) : "l"(a), "l"(b), "l"(c));
  return r;
}
// hopsum with both components in one packed pair: t - dk (a + b + c);
// ndk = (-dk, -dk)
__device__ __forceinline__ Cx<float> hopsum_x2(Cx<float> t, unsigned long long ndk, Cx<float> a, Cx<float> b,
                                               Cx<float> c) {
  return upk2(fma_x2(ndk, add_x2(add_x2(pk2(a), pk2(b)), pk2(c)), pk2(t)));
}
// (re, im) of the pair's first and second cell
__device__ __forceinline__ Cx<float> hi_of(const float4* v) { return Cx<float>{v->z, v->w}; }
__device__ __forceinline__ Cx<float> lo_of(const float4* v) { return Cx<float>{v->x, v->y}; }

// At most 256 threads per block and 80 registers per thread: six blocks of
// 128 threads share an SM.
constexpr int kPairMaxThreads = 256;

template <int D>
__global__ void __launch_bounds__(kPairMaxThreads, 3) k_mmdag_fused_pairs(Geo g, FusedShape fs, const float2* __restrict__ ph,
                                                           float dm, float sigma, const float4* __restrict__ p,
                                                           float4* __restrict__ out) {
  constexpr int S = D + 2;
  static_assert(S % 2 == 0, "ring size");
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int TXP = fs.Ti / 2 + 2, TY = fs.Tj + 2, NT = TXP * TY;
  float4* SA = (float4*)smem_raw;  // [S][NT] p_A pairs
  float4* SB = SA + S * NT;        // [S][NT] p_B pairs
  // u in halves (first cells, second cells): the i-neighbours read one half
  // of a pair, which from 16-byte pairs would take twice its wavefronts
  float2* UAl = (float2*)(SB + S * NT);  // [NT]    u_A(t), first cells
  float2* UAh = UAl + NT;                // [NT]    second cells
  float2* UBl = UAh + NT;                // [2][NT] u_B(t), u_B(t+1), first cells
  float2* UBh = UBl + 2 * NT;            // [2][NT] second cells
  float2* PA = UBh + 2 * NT;             // [S][NT] phi_A pairs
  float2* PB = PA + S * NT;             // [S][NT] phi_B pairs

  const int tid = threadIdx.x;
  int b = blockIdx.x;
  const int bi = b % fs.tiles_i;
  b /= fs.tiles_i;
  const int bj = b % fs.tiles_j;
  const int bt = b / fs.tiles_j;
  const int n2 = g.n >> 1;
  const int i0 = bi * fs.Ti, j0 = bj * fs.Tj, t0 = bt * fs.Tt;
  const int wp = min(fs.Ti, g.n - i0) >> 1, wj = min(fs.Tj, g.m - j0), T = min(fs.Tt, g.nt - t0);
  const int lp = tid % TXP, lj = tid / TXP;
  int gp = ((i0 >> 1) - 1 + lp) % n2;
  if (gp < 0) gp += n2;
  int gj = (j0 - 1 + lj) % g.m;
  if (gj < 0) gj += g.m;
  const int cellp = gj * n2 + gp;  // pair index within a time slice
  const bool active = tid < NT;
  const bool in_tile = active && lp >= 1 && lp <= wp && lj >= 1 && lj <= wj;
  const bool need_uA = active && lj >= 1, need_uB = active && lj <= TY - 2;
  const int nim = max(tid - 1, 0), nip = min(tid + 1, NT - 1);
  const int njm = max(tid - TXP, 0), njp = min(tid + TXP, NT - 1);
  const float dk = g.dkf;
  const int V = g.V >> 1, H = g.H >> 1, nt = g.nt;  // in pairs
  const float4* __restrict__ pg = p + cellp;
  const float2* __restrict__ phg = ph + cellp;
  float4* __restrict__ og = out + cellp;
  const bool wrap_lo = (t0 == 0);
  const int rw_hi = nt - t0 + 1;
  int toff_ld = (wrap_lo ? nt - 1 : t0 - 1) * V;
  int r_ld = 0;

  auto issue = [&](auto JS) {
    constexpr int js = decltype(JS)::value;
    if (active && r_ld <= T + 1) {
      const int slot = js * NT + tid;
      cp_async_n<16>(SA + slot, pg + toff_ld);
      cp_async_n<16>(SB + slot, pg + H + toff_ld);
      cp_async_n<8>(PA + slot, phg + toff_ld);
      cp_async_n<8>(PB + slot, phg + H + toff_ld);
    }
    cp_async_commit();
    ++r_ld;
    toff_ld += V;
    if (toff_ld == H) toff_ld = 0;
  };
  auto negate_own = [&](auto JS) {
    constexpr int js = decltype(JS)::value;
    if (active) {
      float4& a = SA[js * NT + tid];
      float4& c = SB[js * NT + tid];
      a = make_float4(-a.x, -a.y, -a.z, -a.w);
      c = make_float4(-c.x, -c.y, -c.z, -c.w);
    }
  };

  issue(IC<0>{});
  issue(IC<1>{});
  if constexpr (D >= 2) issue(IC<2>{});
  if constexpr (D >= 3) issue(IC<3>{});
  if constexpr (D >= 4) issue(IC<4>{});
  if constexpr (D >= 5) issue(IC<5>{});
  if constexpr (D >= 6) issue(IC<6>{});

  float4 pAc{}, pBc{}, uA_prev{}, uB_cur{};
  Cx<float> ea_c0{}, ea_c1{};
  const unsigned long long ndk = pk2(Cx<float>{-dk, -dk});
  int toff_out = t0 * V;

  auto step = [&](auto JJ, auto OUTC, int k) {
    constexpr int J = decltype(JJ)::value, JN = (J + 1) % S, JL = (J + D + 1) % S;
    constexpr bool OUT = decltype(OUTC)::value;
    cp_async_wait<D - 1>();
    if (!OUT && wrap_lo) negate_own(IC<J>{});
    if (k + 1 >= rw_hi) negate_own(IC<JN>{});
    __syncthreads();
    issue(IC<JL>{});
    if (!OUT && active) {
      pAc = SA[J * NT + tid];
      pBc = SB[J * NT + tid];
    }
    float4 uA{}, uBn{}, pAn{}, pBn{};
    Cx<float> ea_n0{}, ea_n1{}, eb_c0{}, eb_c1{};
    if (active) {
      pAn = SA[JN * NT + tid];
      pBn = SB[JN * NT + tid];
      const float2 fa = PA[JN * NT + tid], fb = PB[J * NT + tid];
      ea_n0 = PhaseF32::eval(fa.x);
      ea_n1 = PhaseF32::eval(fa.y);
      eb_c0 = PhaseF32::eval(fb.x);
      eb_c1 = PhaseF32::eval(fb.y);
    }
    if (need_uA) {
      // u_A(t) = -p_A(t) + (e^{-i phi_A(t+1)} - dm) p_A(t+1) - dk [p_B(i,j) + p_B(i-1,j) + p_B(i,j-1)](t)
      // (of the left pair only its second cell is read)
      const Cx<float> left = hi_of(SB + J * NT + nim);
      const float4 up = SB[J * NT + njm];
      const Cx<float> u0 = hopsum_x2(cfma(Cx<float>{ea_n0.re - dm, -ea_n0.im}, lo_c(pAn), Cx<float>{-pAc.x, -pAc.y}),
                                     ndk, lo_c(pBc), left, lo_c(up));
      const Cx<float> u1 = hopsum_x2(cfma(Cx<float>{ea_n1.re - dm, -ea_n1.im}, hi_c(pAn), Cx<float>{-pAc.z, -pAc.w}),
                                     ndk, hi_c(pBc), lo_c(pBc), hi_c(up));
      uA = pack4(u0, u1);
      UAl[tid] = make_float2(u0.re, u0.im);
      UAh[tid] = make_float2(u1.re, u1.im);
    }
    if (need_uB) {
      // u_B(t+1) = p_B(t+1) + (dm - e^{i phi_B(t)}) p_B(t) - dk [p_A(i,j) + p_A(i+1,j) + p_A(i,j+1)](t+1)
      // (of the right pair only its first cell is read)
      const Cx<float> right = lo_of(SA + JN * NT + nip);
      const float4 down = SA[JN * NT + njp];
      const Cx<float> u0 = hopsum_x2(cfma(Cx<float>{dm - eb_c0.re, -eb_c0.im}, lo_c(pBc), lo_c(pBn)), ndk, lo_c(pAn),
                                     hi_c(pAn), lo_c(down));
      const Cx<float> u1 = hopsum_x2(cfma(Cx<float>{dm - eb_c1.re, -eb_c1.im}, hi_c(pBc), hi_c(pBn)), ndk,
                                     hi_c(pAn), right, hi_c(down));
      uBn = pack4(u0, u1);
      UBl[((J + 1) & 1) * NT + tid] = make_float2(u0.re, u0.im);
      UBh[((J + 1) & 1) * NT + tid] = make_float2(u1.re, u1.im);
    }
    if constexpr (OUT) {
      __syncthreads();
      if (in_tile) {
        const int KB = (J & 1) * NT;  // u_B(t)
        // of the left pair only its second cell, of the right pair only its first is read
        const float2 blh = UBh[KB + nim], arl = UAl[nip];
        const Cx<float> bl{blh.x, blh.y}, ar{arl.x, arl.y};
        const float2 bul = UBl[KB + njm], buh = UBh[KB + njm], adl = UAl[njp], adh = UAh[njp];
        const float4 bu = make_float4(bul.x, bul.y, buh.x, buh.y), ad = make_float4(adl.x, adl.y, adh.x, adh.y);
        // (M u)_A(t) = -u_A(t) + (e^{i phi_A(t)} - dm) u_A(t-1) - dk [u_B(i,j) + u_B(i-1,j) + u_B(i,j-1)](t)
        Cx<float> oA0 = hopsum_x2(cfma(Cx<float>{ea_c0.re - dm, ea_c0.im}, lo_c(uA_prev), Cx<float>{-uA.x, -uA.y}),
                                  ndk, lo_c(uB_cur), bl, lo_c(bu));
        Cx<float> oA1 = hopsum_x2(cfma(Cx<float>{ea_c1.re - dm, ea_c1.im}, hi_c(uA_prev), Cx<float>{-uA.z, -uA.w}),
                                  ndk, hi_c(uB_cur), lo_c(uB_cur), hi_c(bu));
        // (M u)_B(t) = u_B(t) + (dm - e^{-i phi_B(t)}) u_B(t+1) - dk [u_A(i,j) + u_A(i+1,j) + u_A(i,j+1)](t)
        Cx<float> oB0 = hopsum_x2(cfma(Cx<float>{dm - eb_c0.re, eb_c0.im}, lo_c(uBn), lo_c(uB_cur)), ndk, lo_c(uA),
                                  hi_c(uA), lo_c(ad));
        Cx<float> oB1 = hopsum_x2(cfma(Cx<float>{dm - eb_c1.re, eb_c1.im}, hi_c(uBn), hi_c(uB_cur)), ndk, hi_c(uA),
                                  ar, hi_c(ad));
        float4 oA = pack4(oA0, oA1), oB = pack4(oB0, oB1);
        oA.x = fmaf(sigma, pAc.x, oA.x);
        oA.y = fmaf(sigma, pAc.y, oA.y);
        oA.z = fmaf(sigma, pAc.z, oA.z);
        oA.w = fmaf(sigma, pAc.w, oA.w);
        oB.x = fmaf(sigma, pBc.x, oB.x);
        oB.y = fmaf(sigma, pBc.y, oB.y);
        oB.z = fmaf(sigma, pBc.z, oB.z);
        oB.w = fmaf(sigma, pBc.w, oB.w);
        og[toff_out] = oA;
        og[toff_out + H] = oB;
      }
      toff_out += V;
    }
    uA_prev = uA;
    uB_cur = uBn;
    ea_c0 = ea_n0;
    ea_c1 = ea_n1;
    pAc = pAn;
    pBc = pBn;
  };

  step(IC<0>{}, std::false_type{}, 0);
  for (int k0 = 0;; k0 += S) {
    if (k0 + 1 > T) break;
    step(IC<1 % S>{}, std::true_type{}, k0 + 1);
    if (k0 + 2 > T) break;
    step(IC<2 % S>{}, std::true_type{}, k0 + 2);
    if (k0 + 3 > T) break;
    step(IC<3 % S>{}, std::true_type{}, k0 + 3);
    if constexpr (S > 4) {
      if (k0 + 4 > T) break;
      step(IC<4 % S>{}, std::true_type{}, k0 + 4);
      if (k0 + 5 > T) break;
      step(IC<5 % S>{}, std::true_type{}, k0 + 5);
    }
    if constexpr (S > 6) {
      if (k0 + 6 > T) break;
      step(IC<6 % S>{}, std::true_type{}, k0 + 6);
      if (k0 + 7 > T) break;
      step(IC<7 % S>{}, std::true_type{}, k0 + 7);
    }
    if (k0 + S > T) break;
    step(IC<0>{}, std::true_type{}, k0 + S);
  }
  cp_async_wait<0>();
}

// ---------------------------------------------------------------------------
// Host side

static int fused_smem_bytes(int NT, int S, int vbytes, int pbytes) {
  return (2 * S + 6) * NT * vbytes + 2 * S * NT * pbytes;
}

template <typename R>
static int fused_threads_of(const FusedShape& fs) {
  return fs.pairs ? (fs.Ti / 2 + 2) * (fs.Tj + 2) : (fs.Ti + 2) * (fs.Tj + 2);
}

template <typename R>
static int fused_smem_of(const FusedShape& fs) {
  const int NT = fused_threads_of<R>(fs), S = fs.D + 2;
  if (fs.pairs) return (2 * S + 3) * NT * 16 + 2 * S * NT * 8;
  return fused_smem_bytes(NT, S, (int)sizeof(V2<R>), (int)sizeof(typename FusedPhase<R>::type::T));
}

// The prefetch depths with a compiled kernel (the ring of D + 2 slots is a
// multiple of 4).
static bool fused_depth_ok(int D) { return D == 2 || D == 6; }

FusedShape make_fused_shape(const Geo& g, int Ti, int Tj, int Tt, int D, int pairs) {
  FusedShape fs;
  fs.D = D;
  fs.pairs = pairs;
  fs.Ti = std::max(1, std::min(Ti, g.n));
  fs.Tj = std::max(1, std::min(Tj, g.m));
  fs.Tt = std::max(1, std::min(Tt, g.nt));
  fs.tiles_i = (g.n + fs.Ti - 1) / fs.Ti;
  fs.tiles_j = (g.m + fs.Tj - 1) / fs.Tj;
  fs.tiles_t = (g.nt + fs.Tt - 1) / fs.Tt;
  return fs;
}

template <typename R>
bool fused_ok(const Geo& g, const FusedShape& fs) {
  const int NT = fused_threads_of<R>(fs);
  if (!fused_depth_ok(fs.D)) return false;
  if (sizeof(R) == 8 && fs.D != 2) return false;  // FP64: depth 2 only (the deeper ring spills registers)
  if (fs.pairs) {
    // FP32 only; pairs of cells stay aligned in memory and inside the box
    if (sizeof(R) != 4 || (g.n & 1) || (fs.Ti & 1) || fs.Ti < 2 || NT > kPairMaxThreads) return false;
  } else if (NT > fused_max_threads<R>()) {
    return false;
  }
  if (fused_smem_of<R>(fs) > 227 * 1024) return false;
  const long long blocks = (long long)fs.tiles_i * fs.tiles_j * fs.tiles_t;
  return blocks >= 1 && blocks < (1LL << 31);
}

template <typename R>
static void fused_raw_launch(hmc_ctx* c, const Geo& g, const FusedShape& fs, R dm, R sigma, const V2<R>* in,
                             V2<R>* out) {
  static unsigned long long attr_set = 0;  // one bit per device
  const int smem = fused_smem_of<R>(fs);
  const unsigned long long bit = 1ull << (c->device & 63);
  if (!(attr_set & bit)) {
    cudaFuncSetAttribute(k_mmdag_fused<R, 2>, cudaFuncAttributeMaxDynamicSharedMemorySize, 227 * 1024);
    if constexpr (sizeof(R) == 4)
      cudaFuncSetAttribute(k_mmdag_fused<R, 6>, cudaFuncAttributeMaxDynamicSharedMemorySize, 227 * 1024);
    attr_set |= bit;
  }
  const int NT = fused_threads_of<R>(fs);
  const int threads = (NT + 31) / 32 * 32;
  const int blocks = fs.tiles_i * fs.tiles_j * fs.tiles_t;
  if constexpr (sizeof(R) == 4) {
    if (fs.pairs) {
      static unsigned long long pattr = 0;
      if (!(pattr & bit)) {
        cudaFuncSetAttribute(k_mmdag_fused_pairs<2>, cudaFuncAttributeMaxDynamicSharedMemorySize, 227 * 1024);
        cudaFuncSetAttribute(k_mmdag_fused_pairs<6>, cudaFuncAttributeMaxDynamicSharedMemorySize, 227 * 1024);
        pattr |= bit;
      }
      const float2* ph2 = (const float2*)c->ws[WS_PHI32];
      if (fs.D == 2)
        k_mmdag_fused_pairs<2><<<blocks, threads, smem, c->stream>>>(g, fs, ph2, dm, sigma, (const float4*)in,
                                                                     (float4*)out);
      else
        k_mmdag_fused_pairs<6><<<blocks, threads, smem, c->stream>>>(g, fs, ph2, dm, sigma, (const float4*)in,
                                                                     (float4*)out);
      return;
    }
  }
  const typename FusedPhase<R>::type::T* ph;
  if constexpr (sizeof(R) == 4)
    ph = (const float*)c->ws[WS_PHI32];
  else
    ph = (const double2*)c->ws[WS_E];
  if constexpr (sizeof(R) == 8) {
    k_mmdag_fused<R, 2><<<blocks, threads, smem, c->stream>>>(g, fs, ph, dm, sigma, in, out);
  } else if (fs.D == 2) {
    k_mmdag_fused<R, 2><<<blocks, threads, smem, c->stream>>>(g, fs, ph, dm, sigma, in, out);
  } else {
    k_mmdag_fused<R, 6><<<blocks, threads, smem, c->stream>>>(g, fs, ph, dm, sigma, in, out);
  }
}

// Launch-shape tuner: every candidate tile (Ti + 2 threads per box row, Tj
// rows, Tt time slices) is timed over a few applications of this call's
// operands; the fastest is kept for the context and precision. Where the
// operands (p, phi, the result) do not fit in L2 together, each timed
// application starts from a cold L2 (the result vector and the M^dagger
// scratch vector are rewritten first), as in a solve whose vectors stream
// from memory; otherwise the applications run back to back.
template <typename R>
static hmc_status tune_fused(hmc_ctx* c, const Geo& g, R dm, R sigma, const V2<R>* in, V2<R>* out) {
  const int pi = sizeof(R) == 4 ? 0 : 1;
  if (c->fused_tuned[pi]) return HMC_OK;
  c->fused_tuned[pi] = true;
  std::vector<FusedShape> cands;
  const bool aligned16 = ((uintptr_t)in % 16 == 0) && ((uintptr_t)out % 16 == 0);
  // time ranges: short ones, and the lattice's time extent in one, two or
  // three parts (whichever fills the SMs' block slots best)
  const int tts[6] = {4, 8, 16, (g.nt + 2) / 3, (g.nt + 1) / 2, g.nt};
  for (int pairs : {1, 0})
    for (int TX : {16, 32, 64})
      for (int Tj : {4, 6, 8, 10, 14, 30})
        for (int Tt : tts)
          for (int D : {2, 6}) {
            if (pairs && !aligned16) continue;
            if (!pairs && TX == 16) continue;
            // pairs: TX threads per box row carry 2 TX cells, Ti = 2 (TX - 2)
            FusedShape fs = make_fused_shape(g, pairs ? 2 * (TX - 2) : TX - 2, Tj, Tt, D, pairs);
            if (pairs && (fs.Ti & 1)) continue;
            if (!fused_ok<R>(g, fs)) continue;
            bool dup = false;
            for (const auto& o : cands)
              dup = dup || (o.Ti == fs.Ti && o.Tj == fs.Tj && o.Tt == fs.Tt && o.D == fs.D && o.pairs == fs.pairs);
            if (!dup) cands.push_back(fs);
          }
  if (cands.empty()) return fail(c, HMC_ERR_INVALID, "no fused M M^dagger tile fits");
  c->fshape[pi] = cands[0];
  if (cands.size() == 1) return HMC_OK;
  int l2 = 0;
  cudaDeviceGetAttribute(&l2, cudaDevAttrL2CacheSize, c->device);
  const size_t vb = sizeof(V2<R>) * (size_t)g.N;
  bool cold = (2 * vb + (sizeof(R) == 4 ? 4 : 16) * (size_t)g.N) > (size_t)l2;
  void* scratch = nullptr;
  if (cold && ws_get(c, sizeof(R) == 4 ? WS_U32 : WS_U64, vb, &scratch) != HMC_OK) {
    cold = false;  // no room for the scratch vector: the candidates are timed back to back
    c->err.clear();
  }
  cudaEvent_t ev[2][5];
  for (auto& row : ev)
    for (auto& e : row) HMC_CUDA(c, cudaEventCreate(&e));
  float best = 1e30f;
  for (const FusedShape& fs : cands) {
    fused_raw_launch<R>(c, g, fs, dm, sigma, in, out);  // warm
    for (int rep = 0; rep < 5; ++rep) {
      if (cold) {
        HMC_CUDA(c, cudaMemsetAsync(out, 0, vb, c->stream));
        HMC_CUDA(c, cudaMemsetAsync(scratch, 0, vb, c->stream));
      }
      HMC_CUDA(c, cudaEventRecord(ev[0][rep], c->stream));
      fused_raw_launch<R>(c, g, fs, dm, sigma, in, out);
      HMC_CUDA(c, cudaEventRecord(ev[1][rep], c->stream));
    }
    HMC_CUDA(c, cudaEventSynchronize(ev[1][4]));
    HMC_CUDA(c, cudaGetLastError());
    float sum = 0.f;
    for (int rep = 0; rep < 5; ++rep) {
      float ms = 0.f;
      cudaEventElapsedTime(&ms, ev[0][rep], ev[1][rep]);
      sum += ms;
    }
    if (sum < best) {
      best = sum;
      c->fshape[pi] = fs;
    }
  }
  for (auto& row : ev)
    for (auto& e : row) cudaEventDestroy(e);
  return HMC_OK;
}

template <typename R>
hmc_status mmdag_fused_launch(hmc_ctx* c, const Geo& g, R dm, R sigma, const V2<R>* in, V2<R>* out) {
  if (!c->capturing) HMC_TRY(tune_fused<R>(c, g, dm, sigma, in, out));
  const int pi = sizeof(R) == 4 ? 0 : 1;
  FusedShape fs = c->fshape[pi];
  if (!fused_ok<R>(g, fs) || fs.Ti < 1) return fail(c, HMC_ERR_INVALID, "fused M M^dagger shape not tuned");
  // the two-cell kernel needs 16-byte aligned vectors; any other call takes
  // the one-cell kernel on a tile that always fits
  if (fs.pairs && (((uintptr_t)in % 16) || ((uintptr_t)out % 16))) fs = make_fused_shape(g, 30, 8, 16, 2, 0);
  return launch(c, sizeof(R) == 4 ? K_MMDAG_FUSED32 : K_MMDAG_FUSED64,
                [&] { fused_raw_launch<R>(c, g, fs, dm, sigma, in, out); });
}

template hmc_status mmdag_fused_launch<float>(hmc_ctx*, const Geo&, float, float, const float2*, float2*);
template hmc_status mmdag_fused_launch<double>(hmc_ctx*, const Geo&, double, double, const double2*, double2*);

hmc_status set_fused_shape(hmc_ctx* c, int prec, int Ti, int Tj, int Tt, int D, int pairs) {
  const int pi = prec == 32 ? 0 : 1;
  const FusedShape fs = make_fused_shape(c->geo, Ti, Tj, Tt, D, pairs);
  const bool ok = prec == 32 ? fused_ok<float>(c->geo, fs) : fused_ok<double>(c->geo, fs);
  if (!ok) return fail(c, HMC_ERR_INVALID, "fused tile does not fit (threads or shared memory)");
  c->fshape[pi] = fs;
  c->fused_tuned[pi] = true;
  return HMC_OK;
}

}  // namespace hmc
