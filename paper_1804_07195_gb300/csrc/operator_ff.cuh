// The row pairs of the fermion operator M[phi; m_s] and of M^dagger (Eq.
// ferm_op) in float-float arithmetic (ffloat.cuh): FP64-accurate applications
// on the FP32 pipe. Same structure as the pair stencils of operator.cuh: one
// cell-time q, its A row q and its B row H + q, neighbours from Nbr, the
// anti-periodic sign on the hop that wraps around the time circle:
//
//   (M u)_A(x,t)   = -u_A(x,t) + s (e^{+i phi_A(x,t)} - delta m_s) u_A(x,t-1) - delta kappa sum_B
//   (M u)_B(x,t)   = +u_B(x,t) - s (e^{-i phi_B(x,t)} - delta m_s) u_B(x,t+1) - delta kappa sum_A
//   (M^+ p)_A(x,t) = -p_A(x,t) + s (e^{-i phi_A(x,t+1)} - delta m_s) p_A(x,t+1) - delta kappa sum_B
//   (M^+ p)_B(x,t) = +p_B(x,t) - s (e^{+i phi_B(x,t-1)} - delta m_s) p_B(x,t-1) - delta kappa sum_A
//
// The loader L(k) returns site k of the input vector and the phase functor
// E(k) returns e^{i phi_k}, both as complex float-float values. Host and
// device code: the host test runs these very functions over whole lattices.
#pragma once

#include "common.cuh"
#include "ffloat.cuh"

namespace hmc {
namespace ffa {

struct CFF {
  FF re, im;
};

__host__ __device__ __forceinline__ CFF cff_from(double re, double im) {
  return CFF{ff_from_double(re), ff_from_double(im)};
}

__host__ __device__ __forceinline__ CFF cff_neg(CFF a) { return CFF{ff_neg(a.re), ff_neg(a.im)}; }

__host__ __device__ __forceinline__ CFF cff_neg_if(CFF a, bool neg) { return neg ? cff_neg(a) : a; }

// c + z v
__host__ __device__ __forceinline__ CFF cff_fma(CFF z, CFF v, CFF c) {
  const FF re = ff_add(c.re, ff_add(ff_mul(z.re, v.re), ff_neg(ff_mul(z.im, v.im))));
  const FF im = ff_add(c.im, ff_add(ff_mul(z.re, v.im), ff_mul(z.im, v.re)));
  return CFF{re, im};
}

// t - dk (a + b + c)
__host__ __device__ __forceinline__ CFF cff_hopsum(CFF t, FF dk, CFF a, CFF b, CFF c) {
  const FF sr = ff_add(ff_add(a.re, b.re), c.re), si = ff_add(ff_add(a.im, b.im), c.im);
  return CFF{ff_add(t.re, ff_neg(ff_mul(dk, sr))), ff_add(t.im, ff_neg(ff_mul(dk, si)))};
}

struct PairFF {
  CFF a, b;
};

// M at the cell-time of nb; dm = delta m_s, dk = delta kappa.
template <typename PH, typename LD>
__host__ __device__ __forceinline__ PairFF m_pair_ff(int H, const Nbr& nb, FF dm, FF dk, const PH& E, LD L) {
  const CFF ua = L(nb.q), ub = L(H + nb.q);
  // A row: (e^{i phi_A(t)} - dm) u_A(t-1)
  const CFF ea = E(nb.q);
  const CFF za = cff_neg_if(CFF{ff_add(ea.re, ff_neg(dm)), ea.im}, nb.wrap_tm);
  const CFF ta = cff_fma(za, L(nb.tm), cff_neg(ua));
  const CFF oa = cff_hopsum(ta, dk, ub, L(H + nb.im1), L(H + nb.jm1));
  // B row: -(e^{-i phi_B(t)} - dm) u_B(t+1) = (dm - cos, sin) u_B(t+1)
  const CFF eb = E(H + nb.q);
  const CFF zb = cff_neg_if(CFF{ff_add(dm, ff_neg(eb.re)), eb.im}, nb.wrap_tp);
  const CFF tb = cff_fma(zb, L(H + nb.tp), ub);
  const CFF ob = cff_hopsum(tb, dk, ua, L(nb.ip1), L(nb.jp1));
  return PairFF{oa, ob};
}

// M^dagger at the cell-time of nb.
template <typename PH, typename LD>
__host__ __device__ __forceinline__ PairFF mdag_pair_ff(int H, const Nbr& nb, FF dm, FF dk, const PH& E, LD L) {
  const CFF pa = L(nb.q), pb = L(H + nb.q);
  // A row: time partner (x, t+1), phase of A at t+1, conjugated
  const CFF ea = E(nb.tp);
  const CFF za = cff_neg_if(CFF{ff_add(ea.re, ff_neg(dm)), ff_neg(ea.im)}, nb.wrap_tp);
  const CFF ta = cff_fma(za, L(nb.tp), cff_neg(pa));
  const CFF oa = cff_hopsum(ta, dk, pb, L(H + nb.im1), L(H + nb.jm1));
  // B row: time partner (x, t-1), phase of B at t-1; the hop carries a minus sign
  const CFF eb = E(H + nb.tm);
  const CFF zb = cff_neg_if(CFF{ff_add(dm, ff_neg(eb.re)), ff_neg(eb.im)}, nb.wrap_tm);
  const CFF tb = cff_fma(zb, L(H + nb.tm), pb);
  const CFF ob = cff_hopsum(tb, dk, pa, L(nb.ip1), L(nb.jp1));
  return PairFF{oa, ob};
}

}  // namespace ffa
}  // namespace hmc
