// The fermion operator M[phi; m_s] of Eq. ferm_op and its adjoint, as device
// code. One thread handles one cell-time q: the A row q and the B row H + q.
//
//   (M u)_A(x,t)  = -u_A(x,t) + s (e^{+i phi_A(x,t)} - delta m_s) u_A(x,t-1)
//                   - delta kappa [u_B(i,j) + u_B(i-1,j) + u_B(i,j-1)](t)
//   (M u)_B(x,t)  = +u_B(x,t) - s (e^{-i phi_B(x,t)} - delta m_s) u_B(x,t+1)
//                   - delta kappa [u_A(i,j) + u_A(i+1,j) + u_A(i,j+1)](t)
//   (M^+ p)_A(x,t) = -p_A(x,t) + s (e^{-i phi_A(x,t+1)} - delta m_s) p_A(x,t+1) - delta kappa sum_B
//   (M^+ p)_B(x,t) = +p_B(x,t) - s (e^{+i phi_B(x,t-1)} - delta m_s) p_B(x,t-1) - delta kappa sum_A
// with s = -1 on the hop that wraps around the time circle (anti-periodic).
#pragma once

#include "common.cuh"

namespace hmc {

// e^{i phi_k}. FP64: read from a table built once per field. FP32: computed
// from the field rounded to float, with the argument reduced to [-pi, pi] and
// the hardware sine/cosine (absolute error about 4e-7 there), which is below
// what the single-precision inner solver needs.
template <typename R>
struct Phase;

template <>
struct Phase<double> {
  const double2* E;
  __device__ __forceinline__ Cx<double> operator()(int k) const {
    double2 e = E[k];
    return Cx<double>{e.x, e.y};
  }
};

template <>
struct Phase<float> {
  const float* phi;
  __device__ __forceinline__ Cx<float> operator()(int k) const {
    float s, c;
    __sincosf(phi[k], &s, &c);  // phi in [-pi, pi] (phi_to_f32)
    return Cx<float>{c, s};
  }
};

// c + z v with fused multiply-adds.
template <typename R>
__device__ __forceinline__ Cx<R> cfma(Cx<R> z, Cx<R> v, Cx<R> c) {
  Cx<R> o;
  o.re = fma(z.re, v.re, fma(-z.im, v.im, c.re));
  o.im = fma(z.re, v.im, fma(z.im, v.re, c.im));
  return o;
}

// t - dk (a + b + c)
template <typename R>
__device__ __forceinline__ Cx<R> hopsum(Cx<R> t, R dk, Cx<R> a, Cx<R> b, Cx<R> c) {
  Cx<R> o;
  o.re = fma(-dk, a.re + b.re + c.re, t.re);
  o.im = fma(-dk, a.im + b.im + c.im, t.im);
  return o;
}

template <typename R>
struct PairOut {
  Cx<R> a, b;
};

// M^dagger applied at the cell-time of nb, reading p (precision R); PH is any
// functor returning e^{i phi_k}.
template <typename R, typename PH = Phase<R>>
__device__ __forceinline__ PairOut<R> mdag_pair(const Geo& g, const PH& ph, R dm,
                                                const typename Vec2<R>::type* __restrict__ p,
                                                const Nbr& nb) {
  const int H = g.H;
  const R dk = geo_dk(g, R(0));
  Cx<R> pa = ld<R>(p, nb.q), pb = ld<R>(p, H + nb.q);
  // A row: time partner (x, t+1), phase of A at t+1, conjugated
  Cx<R> ea = ph(nb.tp);
  Cx<R> za = cneg_if(Cx<R>{ea.re - dm, -ea.im}, nb.wrap_tp);
  Cx<R> ta = cfma(za, ld<R>(p, nb.tp), Cx<R>{-pa.re, -pa.im});
  Cx<R> oa = hopsum(ta, dk, pb, ld<R>(p, H + nb.im1), ld<R>(p, H + nb.jm1));
  // B row: time partner (x, t-1), phase of B at t-1; the hop carries a minus sign
  Cx<R> eb = ph(H + nb.tm);
  Cx<R> zb = cneg_if(Cx<R>{dm - eb.re, -eb.im}, nb.wrap_tm);
  Cx<R> tb = cfma(zb, ld<R>(p, H + nb.tm), pb);
  Cx<R> ob = hopsum(tb, dk, pa, ld<R>(p, nb.ip1), ld<R>(p, nb.jp1));
  return PairOut<R>{oa, ob};
}

// M^dagger at the cell-time of nb of the vector returned by the loader L, with
// the time-hop factors za (A row) and zb (B row) already formed; used where
// the same stencil is applied to two vectors.
template <typename R, typename LD>
__device__ __forceinline__ PairOut<R> mdag_pair_ld(const Geo& g, Cx<R> za, Cx<R> zb, R dk, const Nbr& nb,
                                                   LD L) {
  const int H = g.H;
  Cx<R> pa = L(nb.q), pb = L(H + nb.q);
  Cx<R> ta = cfma(za, L(nb.tp), Cx<R>{-pa.re, -pa.im});
  Cx<R> oa = hopsum(ta, dk, pb, L(H + nb.im1), L(H + nb.jm1));
  Cx<R> tb = cfma(zb, L(H + nb.tm), pb);
  Cx<R> ob = hopsum(tb, dk, pa, L(nb.ip1), L(nb.jp1));
  return PairOut<R>{oa, ob};
}

// M at the cell-time of nb of the vector returned by the loader L (phases
// from ph); used where the loads need a particular cache policy.
template <typename R, typename PH, typename LD>
__device__ __forceinline__ PairOut<R> m_pair_ld(const Geo& g, const PH& ph, R dm, const Nbr& nb, LD L) {
  const int H = g.H;
  const R dk = geo_dk(g, R(0));
  Cx<R> ua = L(nb.q), ub = L(H + nb.q);
  Cx<R> ea = ph(nb.q);
  Cx<R> za = cneg_if(Cx<R>{ea.re - dm, ea.im}, nb.wrap_tm);
  Cx<R> ta = cfma(za, L(nb.tm), Cx<R>{-ua.re, -ua.im});
  Cx<R> oa = hopsum(ta, dk, ub, L(H + nb.im1), L(H + nb.jm1));
  Cx<R> eb = ph(H + nb.q);
  Cx<R> zb = cneg_if(Cx<R>{dm - eb.re, eb.im}, nb.wrap_tp);
  Cx<R> tb = cfma(zb, L(H + nb.tp), ub);
  Cx<R> ob = hopsum(tb, dk, ua, L(nb.ip1), L(nb.jp1));
  return PairOut<R>{oa, ob};
}

// M applied at the cell-time of nb, reading u (precision R).
template <typename R, typename PH = Phase<R>>
__device__ __forceinline__ PairOut<R> m_pair(const Geo& g, const PH& ph, R dm,
                                             const typename Vec2<R>::type* __restrict__ u,
                                             const Nbr& nb) {
  const int H = g.H;
  const R dk = geo_dk(g, R(0));
  Cx<R> ua = ld<R>(u, nb.q), ub = ld<R>(u, H + nb.q);
  // A row: (e^{i phi_A(t)} - dm) u_A(t-1)
  Cx<R> ea = ph(nb.q);
  Cx<R> za = cneg_if(Cx<R>{ea.re - dm, ea.im}, nb.wrap_tm);
  Cx<R> ta = cfma(za, ld<R>(u, nb.tm), Cx<R>{-ua.re, -ua.im});
  Cx<R> oa = hopsum(ta, dk, ub, ld<R>(u, H + nb.im1), ld<R>(u, H + nb.jm1));
  // B row: -(e^{-i phi_B(t)} - dm) u_B(t+1)
  Cx<R> eb = ph(H + nb.q);
  Cx<R> zb = cneg_if(Cx<R>{dm - eb.re, eb.im}, nb.wrap_tp);
  Cx<R> tb = cfma(zb, ld<R>(u, H + nb.tp), ub);
  Cx<R> ob = hopsum(tb, dk, ua, ld<R>(u, nb.ip1), ld<R>(u, nb.jp1));
  return PairOut<R>{oa, ob};
}

}  // namespace hmc
