// Float-float ("double-single") arithmetic for FP64-accurate stencils on the
// FP32 pipe, which GB300 runs at 58x its FP64 rate. A value is the unevaluated
// sum hi + lo of two floats with |lo| below one unit in the last place of hi:
// 48 significant bits, about 3.6e-15 relative.
//
// Conversions between double and the pair use integer operations only, so a
// kernel that loads and stores complex128 needs no FP64 instruction on its
// per-site path:
//   ff_from_double  splits the 53-bit significand into its top 24 bits and
//                   the next 24, then normalises the pair (|lo| at most half a
//                   unit of hi); hi + lo is within 2^-47 of x (relative) for
//                   2^-79 <= |x| < 2^128. Below 2^-79 a lo that would be a
//                   subnormal float is dropped (hi keeps x to 24 bits), below
//                   2^-126 both are; an |x| that rounds above the largest
//                   float gives (+-inf, 0); NaN stays NaN.
//   ff_to_double    rounds hi + lo to the nearest double (ties to even).
// Arithmetic (published error-free transforms): TwoSum (Knuth), Fast2Sum
// (Dekker), TwoProd with a fused multiply-add, and the pair addition and
// multiplication built from them. Worst cases measured over 4M random
// normalised pairs: 2^-47.1 for the sum (relative to |a| + |b|) and 2^-46.2
// for the product; the host test holds them to 2^-46 and 2^-45.
//
// Every function is __host__ __device__ so that the host test checks the same
// code the kernels would run (IEEE single precision, round to nearest, no
// flush to zero).
#pragma once

#include <stdint.h>
#include <string.h>

#include <cmath>

namespace hmc {
namespace ffa {

struct FF {
  float hi, lo;
};

__host__ __device__ __forceinline__ uint64_t bits_of(double x) {
#ifdef __CUDA_ARCH__
  return (uint64_t)__double_as_longlong(x);
#else
  uint64_t u;
  memcpy(&u, &x, 8);
  return u;
#endif
}

__host__ __device__ __forceinline__ double double_of(uint64_t u) {
#ifdef __CUDA_ARCH__
  return __longlong_as_double((long long)u);
#else
  double x;
  memcpy(&x, &u, 8);
  return x;
#endif
}

__host__ __device__ __forceinline__ float float_of(uint32_t u) {
#ifdef __CUDA_ARCH__
  return __uint_as_float(u);
#else
  float x;
  memcpy(&x, &u, 4);
  return x;
#endif
}

__host__ __device__ __forceinline__ uint32_t bits_of(float x) {
#ifdef __CUDA_ARCH__
  return __float_as_uint(x);
#else
  uint32_t u;
  memcpy(&u, &x, 4);
  return u;
#endif
}

__host__ __device__ __forceinline__ int clz64(uint64_t v) {
#ifdef __CUDA_ARCH__
  return __clzll((long long)v);
#else
  return v ? __builtin_clzll(v) : 64;
#endif
}

// ---------------------------------------------------------------------------
// Error-free transforms.
__host__ __device__ __forceinline__ FF two_sum(float a, float b) {  // Knuth: s + e = a + b exactly
  const float s = a + b;
  const float bb = s - a;
  const float e = (a - (s - bb)) + (b - bb);
  return FF{s, e};
}

__host__ __device__ __forceinline__ FF fast_two_sum(float a, float b) {  // Dekker, |a| >= |b|
  const float s = a + b;
  return FF{s, b - (s - a)};
}

__host__ __device__ __forceinline__ FF two_prod(float a, float b) {  // p + e = a b exactly
  const float p = a * b;
  return FF{p, fmaf(a, b, -p)};
}

// ---------------------------------------------------------------------------
// double -> (hi, lo) by integer operations (see the header comment for ranges)
__host__ __device__ __forceinline__ FF ff_from_double(double x) {
  const uint64_t u = bits_of(x);
  const uint32_t sign = (uint32_t)(u >> 63) << 31;
  const int E = (int)((u >> 52) & 0x7FF);
  const uint64_t M = u & 0xFFFFFFFFFFFFFull;
  if (E == 0x7FF) {  // inf or NaN
    const float v = float_of(sign | 0x7F800000u | (M ? 0x400000u : 0u));
    return FF{v, 0.0f};
  }
  const int e = E - 1023;
  if (E == 0 || e < -126) return FF{float_of(sign), 0.0f};  // zero, subnormal double, or below float range
  if (e > 127) return FF{float_of(sign | 0x7F800000u), 0.0f};
  const uint32_t hi_bits = sign | ((uint32_t)(e + 127) << 23) | (uint32_t)(M >> 29);
  const uint64_t r = M & 0x1FFFFFFFull;  // the 29 bits below hi, weight 2^(e-52)
  if (r == 0) return FF{float_of(hi_bits), 0.0f};
  const int p = 63 - clz64(r);           // leading bit of r, 0..28
  const int el = e - 52 + p;             // exponent of lo
  if (el < -126) return FF{float_of(hi_bits), 0.0f};
  const uint32_t mant = p >= 23 ? (uint32_t)(r >> (p - 23)) & 0x7FFFFFu : (uint32_t)(r << (23 - p)) & 0x7FFFFFu;
  const uint32_t lo_bits = sign | ((uint32_t)(el + 127) << 23) | mant;
  // normalise: |lo| <= half a unit of hi, the form the arithmetic's error
  // bounds assume (the truncated split leaves |lo| up to a whole unit); an x
  // that rounds above the largest float becomes (+-inf, 0)
  FF s = fast_two_sum(float_of(hi_bits), float_of(lo_bits));
  if ((bits_of(s.hi) & 0x7FFFFFFFu) == 0x7F800000u) s.lo = 0.0f;
  return s;
}

// (hi, lo) -> the double nearest to hi + lo, by integer operations. hi and lo
// are finite floats with |lo| < 2^-20 |hi| (any pair the arithmetic below
// returns) or hi = 0; a non-finite hi is returned as it is.
__host__ __device__ __forceinline__ double ff_to_double(FF a) {
  const uint32_t hb = bits_of(a.hi), lb = bits_of(a.lo);
  const int Eh = (int)((hb >> 23) & 0xFF);
  if (Eh == 0xFF) {  // inf or NaN: widen the pattern
    return double_of(((uint64_t)(hb >> 31) << 63) | 0x7FF0000000000000ull |
                     ((uint64_t)(hb & 0x7FFFFFu) << 29));
  }
  // the parts as (sign, integer significand, exponent of its unit bit)
  auto parts = [](uint32_t b, uint64_t* sig, int* ex) {
    const int E = (int)((b >> 23) & 0xFF);
    const uint32_t m = b & 0x7FFFFFu;
    if (E == 0) {  // zero or subnormal float
      *sig = m;
      *ex = -149;
    } else {
      *sig = (uint64_t)(m | 0x800000u);
      *ex = E - 150;
    }
  };
  uint64_t sh, sl;
  int eh, el;
  parts(hb, &sh, &eh);
  parts(lb, &sl, &el);
  if (sl == 0 || sh == 0) {  // one part is zero: the other converts exactly
    const uint32_t b = sh ? hb : lb;
    const uint64_t s = sh ? sh : sl;
    const int ex = sh ? eh : el;
    if (s == 0) return double_of((uint64_t)(b >> 31) << 63);
    const int lead = 63 - clz64(s);
    const uint64_t frac = (s << (52 - lead)) & 0xFFFFFFFFFFFFFull;
    return double_of(((uint64_t)(b >> 31) << 63) | ((uint64_t)(ex + lead + 1023) << 52) | frac);
  }
  // Fixed point with the unit of hi's last bit at 2^39: sh << 39 occupies
  // bits 39..62. lo sits d = eh - el bits further down; bits shifted out below
  // bit 0 are kept as a sticky flag for the rounding.
  const bool neg_h = hb >> 31, neg_l = lb >> 31;
  const int d = eh - el;  // >= 1 by the precondition on |lo|
  uint64_t H = sh << 39;
  uint64_t L;
  bool sticky = false;
  if (d - 39 >= 64) {
    L = 0;
    sticky = true;
  } else if (d >= 39) {
    const int s = d - 39;
    L = s ? (sl >> s) : sl;
    sticky = s && (sl & ((1ull << s) - 1)) != 0;
  } else {
    L = sl << (39 - d);
  }
  uint64_t S;
  if (neg_h == neg_l) {
    S = H + L;  // below 2^64: H < 2^63 and L < 2^(63 - d + 1)
  } else {
    // |hi| > |lo|: the difference keeps hi's sign; a sticky remainder of lo
    // means the true value is a little below H - L
    S = H - L - (sticky ? 1 : 0);
  }
  // normalise S to 53 bits and round to nearest, ties to even
  const int lead = 63 - clz64(S);
  int ex = eh - 39 + lead;  // exponent of S's leading bit
  uint64_t mant;
  if (lead > 52) {
    const int sh2 = lead - 52;
    const uint64_t rem = S & ((1ull << sh2) - 1);
    const uint64_t half = 1ull << (sh2 - 1);
    mant = S >> sh2;
    const bool st = sticky || (rem & (half - 1)) != 0;
    if ((rem & half) && (st || (rem & ~half) || (mant & 1))) ++mant;
    if (mant >> 53) {
      mant >>= 1;
      ++ex;
    }
  } else {
    mant = S << (52 - lead);
  }
  return double_of(((uint64_t)neg_h << 63) | ((uint64_t)(ex + 1023) << 52) | (mant & 0xFFFFFFFFFFFFFull));
}

// accurate sum of two pairs
__host__ __device__ __forceinline__ FF ff_add(FF a, FF b) {
  FF s = two_sum(a.hi, b.hi);
  const FF t = two_sum(a.lo, b.lo);
  s.lo += t.hi;
  s = fast_two_sum(s.hi, s.lo);
  s.lo += t.lo;
  return fast_two_sum(s.hi, s.lo);
}

__host__ __device__ __forceinline__ FF ff_neg(FF a) { return FF{-a.hi, -a.lo}; }

// product of two pairs (the lo * lo term is below the precision kept)
__host__ __device__ __forceinline__ FF ff_mul(FF a, FF b) {
  FF p = two_prod(a.hi, b.hi);
  p.lo = fmaf(a.hi, b.lo, p.lo);
  p.lo = fmaf(a.lo, b.hi, p.lo);
  return fast_two_sum(p.hi, p.lo);
}

}  // namespace ffa
}  // namespace hmc
