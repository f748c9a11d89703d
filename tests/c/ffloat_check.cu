// Host check of the float-float header (csrc/ffloat.cuh) against double and
// long double arithmetic:
//   1. ff_from_double: |lo| is at most half a unit of hi, hi is within half a
//      unit of x, and hi + lo is within 2^-47 of x for 2^-79 <= |x| up to the
//      largest float; above it the pair is (+-inf, 0); zeros and NaN keep
//      their class.
//   2. ff_to_double: bit-identical to (double)hi + (double)lo (one correct
//      rounding) for pairs from (1), from the arithmetic, and for random pairs
//      with exponent gaps from 20 to 90 bits and both sign combinations.
//   3. two_sum and two_prod are exact; ff_add is within 2^-46 of the exact sum
//      (relative to |a| + |b|, so cancellation is included) and ff_mul within
//      2^-45 of the exact product.
//   4. A row of the fermion operator (Eq. ferm_op) in float-float from random
//      doubles agrees with the same row in long double within 1e-13.
// Prints the number of checks and failures; exits non-zero on any failure.
#include <cmath>
#include <cstdint>
#include <cstdio>
#include <cstring>
#include <random>

#include "ffloat.cuh"

using namespace hmc::ffa;

static long long checks = 0, failures = 0;

static void fail(const char* what, double x, double got, double want) {
  if (failures < 20) std::printf("FAIL %s x=%.17g got=%.17g want=%.17g\n", what, x, got, want);
  ++failures;
}

static uint64_t dbits(double x) {
  uint64_t u;
  std::memcpy(&u, &x, 8);
  return u;
}

static double rand_double(std::mt19937_64& g, int emin, int emax) {
  std::uniform_int_distribution<int> E(emin, emax);
  std::uniform_real_distribution<double> m(1.0, 2.0);
  const double s = (g() & 1) ? -1.0 : 1.0;
  return s * std::ldexp(m(g), E(g));
}

static void check_split(double x) {
  const FF a = ff_from_double(x);
  ++checks;
  const double ax = std::fabs(x);
  if (std::isnan(x)) {
    if (!std::isnan(a.hi) || a.lo != 0.0f) fail("split nan", x, a.hi, x);
    return;
  }
  // largest float plus half a unit: from there on x rounds to infinity
  const double top = std::ldexp(2.0 - std::ldexp(1.0, -24), 127);
  if (ax >= top) {
    if (!std::isinf(a.hi) || std::signbit(a.hi) != std::signbit(x) || a.lo != 0.0f)
      fail("split overflow", x, a.hi, x);
    return;
  }
  if (x == 0.0) {
    if (a.hi != 0.0f || a.lo != 0.0f || std::signbit(a.hi) != std::signbit(x)) fail("split zero", x, a.hi, x);
    return;
  }
  if (ax < std::ldexp(1.0, -126)) {
    if (a.hi != 0.0f || a.lo != 0.0f) fail("split tiny", x, a.hi, 0.0);
    return;
  }
  // a normalised pair: hi within half a unit of x, |lo| at most half a unit;
  // below 2^-79 lo may be dropped and hi is x truncated (within one unit)
  const float ah = std::fabs(a.hi);
  const double unit = (double)(std::nextafter(ah, INFINITY) - ah);
  const double hi_tol = ax >= std::ldexp(1.0, -79) ? 0.5 * unit + std::ldexp(ax, -46) : unit;
  if (std::signbit(a.hi) != std::signbit(x) || std::fabs(ax - (double)ah) > hi_tol) fail("split hi", x, a.hi, x);
  if (std::fabs((double)a.lo) > 0.5 * unit) fail("split lo size", x, a.lo, 0.0);
  if (ax >= std::ldexp(1.0, -79)) {
    const long double s = (long double)a.hi + (long double)a.lo;
    if (std::fabs((double)(s - (long double)x)) > std::ldexp(ax, -47)) fail("split accuracy", x, (double)s, x);
  }
}

static void check_join(FF a) {
  ++checks;
  const double got = ff_to_double(a);
  const double want = (double)a.hi + (double)a.lo;  // one rounding of an exact pair
  if (std::isnan(want)) {
    if (!std::isnan(got)) fail("join nan", a.hi, got, want);
    return;
  }
  if (dbits(got) != dbits(want)) fail("join", a.hi, got, want);
}

int main() {
  std::mt19937_64 g(1804071950ull);
  // 1. splitting
  const double specials[] = {0.0, -0.0, 1.0, -1.0, 3.0, 0.1, -0.1, 1e-30, -1e-30, 1e30, 3.4e38, -3.4e38,
                             std::ldexp(1.0, 127) * 1.999999999, std::ldexp(1.0, 127) * 1.99999988,
                             std::ldexp(2.0 - std::ldexp(1.0, -24), 127), std::ldexp(1.0, 128), std::ldexp(1.0, -79),
                             std::ldexp(1.0, -80) * 1.3, std::ldexp(1.0, -126), std::ldexp(1.0, -127),
                             std::ldexp(1.0, -1074), 1.0 + std::ldexp(1.0, -52), 2.0 - std::ldexp(1.0, -52),
                             INFINITY, -INFINITY, NAN};
  for (double x : specials) {
    check_split(x);
    if (std::isfinite(x) && std::fabs(x) < std::ldexp(1.0, 128)) check_join(ff_from_double(x));
  }
  for (int k = 0; k < 400000; ++k) {
    const double x = rand_double(g, -130, 130);
    check_split(x);
    const FF a = ff_from_double(x);
    if (std::isfinite(a.hi)) check_join(a);
  }
  // 2. joining random pairs with wide exponent gaps, both sign combinations
  for (int k = 0; k < 400000; ++k) {
    const float hi = (float)rand_double(g, -60, 60);
    std::uniform_int_distribution<int> gap(20, 90);
    float lo = (float)std::ldexp(rand_double(g, 0, 0), std::ilogb(hi) - gap(g));
    if (g() & 1) lo = -lo;
    check_join(FF{hi, lo});
  }
  // 3. error-free transforms and pair arithmetic
  for (int k = 0; k < 400000; ++k) {
    const float a = (float)rand_double(g, -20, 20), b = (float)rand_double(g, -20, 20);
    const FF s = two_sum(a, b), p = two_prod(a, b);
    ++checks;
    if ((long double)s.hi + s.lo != (long double)a + b) fail("two_sum", a, s.hi, b);
    if ((long double)p.hi + p.lo != (long double)a * b) fail("two_prod", a, p.hi, b);
    const double x = rand_double(g, -10, 10);
    const double y = (k % 4 == 0) ? -x * (1.0 + std::ldexp(rand_double(g, 0, 0), -30)) : rand_double(g, -10, 10);
    const FF fx = ff_from_double(x), fy = ff_from_double(y);
    const long double X = (long double)fx.hi + fx.lo, Y = (long double)fy.hi + fy.lo;
    const FF sum = ff_add(fx, fy), prod = ff_mul(fx, fy);
    check_join(sum);
    check_join(prod);
    const long double ssum = (long double)sum.hi + sum.lo, sprod = (long double)prod.hi + prod.lo;
    if (std::fabs((double)(ssum - (X + Y))) > std::ldexp((double)(fabsl(X) + fabsl(Y)), -46))
      fail("ff_add", x, (double)ssum, (double)(X + Y));
    if (std::fabs((double)(sprod - X * Y)) > std::ldexp(std::fabs((double)(X * Y)), -45))
      fail("ff_mul", x, (double)sprod, (double)(X * Y));
  }
  // 4. one row of M: -u + z u_t - dk (u1 + u2 + u3), z = e^{i phi} - dm, in float-float
  std::uniform_real_distribution<double> U(-1.0, 1.0);
  for (int k = 0; k < 100000; ++k) {
    const double phi = 3.0 * U(g), dm = 0.1 * (U(g) + 1.0), dk = 0.25;
    double u[5][2];
    for (auto& c : u) {
      c[0] = U(g);
      c[1] = U(g);
    }
    const double zr = std::cos(phi) - dm, zi = std::sin(phi);
    // long double reference from the same double inputs
    const long double rr = -(long double)u[0][0] + ((long double)zr * u[1][0] - (long double)zi * u[1][1]) -
                           (long double)dk * ((long double)u[2][0] + u[3][0] + u[4][0]);
    const long double ri = -(long double)u[0][1] + ((long double)zr * u[1][1] + (long double)zi * u[1][0]) -
                           (long double)dk * ((long double)u[2][1] + u[3][1] + u[4][1]);
    FF f[5][2];
    for (int j = 0; j < 5; ++j)
      for (int c = 0; c < 2; ++c) f[j][c] = ff_from_double(u[j][c]);
    const FF Zr = ff_from_double(zr), Zi = ff_from_double(zi), DK = ff_from_double(dk);
    FF tr = ff_add(ff_neg(f[0][0]), ff_add(ff_mul(Zr, f[1][0]), ff_neg(ff_mul(Zi, f[1][1]))));
    FF ti = ff_add(ff_neg(f[0][1]), ff_add(ff_mul(Zr, f[1][1]), ff_mul(Zi, f[1][0])));
    const FF hr = ff_add(ff_add(f[2][0], f[3][0]), f[4][0]);
    const FF hi = ff_add(ff_add(f[2][1], f[3][1]), f[4][1]);
    tr = ff_add(tr, ff_neg(ff_mul(DK, hr)));
    ti = ff_add(ti, ff_neg(ff_mul(DK, hi)));
    const double gr = ff_to_double(tr), gi = ff_to_double(ti);
    const double scale = std::fmax(1.0, std::fmax(std::fabs((double)rr), std::fabs((double)ri)));
    ++checks;
    if (std::fabs(gr - (double)rr) > 1e-13 * scale || std::fabs(gi - (double)ri) > 1e-13 * scale)
      fail("stencil row", phi, gr, (double)rr);
  }
  std::printf("%lld checks, %lld failures\n", checks, failures);
  return failures == 0 ? 0 : 1;
}
