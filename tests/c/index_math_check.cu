// Host-side check of the library's stencil index arithmetic: the multiply-high
// division by a runtime constant (make_fastdiv and its host twin fastdiv_host,
// the formula the kernels evaluate with __umulhi) against plain integer
// division, for every divisor up to 5000 and 200,000 random divisors up to
// 2^29 (cell counts n and n*m of any lattice the library accepts, which has
// fewer than 2^30 sites), at numerators around every multiple boundary that
// matters and at random numerators below 2^30. Prints the number of checks and
// failures; exits non-zero on any failure.
#include <cstdint>
#include <cstdio>
#include <random>

#include "common.cuh"

using namespace hmc;

static long long checks = 0, failures = 0;

static void check(uint32_t d, uint32_t x) {
  const FastDiv f = make_fastdiv(d);
  const uint32_t q = fastdiv_host(x, f);
  ++checks;
  if (q != x / d) {
    if (failures < 10) std::printf("FAIL d=%u x=%u got %u want %u\n", d, x, q, x / d);
    ++failures;
  }
}

static void around_multiples(uint32_t d, std::mt19937_64& rng) {
  const uint32_t top = (1u << 30) - 1;
  for (uint32_t k = 0; k <= 3; ++k) {
    const uint64_t b = (uint64_t)k * d;
    for (int o = -1; o <= 1; ++o)
      if ((int64_t)b + o >= 0 && b + o <= top) check(d, (uint32_t)(b + o));
  }
  const uint64_t kmax = top / d;
  for (uint64_t k = kmax > 2 ? kmax - 2 : 0; k <= kmax; ++k) {
    const uint64_t b = k * d;
    for (int o = -1; o <= 1; ++o)
      if ((int64_t)b + o >= 0 && b + o <= top) check(d, (uint32_t)(b + o));
  }
  check(d, top);
  std::uniform_int_distribution<uint32_t> X(0, top);
  for (int r = 0; r < 8; ++r) check(d, X(rng));
}

int main() {
  std::mt19937_64 rng(20180419);
  for (uint32_t d = 1; d <= 5000; ++d) {
    for (uint32_t x = 0; x < 3 * d + 3; ++x) check(d, x);
    around_multiples(d, rng);
  }
  std::uniform_int_distribution<uint32_t> D(1, 1u << 29);
  for (int r = 0; r < 200000; ++r) around_multiples(D(rng), rng);
  for (int s = 0; s <= 29; ++s) around_multiples(1u << s, rng);
  std::printf("%lld checks, %lld failures\n", checks, failures);
  return failures == 0 ? 0 : 1;
}
