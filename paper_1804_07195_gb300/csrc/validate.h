// Host-side argument checks shared by every C entry point. They run before any
// CUDA call, so a rejected argument never reaches a kernel.
#pragma once

#include <cmath>
#include <cstddef>
#include <cstdint>

#include "hmc.h"

namespace hmc {

// Kernels index sites with 32-bit signed integers: N = 2 n m nt stays below 2^30.
constexpr long long kMaxSites = 1LL << 30;

// N = 2 n m nt of the lattice, or -1 when a dimension is out of range or the
// site count reaches kMaxSites. Every factor is below 2^31, and each partial
// product is bounded before the next multiplication, so nothing overflows
// 64 bits whatever the inputs.
inline long long lattice_sites(const hmc_lattice* L) {
  if (!L || L->n < 1 || L->m < 1 || L->nt < 2) return -1;
  const long long V = (long long)L->n * (long long)L->m;  // < 2^62
  if (V >= kMaxSites) return -1;
  const long long H = V * (long long)L->nt;  // < 2^30 * 2^31
  if (H >= kMaxSites / 2) return -1;
  return 2 * H;
}

// The lattice of Section 2 is usable: dimensions in range (see lattice_sites),
// couplings finite, beta > 0 and U > 0 (the Gaussian weight 1/(delta U) of
// Eq. hamiltonian needs both).
inline bool bad_lattice(const hmc_lattice* L) {
  if (lattice_sites(L) < 0) return true;
  if (!std::isfinite(L->kappa) || !std::isfinite(L->U) || !std::isfinite(L->beta)) return true;
  if (!(L->beta > 0.0) || !(L->U > 0.0)) return true;
  return false;
}

// True when the byte ranges [a, a + bytes) and [b, b + bytes) share a byte.
inline bool ranges_overlap(const void* a, const void* b, size_t bytes) {
  const uintptr_t x = (uintptr_t)a, y = (uintptr_t)b;
  return x < y + bytes && y < x + bytes;
}

}  // namespace hmc
