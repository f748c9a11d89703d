// Launch helpers shared by the kernel translation units: the phase tables of
// the context's current field, and launches with programmatic dependent launch.
#pragma once

#include <type_traits>

#include "kernels.h"
#include "operator.cuh"

namespace hmc {

// Phases of the context's field: the FP64 table e^{i phi}, or phi as float.
template <typename R>
inline Phase<R> phase_of(hmc_ctx* c);
template <>
inline Phase<double> phase_of<double>(hmc_ctx* c) {
  return Phase<double>{(const double2*)c->ws[WS_E]};
}
template <>
inline Phase<float> phase_of<float>(hmc_ctx* c) {
  return Phase<float>{(const float*)c->ws[WS_PHI32]};
}

// Launch with the programmatic-serialization attribute (see pdl_wait).
// Programmatic launches are used only between consecutive kernels of a
// captured iteration chunk: the first kernel of a capture (no kernel before it
// in the graph) and every launch outside a capture are ordinary launches.
template <typename... KA, typename... A>
inline void launch_pdl_smem(hmc_ctx* c, void (*k)(KA...), dim3 grid, int threads, int smem, cudaStream_t s,
                            A... args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = grid;
  cfg.blockDim = dim3(threads);
  cfg.dynamicSmemBytes = (size_t)smem;
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  const bool pdl = c->capturing && c->pdl_armed;
  cfg.attrs = pdl ? attr : nullptr;
  cfg.numAttrs = pdl ? 1 : 0;
  (void)cudaLaunchKernelEx(&cfg, k, ((KA)args)...);  // errors surface through cudaGetLastError
  if (c->capturing) c->pdl_armed = true;
}
template <typename... KA, typename... A>
inline void launch_pdl(hmc_ctx* c, void (*k)(KA...), dim3 grid, int threads, cudaStream_t s, A... args) {
  launch_pdl_smem(c, k, grid, threads, 0, s, args...);
}

template <int J>
using IC = std::integral_constant<int, J>;

}  // namespace hmc
