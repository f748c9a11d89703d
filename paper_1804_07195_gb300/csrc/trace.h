// NVTX ranges around the library's entry points and the steps of a trajectory,
// so that a timeline profiler shows operator applications, solves, forces and
// MD steps by name. NVTX v3 is header-only: without a profiler attached a range
// costs a few nanoseconds.
#pragma once

#include <nvtx3/nvToolsExt.h>

namespace hmc {

struct TraceRange {
  explicit TraceRange(const char* name) { nvtxRangePushA(name); }
  ~TraceRange() { nvtxRangePop(); }
  TraceRange(const TraceRange&) = delete;
  TraceRange& operator=(const TraceRange&) = delete;
};

}  // namespace hmc

#define HMC_TRACE(name) ::hmc::TraceRange hmc_trace_range_(name)
