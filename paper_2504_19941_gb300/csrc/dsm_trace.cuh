// dsm_trace.cuh -- NVTX ranges around the library's entry points, so that a
// profiler's timeline shows the moments pass, the fused pass, the energy
// evaluations and the L-BFGS loop by name.  Header-only NVTX v3: without a
// profiler attached each range costs one call through a stub.
#pragma once

#include <nvtx3/nvToolsExt.h>

namespace dsm {

struct TraceRange {
  explicit TraceRange(const char *name) { nvtxRangePushA(name); }
  ~TraceRange() { nvtxRangePop(); }
  TraceRange(const TraceRange &) = delete;
  TraceRange &operator=(const TraceRange &) = delete;
};

}  // namespace dsm
