// nvtx_range.h -- a named NVTX range around a host entry point of the library, so
// that a profiler's timeline shows its calls (set-up, solve, sampler, warm-start
// steps) by name. NVTX3 is header-only: without an attached tool the push and pop
// return at once. Host code only.
#pragma once
#include <nvtx3/nvToolsExt.h>

namespace tb {

struct NvtxRange {
  explicit NvtxRange(const char *name) { nvtxRangePushA(name); }
  ~NvtxRange() { nvtxRangePop(); }
  NvtxRange(const NvtxRange &) = delete;
  NvtxRange &operator=(const NvtxRange &) = delete;
};

} // namespace tb
