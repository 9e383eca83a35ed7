// NVTX ranges around the C-ABI compute calls, so that a profiler with an NVTX
// tool attached (ncu --nvtx, for example) can group the kernels a call
// launched.  Without a tool attached each push and pop is a no-op.
#pragma once
#include <nvtx3/nvToolsExt.h>

namespace swept_trace {
struct Range {
  explicit Range(const char* name) { nvtxRangePushA(name); }
  ~Range() { nvtxRangePop(); }
  Range(const Range&) = delete;
  Range& operator=(const Range&) = delete;
};
}  // namespace swept_trace
