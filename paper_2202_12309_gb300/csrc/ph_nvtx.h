// ph_nvtx.h -- NVTX ranges around the library's kernel launches and entry
// points, so that a profiler's timeline names each step of a cycle (stage,
// ghost exchange, flux correction, dt, remesh, copies).  NVTX v3 is
// header-only: without an attached tool a range costs a few nanoseconds.
// Launches recorded into a CUDA graph get their range at capture time.
#pragma once
#include <nvtx3/nvToolsExt.h>

namespace ph {

struct NvtxRange {
  explicit NvtxRange(const char* name) { nvtxRangePushA(name); }
  ~NvtxRange() { nvtxRangePop(); }
  NvtxRange(const NvtxRange&) = delete;
  NvtxRange& operator=(const NvtxRange&) = delete;
};

}  // namespace ph

#define PH_NVTX_CAT2(a, b) a##b
#define PH_NVTX_CAT(a, b) PH_NVTX_CAT2(a, b)
// A range named `name` from here to the end of the enclosing scope.
#define PH_RANGE(name) ::ph::NvtxRange PH_NVTX_CAT(ph_nvtx_range_, __LINE__)(name)
