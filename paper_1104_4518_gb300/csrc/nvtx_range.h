// NVTX range around a public call of the library: the call shows as a named
// range on Nsight timelines, and `ncu --nvtx --nvtx-include <name>/` captures
// only the kernels it launches.  Header-only NVTX 3: without a tool attached a
// push or pop is one check of a function pointer.
#pragma once

#include <nvtx3/nvToolsExt.h>

namespace bfsint {

class NvtxRange {
 public:
  explicit NvtxRange(const char* name) { nvtxRangePushA(name); }
  ~NvtxRange() { nvtxRangePop(); }
  NvtxRange(const NvtxRange&) = delete;
  NvtxRange& operator=(const NvtxRange&) = delete;
};

}  // namespace bfsint
