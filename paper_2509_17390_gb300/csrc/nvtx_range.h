// Named NVTX ranges around the library's public calls and serving ticks, for
// timeline tools.  nvtx3 is header-only: without an attached tool a range
// costs a null-pointer check.
#pragma once

#include <nvtx3/nvToolsExt.h>

namespace fgl {

struct NvtxRange {
  explicit NvtxRange(const char* name) { nvtxRangePushA(name); }
  ~NvtxRange() { nvtxRangePop(); }
  NvtxRange(const NvtxRange&) = delete;
  NvtxRange& operator=(const NvtxRange&) = delete;
};

}  // namespace fgl
