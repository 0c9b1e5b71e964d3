// xcorr_nvtx.h -- NVTX ranges around the library's public calls, so that a
// timeline profiler (Nsight Systems) shows each call and the kernels it
// launched under its name.  NVTX is header-only: with no tool attached a range
// costs one check of a function pointer.
#pragma once

#include <nvtx3/nvToolsExt.h>

namespace xc {

class NvtxRange {
 public:
  explicit NvtxRange(const char* name) { nvtxRangePushA(name); }
  ~NvtxRange() { nvtxRangePop(); }
  NvtxRange(const NvtxRange&) = delete;
  NvtxRange& operator=(const NvtxRange&) = delete;
};

}  // namespace xc
