// cf_nvtx.h -- NVTX range over one call of the C ABI, named after the entry
// point: seen by profilers that read NVTX; without one attached a push and a
// pop cost next to nothing (NVTX 3 is header-only, nothing is linked).
#pragma once
#include <nvtx3/nvToolsExt.h>

namespace cf {

struct CfRange {
  explicit CfRange(const char *name) { nvtxRangePushA(name); }
  ~CfRange() { nvtxRangePop(); }
  CfRange(const CfRange &) = delete;
  CfRange &operator=(const CfRange &) = delete;
};

}  // namespace cf
