// nvtx_range.h -- NVTX ranges around the library's entry points, for a
// profiler's timeline (nsys, ncu's range filters).  Header-only NVTX v3: with
// no tool attached a range costs one branch.
#pragma once
#include <nvtx3/nvToolsExt.h>

namespace lbm {

struct NvtxRange {
    explicit NvtxRange(const char* name) { nvtxRangePushA(name); }
    ~NvtxRange() { nvtxRangePop(); }
    NvtxRange(const NvtxRange&) = delete;
    NvtxRange& operator=(const NvtxRange&) = delete;
};

}  // namespace lbm

#define LBM_RANGE(name) ::lbm::NvtxRange lbm_nvtx_range_(name)
