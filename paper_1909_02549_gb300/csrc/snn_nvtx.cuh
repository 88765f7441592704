// NVTX ranges around the library's host entry points, so that Nsight timelines
// show which call launched which kernels.  NVTX v3 is header-only: without a
// profiler attached each push and pop is a cheap no-op.
#pragma once
#include <nvtx3/nvToolsExt.h>

namespace snn {

// One range for the lifetime of the object (every return path pops it).
struct NvtxRange {
    explicit NvtxRange(const char* name) { nvtxRangePushA(name); }
    ~NvtxRange() { nvtxRangePop(); }
    NvtxRange(const NvtxRange&) = delete;
    NvtxRange& operator=(const NvtxRange&) = delete;
};

}  // namespace snn
