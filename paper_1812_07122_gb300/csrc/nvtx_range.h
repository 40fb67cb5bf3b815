// NVTX ranges around the library's host-side phases (measurement support; no counterpart in the
// paper).  The header-only NVTX v3 API costs a few nanoseconds per range when no tool is
// attached; under a profiler the ranges name the work each launch belongs to (e.g. ncu --nvtx
// --nvtx-include "blfls_smooth/").
#pragma once

#include <nvtx3/nvToolsExt.h>

namespace blfls {

class NvtxRange {
public:
    explicit NvtxRange(const char* name) { nvtxRangePushA(name); }
    ~NvtxRange() { nvtxRangePop(); }
    NvtxRange(const NvtxRange&) = delete;
    NvtxRange& operator=(const NvtxRange&) = delete;
};

}  // namespace blfls
