// NVTX range for tracing: one named range per library call (load, iterate,
// batch round, serving round) in profiler timelines; costs nothing when no
// tool is attached.
#pragma once

#include <nvtx3/nvToolsExt.h>

struct NvtxRange {
    explicit NvtxRange(const char* name) { nvtxRangePushA(name); }
    ~NvtxRange() { nvtxRangePop(); }
    NvtxRange(const NvtxRange&) = delete;
    NvtxRange& operator=(const NvtxRange&) = delete;
};
