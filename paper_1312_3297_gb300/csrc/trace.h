// Named ranges around the library's entry points, visible to NVIDIA's profilers (NVTX v3,
// header-only). When no profiling tool is attached, each range costs one check of a
// function pointer.
#pragma once

#include <nvtx3/nvToolsExt.h>

namespace lbmrv {

struct TraceRange {
    explicit TraceRange(const char* name) { nvtxRangePushA(name); }
    ~TraceRange() { nvtxRangePop(); }
    TraceRange(const TraceRange&) = delete;
    TraceRange& operator=(const TraceRange&) = delete;
};

}  // namespace lbmrv
