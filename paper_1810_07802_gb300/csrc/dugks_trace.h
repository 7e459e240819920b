// dugks_trace.h -- NVTX ranges around the C-ABI calls, so that a profiler
// timeline (nsys, ncu's range filters) shows create / step / macros / reduce
// and the batch calls by name.  NVTX v3 is header-only: without a tool
// attached, a range costs a few nanoseconds.
#pragma once

#include <nvtx3/nvToolsExt.h>

namespace dugks {
struct TraceRange {
    explicit TraceRange(const char *name) { nvtxRangePushA(name); }
    ~TraceRange() { nvtxRangePop(); }
    TraceRange(const TraceRange &) = delete;
    TraceRange &operator=(const TraceRange &) = delete;
};
}  // namespace dugks
