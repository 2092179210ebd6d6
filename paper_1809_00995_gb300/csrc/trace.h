// trace.h -- NVTX ranges around the library's host entry points (a step
// sequence, a diagnostics pass, autotuning, batch and server rounds), so that
// a timeline profiler shows the phases of a run.  With no profiler attached
// the NVTX calls return at once.
#pragma once

#include <nvtx3/nvToolsExt.h>

namespace ah {

struct TraceRange {
    explicit TraceRange(const char *name) { nvtxRangePushA(name); }
    ~TraceRange() { nvtxRangePop(); }
    TraceRange(const TraceRange &) = delete;
    TraceRange &operator=(const TraceRange &) = delete;
};

}  // namespace ah
