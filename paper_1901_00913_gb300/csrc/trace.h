// NVTX ranges around the library's host-side phases (setup, factorisation,
// Lipschitz estimate, graph capture, solves, tuning).  They cost nothing
// unless a profiler is attached.  Library-internal.
#pragma once

#include <nvtx3/nvToolsExt.h>

namespace sfista {

struct TraceRange {
    explicit TraceRange(const char *name) { nvtxRangePushA(name); }
    ~TraceRange() { nvtxRangePop(); }
    TraceRange(const TraceRange &) = delete;
    TraceRange &operator=(const TraceRange &) = delete;
};

}  // namespace sfista
