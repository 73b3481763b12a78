// NVTX ranges around the host-side phases of the engine (load, layout build,
// superstep, exchange, cache update, pipeline copies, serving loop), so that
// a profiler's timeline shows where the time goes. NVTX is header-only: with
// no tool attached a range costs a couple of function calls.
#pragma once

#include <nvtx3/nvToolsExt.h>

namespace gxp {

class TraceRange {
public:
    explicit TraceRange(const char* name) { nvtxRangePushA(name); }
    ~TraceRange() { nvtxRangePop(); }
    TraceRange(const TraceRange&) = delete;
    TraceRange& operator=(const TraceRange&) = delete;
};

}  // namespace gxp
