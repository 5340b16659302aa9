// mfs_trace.h -- NVTX ranges around the library's entry points, so that a timeline tool shows each
// call (create, iterate, solve, residuals, ...) over the kernels it launched. NVTX 3 is header-only:
// without an attached tool a range costs a null check.
#pragma once

#include <nvtx3/nvToolsExt.h>

namespace mfs {

struct TraceRange {
    explicit TraceRange(const char* name) { nvtxRangePushA(name); }
    ~TraceRange() { nvtxRangePop(); }
    TraceRange(const TraceRange&) = delete;
    TraceRange& operator=(const TraceRange&) = delete;
};

}  // namespace mfs

#define MFS_TRACE(name) ::mfs::TraceRange mfs_trace_range_(name)
