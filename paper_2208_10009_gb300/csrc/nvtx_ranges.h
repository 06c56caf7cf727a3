// nvtx_ranges.h -- named host-side ranges around the library's kernel enqueues (NVTX v3,
// header only: a push/pop costs nothing measurable when no profiler is attached), so that
// a timeline shows launch / raygen / trace / dedup / refine / validity by name.
#pragma once

#include <nvtx3/nvToolsExt.h>

namespace sbr {

struct Range {
    explicit Range(const char *name) { nvtxRangePushA(name); }
    ~Range() { nvtxRangePop(); }
    Range(const Range &) = delete;
    Range &operator=(const Range &) = delete;
};

}  // namespace sbr
