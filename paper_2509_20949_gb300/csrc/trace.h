// trace.h -- NVTX ranges around the library's calls (sweeps, colour phases,
// pair counts, batch chunks, exchanges), visible in Nsight timelines and
// usable as ncu --nvtx filters; a few nanoseconds when no tool is attached.
#pragma once

#include <nvtx3/nvToolsExt.h>

namespace smcx {

struct TraceRange {
  explicit TraceRange(const char* name) { nvtxRangePushA(name); }
  ~TraceRange() { nvtxRangePop(); }
  TraceRange(const TraceRange&) = delete;
  TraceRange& operator=(const TraceRange&) = delete;
};

}  // namespace smcx
