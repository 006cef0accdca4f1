// Host-side trace ranges around the library's entry points (NVTX v3, header
// only).  With no profiler attached the calls do nothing; under ncu or a
// timeline tool every ms_step / ms_grad / ms_diag / batched or sparse step
// shows as a named range, so its kernels can be selected by range
// (`ncu --nvtx --nvtx-include "ms_step/"`).  Without the NVTX headers the
// ranges compile away.
#pragma once

#if defined(__has_include)
#if __has_include(<nvtx3/nvToolsExt.h>)
#include <nvtx3/nvToolsExt.h>
#define MS_HAVE_NVTX 1
#endif
#endif

namespace msgb {

struct TraceRange {
  explicit TraceRange(const char* name) {
#ifdef MS_HAVE_NVTX
    nvtxRangePushA(name);
#else
    (void)name;
#endif
  }
  ~TraceRange() {
#ifdef MS_HAVE_NVTX
    nvtxRangePop();
#endif
  }
  TraceRange(const TraceRange&) = delete;
  TraceRange& operator=(const TraceRange&) = delete;
};

}  // namespace msgb
