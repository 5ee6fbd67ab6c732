// trace.h -- NVTX ranges around the C-ABI calls, compiled in with -DPTG_NVTX (the "nvtx" variant
// of the build, libptg_nvtx.so).  Every range lives in the NVTX domain "ptg" and carries the
// entry point's name (the batch phases add a nested range per phase).  A range opens when the
// call starts and closes when it returns, so on a profiler's timeline it spans the host time
// that enqueues the call's launches; the launches themselves show up under it through NVTX's
// CUDA correlation.  During stream capture a range marks the capture, not the graph's replays.
// With no tool attached the NVTX calls return at once.  Without PTG_NVTX, PTG_TRACE expands to
// nothing and the library holds no NVTX code.
#pragma once

#ifdef PTG_NVTX
#include <nvtx3/nvToolsExt.h>

namespace ptg {

inline nvtxDomainHandle_t trace_domain() {
  static const nvtxDomainHandle_t domain = nvtxDomainCreateA("ptg");
  return domain;
}

class TraceRange {
 public:
  explicit TraceRange(const char* name) {
    nvtxEventAttributes_t a = {};
    a.version = NVTX_VERSION;
    a.size = NVTX_EVENT_ATTRIB_STRUCT_SIZE;
    a.messageType = NVTX_MESSAGE_TYPE_ASCII;
    a.message.ascii = name;
    nvtxDomainRangePushEx(trace_domain(), &a);
  }
  ~TraceRange() { nvtxDomainRangePop(trace_domain()); }
  TraceRange(const TraceRange&) = delete;
  TraceRange& operator=(const TraceRange&) = delete;
};

}  // namespace ptg

#define PTG_TRACE_CAT2(a, b) a##b
#define PTG_TRACE_CAT(a, b) PTG_TRACE_CAT2(a, b)
#define PTG_TRACE(name) ::ptg::TraceRange PTG_TRACE_CAT(ptg_trace_range_, __LINE__)(name)
#define PTG_TRACE_ENABLED 1
#else
#define PTG_TRACE(name) ((void)0)
#define PTG_TRACE_ENABLED 0
#endif
