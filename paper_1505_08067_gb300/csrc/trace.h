// NVTX ranges around the library's host entry points (plan creation,
// execution, serving, the work queue), in a domain of their own ("gbfft") so
// that they do not change the push/pop range stack of the caller's default
// domain.  NVTX is header-only: without a profiler attached a range costs a
// few nanoseconds.
#pragma once
#include <nvtx3/nvToolsExt.h>

namespace gbfft {

inline nvtxDomainHandle_t trace_domain() {
  static nvtxDomainHandle_t d = nvtxDomainCreateA("gbfft");
  return d;
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

}  // namespace gbfft
