// ci_trace.h -- host-side trace ranges of the library, in the NVTX domain
// "ci_prng" (header-only NVTX 3; no-ops unless a profiling tool is attached).
// A separate domain keeps them out of range filters on the default domain.
#pragma once

#include <nvtx3/nvToolsExt.h>

namespace ci {

inline nvtxDomainHandle_t trace_domain() {
    static nvtxDomainHandle_t d = nvtxDomainCreateA("ci_prng");
    return d;
}

struct TraceRange {
    explicit TraceRange(const char *name) {
        nvtxEventAttributes_t a = {};
        a.version = NVTX_VERSION;
        a.size = NVTX_EVENT_ATTRIB_STRUCT_SIZE;
        a.messageType = NVTX_MESSAGE_TYPE_ASCII;
        a.message.ascii = name;
        nvtxDomainRangePushEx(trace_domain(), &a);
    }
    ~TraceRange() { nvtxDomainRangePop(trace_domain()); }
    TraceRange(const TraceRange &) = delete;
    TraceRange &operator=(const TraceRange &) = delete;
};

}  // namespace ci
