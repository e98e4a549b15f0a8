// Tracing: an NVTX range around each C-ABI call, in the domain "semiring", and one
// around each pivot block of the closure schedules (payload: the block index).
//
// NVTX 3 is header-only.  With no tool attached (Nsight Systems, ncu --nvtx, or any
// library named by NVTX_INJECTION64_PATH) a push or pop is one call through an empty
// function slot, so the ranges stay on in every build.  Ranges are host-side: they
// bracket the call's enqueue work on the calling thread, not the kernels' device time.
#pragma once

#include <nvtx3/nvToolsExt.h>

namespace sr {

inline nvtxDomainHandle_t trace_domain()
{
    static nvtxDomainHandle_t d = nvtxDomainCreateA("semiring");
    return d;
}

class TraceRange {
public:
    explicit TraceRange(const char *name)
    {
        nvtxEventAttributes_t a = {};
        a.version = NVTX_VERSION;
        a.size = NVTX_EVENT_ATTRIB_STRUCT_SIZE;
        a.messageType = NVTX_MESSAGE_TYPE_ASCII;
        a.message.ascii = name;
        nvtxDomainRangePushEx(trace_domain(), &a);
    }
    // with an integer payload (a closure's pivot block index)
    TraceRange(const char *name, long long payload)
    {
        nvtxEventAttributes_t a = {};
        a.version = NVTX_VERSION;
        a.size = NVTX_EVENT_ATTRIB_STRUCT_SIZE;
        a.messageType = NVTX_MESSAGE_TYPE_ASCII;
        a.message.ascii = name;
        a.payloadType = NVTX_PAYLOAD_TYPE_INT64;
        a.payload.llValue = payload;
        nvtxDomainRangePushEx(trace_domain(), &a);
    }
    ~TraceRange() { nvtxDomainRangePop(trace_domain()); }
    TraceRange(const TraceRange &) = delete;
    TraceRange &operator=(const TraceRange &) = delete;
};

}  // namespace sr

#define SR_TRACE(name) ::sr::TraceRange sr_trace_range_(name)
// one pivot block of a closure schedule: the enqueue of its launches on every stream
#define SR_TRACE_BLOCK(name, kb) ::sr::TraceRange sr_trace_block_(name, (long long)(kb))
