// trace.h -- tracing and the debug switch of the readout library.
//
// Every public call that enqueues GPU work opens an NVTX range named after
// it (rfr_push_into, rfr_batch_push, ...), so a timeline profiler shows the
// library's calls around their kernels; without an attached tool an NVTX
// range costs a few nanoseconds.  RFR_DEBUG=1 in the environment makes those
// calls synchronise their stream after enqueueing (unless it is being
// captured into a graph) and check for CUDA errors and the plan's device
// status word, so that an error surfaces at the call that caused it.
#pragma once
#include <cuda_runtime.h>
#include <nvtx3/nvToolsExt.h>

#include <cstdlib>
#include <cstring>

namespace rfr {

class TraceRange {
public:
    explicit TraceRange(const char* name) { nvtxRangePushA(name); }
    ~TraceRange() { nvtxRangePop(); }
    TraceRange(const TraceRange&) = delete;
    TraceRange& operator=(const TraceRange&) = delete;
};

inline bool debug_enabled() {
    static const bool on = [] {
        const char* v = std::getenv("RFR_DEBUG");
        return v != nullptr && std::strcmp(v, "0") != 0 && v[0] != '\0';
    }();
    return on;
}

// The stream may be synchronised: debugging is on and it is not capturing.
inline bool debug_sync_allowed(cudaStream_t st) {
    if (!debug_enabled()) return false;
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(st, &cs) != cudaSuccess) return false;
    return cs == cudaStreamCaptureStatusNone;
}

}  // namespace rfr
