// demod_stub.cu -- placeholder entry points of the demodulation path.
#include "rfr_internal.h"

namespace rfr {
cudaError_t demod_build_taps(const double*, const uint64_t*, int, int, int, int, int, void*, void*,
                             cudaStream_t) {
    return cudaErrorNotSupported;
}
cudaError_t demod_launch(const DemodLaunch&, cudaStream_t) { return cudaErrorNotSupported; }
size_t demod_xs_rows(int64_t F, int L, int D) { return static_cast<size_t>(F + (L + D - 1) / D); }
cudaError_t plain_demod(const int16_t*, int64_t, int, int, const float*, const uint64_t*, int, void*,
                        int64_t, cudaStream_t) {
    return cudaErrorNotSupported;
}
}  // namespace rfr
