// score_tc.cu -- window score on the tensor cores (tcgen05 implicit GEMM).
// Placeholder until the tensor-core kernel lands: reports no support, so
// hog_window_score uses the CUDA-core kernel for every weight type.
#include "internal.cuh"

namespace fasthog {

bool score_tc_supported(int, int, int, int, int, int) { return false; }

hog_status launch_score_tc(const uint16_t*, int, int, int, int, int, int, const void*, int, float, void*,
                           cudaStream_t) {
    return HOG_ERR_UNSUPPORTED;
}

}  // namespace fasthog
