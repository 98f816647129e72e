// selftest.cu -- hog_selftest_wait_timeout: one bounded device-side wait
// that is made to run out, so the timeout path (status bit, early return)
// can be tested on a GPU without a fault or a hang.
#include "internal.cuh"
#include "onepass.cuh"
#include "ptx.cuh"

namespace fasthog {

namespace {

// A flag no kernel ever raises (static device memory starts zero-filled).
__device__ uint32_t g_never_raised;

__global__ void __launch_bounds__(32) wait_timeout_kernel(int mode, uint64_t limit_ns, unsigned int* status) {
    __shared__ __align__(8) uint64_t bar;
    if (threadIdx.x == 0) {
        ptx::mbar_init(&bar, 1);  // one arrival expected; none ever comes
        ptx::fence_mbar_init();
    }
    __syncwarp();
    if (threadIdx.x != 0) return;
    const bool ok = mode == 0 ? ptx::mbar_wait_bounded(&bar, 0, limit_ns)
                              : onepass::wait_flag(&g_never_raised, 1u, limit_ns);
    if (!ok) atomicOr(status, kStatusTimeout);
}

}  // namespace

}  // namespace fasthog

using namespace fasthog;

extern "C" hog_status hog_selftest_wait_timeout(int mode, int limit_us, hog_stream_t stream) {
    if ((mode != 0 && mode != 1) || limit_us < 1 || limit_us > 1000000) return HOG_ERR_ARG;
    unsigned int* status = nullptr;
    const hog_status s = device_status_word(&status);
    if (s != HOG_OK) return s;
    wait_timeout_kernel<<<1, 32, 0, reinterpret_cast<cudaStream_t>(stream)>>>(mode, (uint64_t)limit_us * 1000ull,
                                                                            status);
    return check_launch();
}
