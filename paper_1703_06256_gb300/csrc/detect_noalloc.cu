// detect_noalloc.cu -- hog_detect for callers that cannot hand the library
// any scratch memory.
//
// hog_detect needs a small workspace (a tag word and one status word per
// tile of 2048 scores) that the caller allocates.  Some callers cannot do
// that: a plugin that only receives its input and output buffers from a
// host application that owns all device memory, or a latency-critical loop
// that must never call cudaMalloc (which may synchronise the device and has
// unbounded latency).  hog_detect_noalloc runs the same kernel with the
// workspace taken from a fixed array in the library's own device memory.
//
// The array below is a file-scope __device__ variable, so every GPU that
// loads the library holds it (128 KiB + 64 bytes) until the process exits.
// Host code cannot pass the variable's name to a kernel (on the host the
// name is a stand-in, not a device address), so its device address is
// looked up with cudaGetSymbolAddress once per device, with that device
// current, the first time the entry point is called on it.  That first
// call therefore belongs before any stream capture.  Every call shares the
// array: calls whose work overlaps on the GPU (different streams, or
// different host threads without ordering) race on it and give wrong
// lists.  The array starts zero-filled (static device memory is zeroed when
// the library is loaded), which is the state the kernel needs before its
// first launch, and every call leaves it ready for the next one: nothing
// has to be cleared between calls.
#include <mutex>

#include "internal.cuh"

namespace fasthog {

namespace {

constexpr int kNoAllocTiles = 16384;  // tiles of 2048 scores: 33,554,432 scores per call at most
constexpr int kMaxDevices = 64;

// 64-byte header (the launch tag) + one 8-byte status word per tile
static __device__ __align__(256) unsigned long long g_detect_scratch[8 + kNoAllocTiles];

std::mutex g_setup_mutex;
void* g_scratch_addr[kMaxDevices] = {nullptr};

// Device address of g_detect_scratch on the current device.
hog_status scratch_address(void** out) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return cuda_fail(e);
    if (dev < 0 || dev >= kMaxDevices) return HOG_ERR_UNSUPPORTED;
    std::lock_guard<std::mutex> lock(g_setup_mutex);
    if (g_scratch_addr[dev] == nullptr) {
        void* p = nullptr;
        e = cudaGetSymbolAddress(&p, g_detect_scratch);
        if (e != cudaSuccess) return cuda_fail(e);
        g_scratch_addr[dev] = p;
    }
    *out = g_scratch_addr[dev];
    return HOG_OK;
}

}  // namespace

}  // namespace fasthog

using namespace fasthog;

extern "C" hog_status hog_detect_noalloc(const void* scores, int score_dtype, int nx, int ny, int stride, float thr,
                                         int image, int level, hog_det* out, int max_out, int32_t* d_count,
                                         hog_stream_t stream) {
    if (scores == nullptr || d_count == nullptr) return HOG_ERR_ARG;
    if (out == nullptr && max_out > 0) return HOG_ERR_ARG;
    if (reinterpret_cast<uintptr_t>(out) % alignof(hog_det) != 0) return HOG_ERR_ARG;
    if (nx < 0 || ny < 0 || stride < 1 || max_out < 0) return HOG_ERR_ARG;
    if ((long)nx * ny > (long)HOG_DETECT_NOALLOC_MAX_SCORES) return HOG_ERR_ARG;  // beyond the fixed scratch
    if (score_dtype != HOG_F32 && score_dtype != HOG_I32) return HOG_ERR_ARG;
    if (thr != thr) return HOG_ERR_ARG;  // NaN
    if (detect_tiles((long)nx * ny) > kNoAllocTiles) return HOG_ERR_ARG;  // one status word per tile
    static_assert(sizeof(g_detect_scratch) >= 64 + 8 * (size_t)kNoAllocTiles, "scratch holds every tile");
    void* scratch = nullptr;
    const hog_status s = scratch_address(&scratch);
    if (s != HOG_OK) return s;
    return launch_detect(scores, score_dtype, nx, ny, stride, thr, image, level, out, max_out, d_count, scratch,
                         reinterpret_cast<cudaStream_t>(stream));
}
