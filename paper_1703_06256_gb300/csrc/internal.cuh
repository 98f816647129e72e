// internal.cuh -- declarations shared by the translation units of libfasthog.
// Not installed; the public interface is include/fasthog.h.
#pragma once

#include <atomic>
#include <mutex>

#include <cuda_runtime.h>
#include <cstddef>
#include <cstdint>

#include "../../include/fasthog.h"

namespace fasthog {

constexpr int kLutSide = HOG_LUT_SIDE;   // 511
constexpr int kLutPitch = HOG_LUT_PITCH; // 512
constexpr int kLutQuadOffset = HOG_LUT_QUAD_OFFSET;
constexpr int kLutTotal = HOG_LUT_BYTES;
constexpr int kDMax = 255;
constexpr int kMaxBins = 64;
constexpr uint8_t kNoBin = HOG_NO_BIN;
constexpr int kNumSMs = 152;             // GB300: 2 dies x 76 SMs (queried at run time too)

// Record a CUDA failure for hog_last_cuda_error() and map it to a status.
hog_status cuda_fail(cudaError_t e);
// Check the launch that was just enqueued.
hog_status check_launch();
// Number of SMs of the current device (cached per device).
int sm_count();
// Current value of a launch-shape knob (hog_tune_knob); 0 = the library's choice.
int tune_get(int knob);
// Device address of the library's status word on the current device.
hog_status device_status_word(unsigned int** out);

// ---- launchers (one per kernel family), called by api.cu after argument checks
struct LutParams {
    int n_bins;
    // Boundary directions theta_k = 2*pi*k/N_b, k = 1..N_b-1, as fixed-point
    // cos/sin scaled by 2^40 (see lut.cu).
    long long c[kMaxBins];
    long long s[kMaxBins];
};
hog_status launch_build_lut(const LutParams& p, uint8_t* lut, cudaStream_t st);

hog_status launch_bin_map(const uint8_t* img, int W, int H, int channels, size_t pitch,
                          const uint8_t* lut, int n_bins, uint8_t* bins, unsigned int* status,
                          cudaStream_t st);

size_t integral_workspace_bytes(int W, int H, int n_bins);
// Leading bytes of an integral workspace that must be zero-filled before its first use.
size_t integral_sync_bytes(int W, int H);
// Whether hog_integral of this size, under the current knobs, takes the single
// pass, the one schedule that reads the workspace's tag and flags (the others
// never touch that region).
bool integral_uses_sync(int W, int H, int n_bins, int ii_dtype);
// Kernel launches hog_integral makes for this size under the current knobs.
int integral_launches(int W, int H, int n_bins);
hog_status launch_integral(const uint8_t* bins, int W, int H, int n_bins, int ii_dtype, void* ii,
                           void* ws, cudaStream_t st);

hog_status launch_cell_hist(const void* ii, int W, int H, int n_bins, int ii_dtype, int cell,
                            int stride, int cell_dtype, void* cells, cudaStream_t st);

hog_status launch_score_cuda_cores(const void* cells, int cell_dtype, int ncx, int ncy, int n_bins,
                                   int cells_x, int cells_y, int r, const void* w, int w_dtype,
                                   float bias, void* scores, cudaStream_t st);
bool score_slide_supported(const void* cells, int n_bins, int cells_x, int cells_y, int r);
hog_status launch_score_slide(const void* cells, int cell_dtype, int ncx, int ncy, int r, const void* w,
                              int w_dtype, float bias, void* scores, cudaStream_t st);
bool score_tc_supported(int cell_dtype, int n_bins, int cells_x, int cells_y, int r, int ncx);
// Whether the tensor-core score's grid gives every SM a CTA for this map.
bool score_tc_fills_gpu(int ncx, int ncy, int n_bins, int r);
hog_status launch_score_tc(const uint16_t* cells_bf16, int ncx, int ncy, int n_bins, int cells_x,
                           int cells_y, int r, const void* w, int w_dtype, float bias,
                           void* scores, cudaStream_t st);
// The row-GEMM tensor-core score (score_rows.cu): bf16 cells of 8 bins, 8 x 16-cell windows.
bool score_rows_supported(const void* cells, int cell_dtype, int n_bins, int cells_x, int cells_y, int r);
// n_filters filters of 1024 weights each, host biases (rounded for int8 weights by the launcher).
hog_status launch_score_rows(const uint16_t* cells_bf16, int ncx, int ncy, int r, const void* w, int w_dtype,
                             int n_filters, const float* biases, void* scores, cudaStream_t st);
bool cells_soft_supported(int n_bins, int cell, int stride);
hog_status launch_build_soft_lut(int n_bins, uint16_t* lut, cudaStream_t st);
hog_status launch_cells_soft(const uint8_t* img, int W, int H, int channels, size_t pitch, const uint16_t* lut,
                             int n_bins, int cell, int stride, int cell_dtype, void* cells, cudaStream_t st);
hog_status launch_block_norm(const void* cells, int cell_dtype, int ncx, int ncy, int nb, int r, float eps,
                             float* blocks, cudaStream_t st);
hog_status launch_score_tc_multi(const uint16_t* cells_bf16, int ncx, int ncy, int n_bins, int r, const void* w,
                                 int w_dtype, int n_filters, const float* biases, void* scores, cudaStream_t st);

bool cells_fused_supported(int n_bins, int cell, int stride);
hog_status launch_cells_fused(const uint8_t* img, int W, int H, int channels, size_t pitch, const uint8_t* lut,
                              int n_bins, int cell, int stride, int cell_dtype, void* cells, unsigned int* status,
                              cudaStream_t st);

size_t detect_workspace_bytes(int nx, int ny);
int detect_tiles(long n_scores);  // 2048-score tiles of a map (0 for an empty map)
hog_status launch_detect(const void* scores, int score_dtype, int nx, int ny, int stride, float thr,
                         int image, int level, hog_det* out, int max_out, int32_t* d_count, void* ws,
                         cudaStream_t st);

// ---- programmatic dependent launch
// Kernels of the detection path launch with programmatic stream
// serialisation: a kernel may start while its stream predecessor is still
// finishing.  Every such kernel calls pdl_wait() before it reads its
// predecessor's results or writes memory an earlier kernel reads (only
// independent set-up -- tables, weights, barriers -- runs before it), and
// pdl_trigger() right after: its successor is then scheduled while it runs,
// but no further ahead.  Triggering before the wait would let the whole
// chain of later kernels become resident and wait on the SMs at once, where
// their shared-memory reservations shrink the L1 cache of the kernel that is
// actually running.  The score and detection kernels at the tail of the
// path trigger before they wait: what follows them is small, and launching
// it early hides its launch latency.  Under stream capture the dependency
// becomes a programmatic graph edge.
template <typename... KArgs, typename... Args>
hog_status launch_pdl(void (*kernel)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t st,
                      Args&&... args) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    const cudaError_t e = cudaLaunchKernelEx(&cfg, kernel, static_cast<KArgs>(args)...);
    return e == cudaSuccess ? HOG_OK : cuda_fail(e);
}
// Raise kernel Kern's dynamic shared-memory limit on the current device to at
// least `bytes`.  The driver is called only when a launch needs more than the
// limit already set there (once per kernel and device in practice), so the
// attribute costs no host time on every launch.  Kern is the kernel itself,
// so every kernel keeps its own record.
template <auto Kern>
cudaError_t smem_at_least(size_t bytes) {
    constexpr int kDevices = 64;
    static std::atomic<int> have[kDevices];
    static std::mutex mu;
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    const int want = (int)bytes;
    if (dev < 0 || dev >= kDevices) return cudaFuncSetAttribute(Kern, cudaFuncAttributeMaxDynamicSharedMemorySize, want);
    if (have[dev].load(std::memory_order_acquire) >= want) return cudaSuccess;
    std::lock_guard<std::mutex> lock(mu);
    if (have[dev].load(std::memory_order_relaxed) >= want) return cudaSuccess;
    e = cudaFuncSetAttribute(Kern, cudaFuncAttributeMaxDynamicSharedMemorySize, want);
    if (e == cudaSuccess) have[dev].store(want, std::memory_order_release);
    return e;
}

__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void pdl_trigger() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }

// ---- small device helpers
__device__ __forceinline__ uint16_t f32_to_bf16_exact_int(float v) {
    // Only called on small integers (|v| < 2^8) and on values already
    // representable in bf16, where dropping the low 16 bits is exact.
    return static_cast<uint16_t>(__float_as_uint(v) >> 16);
}
__device__ __forceinline__ float bf16_to_f32(uint16_t h) {
    return __uint_as_float(static_cast<uint32_t>(h) << 16);
}

inline int ceil_div(long a, long b) { return static_cast<int>((a + b - 1) / b); }
// Positions of a box of `box` pixels stepped by `stride` along `extent` pixels.
inline int n_pos(int extent, int box, int stride) { return extent < box ? 0 : (extent - box) / stride + 1; }

}  // namespace fasthog
