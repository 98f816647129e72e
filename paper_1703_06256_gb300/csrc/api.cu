// api.cu -- the extern "C" entry points of libfasthog (include/fasthog.h):
// argument checks, then one launcher per stage.  No entry point allocates,
// synchronises or falls back to the host: a stage runs on the GPU or the
// call returns an error without enqueueing anything.
#include <atomic>
#include <cmath>
#include <cstring>

#include "internal.cuh"

namespace fasthog {

namespace {
std::atomic<int> g_tune[HOG_TUNE_KNOBS];
thread_local int t_last_cuda_error = 0;
constexpr int kMaxDevices = 64;
int g_sm_count[kMaxDevices] = {0};
unsigned int* g_status_ptr[kMaxDevices] = {nullptr};
}  // namespace

// Device-side status bits (kStatusTimeout, ...), OR-ed by kernels whose
// bounded waits gave up.  Read and cleared by hog_device_status().
__device__ unsigned int g_device_status;

hog_status cuda_fail(cudaError_t e) {
    t_last_cuda_error = (int)e;
    return HOG_ERR_CUDA;
}

hog_status check_launch() {
    const cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? HOG_OK : cuda_fail(e);
}

int sm_count() {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return kNumSMs;
    if (g_sm_count[dev] == 0) {
        int n = 0;
        if (cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || n <= 0) n = kNumSMs;
        g_sm_count[dev] = n;
    }
    return g_sm_count[dev];
}

// Device address of g_device_status on the current device (looked up once
// per device, with that device current).
hog_status device_status_word(unsigned int** out) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return cuda_fail(e);
    if (dev < 0 || dev >= kMaxDevices) return HOG_ERR_UNSUPPORTED;
    if (g_status_ptr[dev] == nullptr) {
        void* p = nullptr;
        e = cudaGetSymbolAddress(&p, g_device_status);
        if (e != cudaSuccess) return cuda_fail(e);
        g_status_ptr[dev] = static_cast<unsigned int*>(p);
    }
    *out = g_status_ptr[dev];
    return HOG_OK;
}

int tune_get(int knob) {
    return knob >= 0 && knob < HOG_TUNE_KNOBS ? g_tune[knob].load(std::memory_order_relaxed) : 0;
}

// int8 weights promise exact int32 scores.  Every kernel accumulates in f32,
// which is exact while every partial sum is an integer below 2^24 in
// magnitude.  A cell of hard votes holds at most cell^2 counts over all its
// bins, so |partial sum| <= 127 * cells_x * cells_y * cell^2 + |round(bias)|.
static bool i8_exact(int cells_x, int cells_y, int cell, double bias_rounded) {
    const double bound = 127.0 * cells_x * cells_y * (double)cell * cell + std::fabs(bias_rounded);
    return bound < 16777216.0;
}

static bool size_ok(int W, int H) { return W >= 1 && H >= 1 && W <= 65535 && H <= 65535 && (long)W * H < (1L << 31); }

}  // namespace fasthog

using namespace fasthog;

extern "C" {

hog_status hog_tune_set(int knob, int value) {
    bool ok = value == 0;
    switch (knob) {
        case HOG_TUNE_INTEGRAL_BAND_ROWS: ok = ok || value == 4 || value == 8 || value == 16 || value == 32; break;
        case HOG_TUNE_BINMAP_CTAS_PER_SM: ok = ok || (value >= 1 && value <= 8); break;
        case HOG_TUNE_FUSED_CTAS_PER_SM: ok = ok || value == 1 || value == 2; break;
        case HOG_TUNE_SCORE_TC_ROWS:
            ok = ok || value == 1 || value == 2 || value == 4 || value == 8 || value == 16 || value == 32 ||
                 value == 64;
            break;
        case HOG_TUNE_TABLE: ok = ok || value == 1 || value == 2; break;
        case HOG_TUNE_CELL_ROWS: ok = ok || value == 1 || value == 4 || value == 8 || value == 16; break;
        case HOG_TUNE_SCORE_PATH: ok = ok || value == 1 || value == 2 || value == 3; break;
        case HOG_TUNE_SLIDE_WINDOWS: ok = ok || value == 8 || value == 16; break;
        case HOG_TUNE_INTEGRAL_PATH: ok = ok || value == 1 || value == 2 || value == 3; break;
        case HOG_TUNE_INTEGRAL_WARP_ROWS: ok = ok || value == 2 || value == 4 || value == 8; break;
        case HOG_TUNE_BINMAP_SCHEDULE: ok = ok || value == 1 || value == 2; break;
        case HOG_TUNE_FUSED_TILE_ROWS: ok = ok || value == 4 || value == 8 || value == 16; break;
        default: return HOG_ERR_ARG;
    }
    if (!ok) return HOG_ERR_ARG;
    g_tune[knob].store(value, std::memory_order_relaxed);
    return HOG_OK;
}

int hog_tune_get(int knob) {
    return knob >= 0 && knob < HOG_TUNE_KNOBS ? g_tune[knob].load(std::memory_order_relaxed) : -1;
}

const char* hog_status_string(hog_status s) {
    switch (s) {
        case HOG_OK: return "HOG_OK";
        case HOG_ERR_ARG: return "HOG_ERR_ARG";
        case HOG_ERR_UNSUPPORTED: return "HOG_ERR_UNSUPPORTED";
        case HOG_ERR_CUDA: return "HOG_ERR_CUDA";
        case HOG_ERR_TIMEOUT: return "HOG_ERR_TIMEOUT";
    }
    return "HOG_ERR_UNKNOWN";
}

int hog_last_cuda_error(void) { return t_last_cuda_error; }

int hog_version(void) { return 100; }

hog_status hog_device_status(uint32_t* flags, int clear) {
    if (flags == nullptr) return HOG_ERR_ARG;
    unsigned int* p = nullptr;
    hog_status s = device_status_word(&p);
    if (s != HOG_OK) return s;
    unsigned int v = 0;
    cudaError_t e = cudaMemcpy(&v, p, sizeof(v), cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return cuda_fail(e);
    if (clear) {
        const unsigned int z = 0;
        e = cudaMemcpy(p, &z, sizeof(z), cudaMemcpyHostToDevice);
        if (e != cudaSuccess) return cuda_fail(e);
    }
    *flags = v;
    return HOG_OK;
}

hog_status hog_build_lut(int n_bins, uint8_t* lut, hog_stream_t stream) {
    if (lut == nullptr || n_bins < 1 || n_bins > kMaxBins) return HOG_ERR_ARG;
    if (reinterpret_cast<uintptr_t>(lut) % 16 != 0) return HOG_ERR_ARG;
    LutParams p;
    std::memset(&p, 0, sizeof(p));
    p.n_bins = n_bins;
    const long long one = 1LL << 40;
    const long long half_sqrt2 = std::llround(std::ldexp(std::sqrt(0.5), 40));
    static const int dir8[8][2] = {{1, 0}, {1, 1}, {0, 1}, {-1, 1}, {-1, 0}, {-1, -1}, {0, -1}, {1, -1}};
    for (int k = 1; k < n_bins; ++k) {
        if ((8 * k) % n_bins == 0) {
            // multiple of pi/4: exact directions (equal magnitudes on the diagonals)
            const int m = 8 * k / n_bins;
            const long long mag = (m & 1) ? half_sqrt2 : one;
            p.c[k] = dir8[m][0] * mag;
            p.s[k] = dir8[m][1] * mag;
        } else {
            const double th = 2.0 * M_PI * (double)k / (double)n_bins;
            p.c[k] = std::llround(std::ldexp(std::cos(th), 40));
            p.s[k] = std::llround(std::ldexp(std::sin(th), 40));
        }
    }
    return launch_build_lut(p, lut, reinterpret_cast<cudaStream_t>(stream));
}

hog_status hog_bin_map(const uint8_t* img, int W, int H, int channels, size_t pitch_bytes, const uint8_t* lut,
                       int n_bins, uint8_t* bins, hog_stream_t stream) {
    if (img == nullptr || lut == nullptr || bins == nullptr) return HOG_ERR_ARG;
    if (!size_ok(W, H) || (channels != 1 && channels != 3)) return HOG_ERR_ARG;
    if (pitch_bytes < (size_t)W * channels || n_bins < 1 || n_bins > kMaxBins) return HOG_ERR_ARG;
    if (reinterpret_cast<uintptr_t>(lut) % 16 != 0) return HOG_ERR_ARG;
    unsigned int* status = nullptr;
    hog_status s = device_status_word(&status);
    if (s != HOG_OK) return s;
    return launch_bin_map(img, W, H, channels, pitch_bytes, lut, n_bins, bins, status,
                          reinterpret_cast<cudaStream_t>(stream));
}

size_t hog_integral_workspace_bytes(int W, int H, int n_bins) {
    if (!size_ok(W, H) || n_bins < 1 || n_bins > kMaxBins) return 0;
    return integral_workspace_bytes(W, H, n_bins);
}

int hog_integral_launches(int W, int H, int n_bins) {
    if (!size_ok(W, H) || n_bins < 1 || n_bins > kMaxBins) return 0;
    return integral_launches(W, H, n_bins);
}

hog_status hog_integral(const uint8_t* bins, int W, int H, int n_bins, int ii_dtype, void* ii, void* workspace,
                        size_t workspace_bytes, hog_stream_t stream) {
    if (bins == nullptr || ii == nullptr || workspace == nullptr) return HOG_ERR_ARG;
    if (!size_ok(W, H) || n_bins < 1 || n_bins > kMaxBins) return HOG_ERR_ARG;
    if (ii_dtype != HOG_I32 && ii_dtype != HOG_U16) return HOG_ERR_ARG;
    if (reinterpret_cast<uintptr_t>(workspace) % 256 != 0) return HOG_ERR_ARG;
    if (workspace_bytes < integral_workspace_bytes(W, H, n_bins)) return HOG_ERR_ARG;
    return launch_integral(bins, W, H, n_bins, ii_dtype, ii, workspace, reinterpret_cast<cudaStream_t>(stream));
}

hog_status hog_cell_hist(const void* ii, int W, int H, int n_bins, int ii_dtype, int cell, int stride,
                         int cell_dtype, void* cells, hog_stream_t stream) {
    if (ii == nullptr || cells == nullptr) return HOG_ERR_ARG;
    if (!size_ok(W, H) || n_bins < 1 || n_bins > kMaxBins) return HOG_ERR_ARG;
    if (ii_dtype != HOG_I32 && ii_dtype != HOG_U16) return HOG_ERR_ARG;
    if (cell < 1 || cell > 64 || stride < 1 || stride > cell) return HOG_ERR_ARG;
    if (cell_dtype != HOG_I32 && cell_dtype != HOG_BF16 && cell_dtype != HOG_F32) return HOG_ERR_ARG;
    if (cell_dtype == HOG_BF16 && cell > 16) return HOG_ERR_ARG;  // counts above 256 are not exact in bf16
    return launch_cell_hist(ii, W, H, n_bins, ii_dtype, cell, stride, cell_dtype, cells,
                            reinterpret_cast<cudaStream_t>(stream));
}

hog_status hog_cell_hist_fused(const uint8_t* img, int W, int H, int channels, size_t pitch_bytes,
                               const uint8_t* lut, int n_bins, int cell, int stride, int cell_dtype, void* cells,
                               hog_stream_t stream) {
    if (img == nullptr || lut == nullptr || cells == nullptr) return HOG_ERR_ARG;
    if (!size_ok(W, H) || (channels != 1 && channels != 3)) return HOG_ERR_ARG;
    if (pitch_bytes < (size_t)W * channels || n_bins < 1 || n_bins > kMaxBins) return HOG_ERR_ARG;
    if (reinterpret_cast<uintptr_t>(lut) % 16 != 0) return HOG_ERR_ARG;
    if (cell < 1 || cell > 64 || stride < 1 || stride > cell) return HOG_ERR_ARG;
    if (cell_dtype != HOG_I32 && cell_dtype != HOG_BF16 && cell_dtype != HOG_F32) return HOG_ERR_ARG;
    if (cell_dtype == HOG_BF16 && cell > 16) return HOG_ERR_ARG;
    if (!cells_fused_supported(n_bins, cell, stride)) return HOG_ERR_UNSUPPORTED;
    unsigned int* status = nullptr;
    hog_status s = device_status_word(&status);
    if (s != HOG_OK) return s;
    return launch_cells_fused(img, W, H, channels, pitch_bytes, lut, n_bins, cell, stride, cell_dtype, cells, status,
                              reinterpret_cast<cudaStream_t>(stream));
}

hog_status hog_window_score(const void* cells, int cell_dtype, int ncx, int ncy, int n_bins, int cells_x, int cells_y,
                            int cell, int stride, const void* w, int w_dtype, float bias, void* scores,
                            hog_stream_t stream) {
    if (cells == nullptr || w == nullptr || scores == nullptr) return HOG_ERR_ARG;
    if (ncx < 0 || ncy < 0 || n_bins < 1 || n_bins > kMaxBins) return HOG_ERR_ARG;
    if (cells_x < 1 || cells_y < 1 || cells_x > 64 || cells_y > 64) return HOG_ERR_ARG;
    if (cell < 1 || stride < 1 || cell % stride != 0) return HOG_ERR_ARG;
    if (cell_dtype != HOG_I32 && cell_dtype != HOG_BF16 && cell_dtype != HOG_F32) return HOG_ERR_ARG;
    if (w_dtype != HOG_F32 && w_dtype != HOG_BF16 && w_dtype != HOG_I8) return HOG_ERR_ARG;
    if (!std::isfinite(bias)) return HOG_ERR_ARG;
    if (w_dtype == HOG_I8 && !i8_exact(cells_x, cells_y, cell, (double)std::llround((double)bias)))
        return HOG_ERR_UNSUPPORTED;
    const int r = cell / stride;
    const float b = w_dtype == HOG_I8 ? (float)std::llround((double)bias) : bias;
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    const bool rows = score_rows_supported(cells, cell_dtype, n_bins, cells_x, cells_y, r);
    const bool tc = score_tc_supported(cell_dtype, n_bins, cells_x, cells_y, r, ncx);
    const bool slide = score_slide_supported(cells, n_bins, cells_x, cells_y, r);
    const int path = tune_get(HOG_TUNE_SCORE_PATH);
    // automatic: bf16 cells of 8 bins on the row-GEMM tensor-core kernel (any weights); other bf16 cells
    // on the banded tensor-core kernel for bf16 and int8 weights, and for f32 weights (three MMAs per
    // step) when the map alone fills the GPU, else on the CUDA cores
    if (rows && path != 1)
        return launch_score_rows(static_cast<const uint16_t*>(cells), ncx, ncy, r, w, w_dtype, 1, &b, scores, st);
    const bool auto_tc = w_dtype != HOG_F32 || !slide || score_tc_fills_gpu(ncx, ncy, n_bins, r);
    const bool use_tc = tc && (path == 2 || (path == 0 && auto_tc));
    if (use_tc)
        return launch_score_tc(static_cast<const uint16_t*>(cells), ncx, ncy, n_bins, cells_x, cells_y, r, w,
                               w_dtype, b, scores, st);
    if (slide)
        return launch_score_slide(cells, cell_dtype, ncx, ncy, r, w, w_dtype, b, scores, st);
    return launch_score_cuda_cores(cells, cell_dtype, ncx, ncy, n_bins, cells_x, cells_y, r, w, w_dtype, b, scores,
                                   st);
}

hog_status hog_build_soft_lut(int n_bins, uint16_t* lut, hog_stream_t stream) {
    if (lut == nullptr || reinterpret_cast<uintptr_t>(lut) % 4 != 0) return HOG_ERR_ARG;
    if (n_bins < 1 || n_bins > kMaxBins) return HOG_ERR_ARG;
    return launch_build_soft_lut(n_bins, lut, reinterpret_cast<cudaStream_t>(stream));
}

hog_status hog_cell_hist_soft(const uint8_t* img, int W, int H, int channels, size_t pitch_bytes,
                              const uint16_t* soft_lut, int n_bins, int cell, int stride, int cell_dtype,
                              void* cells, hog_stream_t stream) {
    if (img == nullptr || soft_lut == nullptr || cells == nullptr) return HOG_ERR_ARG;
    if (!size_ok(W, H) || (channels != 1 && channels != 3)) return HOG_ERR_ARG;
    if (pitch_bytes < (size_t)W * channels || n_bins < 1 || n_bins > kMaxBins) return HOG_ERR_ARG;
    if (cell < 1 || cell > 64 || stride < 1 || stride > cell) return HOG_ERR_ARG;
    if (cell_dtype != HOG_I32 && cell_dtype != HOG_F32) return HOG_ERR_ARG;
    if (reinterpret_cast<uintptr_t>(cells) % 4 != 0 || reinterpret_cast<uintptr_t>(soft_lut) % 4 != 0)
        return HOG_ERR_ARG;
    if (!cells_soft_supported(n_bins, cell, stride)) return HOG_ERR_UNSUPPORTED;
    return launch_cells_soft(img, W, H, channels, pitch_bytes, soft_lut, n_bins, cell, stride, cell_dtype, cells,
                             reinterpret_cast<cudaStream_t>(stream));
}

hog_status hog_block_norm(const void* cells, int cell_dtype, int ncx, int ncy, int n_bins, int r, float eps,
                          float* blocks, hog_stream_t stream) {
    if (cells == nullptr || blocks == nullptr) return HOG_ERR_ARG;
    if (ncx < 0 || ncy < 0 || n_bins < 1 || n_bins > kMaxBins || r < 1) return HOG_ERR_ARG;
    if (cell_dtype != HOG_I32 && cell_dtype != HOG_BF16 && cell_dtype != HOG_F32) return HOG_ERR_ARG;
    if (!(eps >= 0.f) || !std::isfinite(eps)) return HOG_ERR_ARG;
    if ((long)(ncx - r > 0 ? ncx - r : 0) * (ncy - r > 0 ? ncy - r : 0) * 4 * n_bins >= (1L << 31)) return HOG_ERR_ARG;
    return launch_block_norm(cells, cell_dtype, ncx, ncy, n_bins, r, eps, blocks,
                             reinterpret_cast<cudaStream_t>(stream));
}

hog_status hog_window_score_multi(const void* cells, int cell_dtype, int ncx, int ncy, int n_bins, int cells_x,
                                  int cells_y, int cell, int stride, const void* w, int w_dtype, int n_filters,
                                  const float* biases, void* scores, hog_stream_t stream) {
    if (cells == nullptr || w == nullptr || scores == nullptr || biases == nullptr) return HOG_ERR_ARG;
    if (n_filters < 1 || n_filters > 1024) return HOG_ERR_ARG;
    if (ncx < 0 || ncy < 0 || n_bins < 1 || n_bins > kMaxBins) return HOG_ERR_ARG;
    if (cells_x < 1 || cells_y < 1 || cells_x > 64 || cells_y > 64) return HOG_ERR_ARG;
    if (cell < 1 || stride < 1 || cell % stride != 0) return HOG_ERR_ARG;
    if (cell_dtype != HOG_I32 && cell_dtype != HOG_BF16 && cell_dtype != HOG_F32) return HOG_ERR_ARG;
    if (w_dtype != HOG_F32 && w_dtype != HOG_BF16 && w_dtype != HOG_I8) return HOG_ERR_ARG;
    for (int f = 0; f < n_filters; ++f) {
        if (!std::isfinite(biases[f])) return HOG_ERR_ARG;
        if (w_dtype == HOG_I8 && !i8_exact(cells_x, cells_y, cell, (double)std::llround((double)biases[f])))
            return HOG_ERR_UNSUPPORTED;
    }
    const int r = cell / stride;
    const long nx = (long)ncx - (long)(cells_x - 1) * r, ny = (long)ncy - (long)(cells_y - 1) * r;
    if (nx <= 0 || ny <= 0) return HOG_OK;
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    // 8 bins: the row-GEMM kernel, several filters per pass, each scored exactly as alone
    if (score_rows_supported(cells, cell_dtype, n_bins, cells_x, cells_y, r) &&
        tune_get(HOG_TUNE_SCORE_PATH) != 1)
        return launch_score_rows(static_cast<const uint16_t*>(cells), ncx, ncy, r, w, w_dtype, n_filters, biases,
                                 scores, st);
    if (score_tc_supported(cell_dtype, n_bins, cells_x, cells_y, r, ncx) &&
        reinterpret_cast<uintptr_t>(cells) % 16 == 0)
        return launch_score_tc_multi(static_cast<const uint16_t*>(cells), ncx, ncy, n_bins, r, w, w_dtype, n_filters,
                                     biases, scores, st);
    // otherwise the single-filter kernels, one filter at a time
    const size_t esize = w_dtype == HOG_F32 ? 4 : (w_dtype == HOG_BF16 ? 2 : 1);
    const size_t k = (size_t)cells_x * cells_y * n_bins;
    for (int f = 0; f < n_filters; ++f) {
        hog_status s = hog_window_score(cells, cell_dtype, ncx, ncy, n_bins, cells_x, cells_y, cell, stride,
                                        static_cast<const uint8_t*>(w) + f * k * esize, w_dtype, biases[f],
                                        static_cast<uint8_t*>(scores) + (size_t)f * nx * ny * 4, stream);
        if (s != HOG_OK) return s;
    }
    return HOG_OK;
}

size_t hog_detect_workspace_bytes(int nx, int ny) {
    if (nx < 0 || ny < 0) return 0;
    return detect_workspace_bytes(nx, ny);
}

hog_status hog_detect(const void* scores, int score_dtype, int nx, int ny, int stride, float thr, int image,
                      int level, hog_det* out, int max_out, int32_t* d_count, void* workspace, size_t workspace_bytes,
                      hog_stream_t stream) {
    if (scores == nullptr || d_count == nullptr || workspace == nullptr) return HOG_ERR_ARG;
    if (out == nullptr && max_out > 0) return HOG_ERR_ARG;
    if (reinterpret_cast<uintptr_t>(out) % alignof(hog_det) != 0) return HOG_ERR_ARG;
    if (nx < 0 || ny < 0 || (long)nx * ny >= (1L << 31) || stride < 1 || max_out < 0) return HOG_ERR_ARG;
    if (score_dtype != HOG_F32 && score_dtype != HOG_I32) return HOG_ERR_ARG;
    if (std::isnan(thr)) return HOG_ERR_ARG;
    if (workspace_bytes < detect_workspace_bytes(nx, ny)) return HOG_ERR_ARG;
    if (reinterpret_cast<uintptr_t>(workspace) % 8 != 0) return HOG_ERR_ARG;
    return launch_detect(scores, score_dtype, nx, ny, stride, thr, image, level, out, max_out, d_count, workspace,
                         reinterpret_cast<cudaStream_t>(stream));
}

}  // extern "C"
