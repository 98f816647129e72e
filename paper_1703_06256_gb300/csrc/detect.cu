// detect.cu -- threshold the score map and compact the windows that pass
// into a list in row-major order (the detection step the paper's pipeline
// ends with, Sections 1 and 4).
//
// Two launches, no waiting between CTAs:
//   count    one CTA per tile of 2048 scores writes the tile's number of
//            windows with score >= thr to the workspace;
//   scatter  one CTA per tile sums the counts of the tiles before it (a block
//            reduction over at most a few thousand ints), scans its own flags
//            (warp shuffles + one cross-warp step), builds its run of the
//            list in shared memory and writes it with coalesced stores.  The
//            last tile writes the total.
// A map of a single tile skips the count launch.  Integer scores compare
// against ceil(thr), which for integers is the same test as >= thr.
#include <cmath>
#include <type_traits>

#include "detect_core.cuh"
#include "internal.cuh"

namespace fasthog {

namespace {

using detect::kDetWords;
using detect::kPer;
using detect::kThreads;
using detect::kTile;

template <typename T>
__global__ void __launch_bounds__(kThreads)
    detect_count_kernel(const T* __restrict__ scores, long n, float thr_f, int thr_i, int* __restrict__ tile_count) {
    __shared__ int red[kThreads / 32];
    pdl_trigger();
    pdl_wait();
    const int c = detect::tile_count<T>(scores, n, blockIdx.x, thr_f, thr_i, red);
    if (threadIdx.x == 0) tile_count[blockIdx.x] = c;
}

template <typename T>
__global__ void __launch_bounds__(kThreads)
    detect_scatter_kernel(const T* __restrict__ scores, int nx, long n, int stride, float thr_f, int thr_i,
                          int image, int level, const int* __restrict__ tile_count, hog_det* __restrict__ out,
                          int max_out, int* __restrict__ d_count) {
    __shared__ int red[kThreads / 32];
    __shared__ int wsum[kThreads / 32];
    __shared__ uint32_t stage[kTile * kDetWords];
    pdl_trigger();
    pdl_wait();
    // detections in the tiles before this one
    int before = 0;
    if (tile_count != nullptr)
        for (int t = threadIdx.x; t < (int)blockIdx.x; t += kThreads) before += __ldg(tile_count + t);
    before = detect::block_sum(before, red);
    const int tile_total = detect::tile_scatter<T>(scores, nx, n, blockIdx.x, stride, thr_f, thr_i, image, level,
                                                   before, out, max_out, stage, wsum);
    if (blockIdx.x == gridDim.x - 1 && threadIdx.x == 0) *d_count = before + tile_total;
}

template <typename T>
hog_status launch_t(const void* scores, int nx, int ny, int stride, float thr, int image, int level, hog_det* out,
                    int max_out, int32_t* d_count, void* ws, cudaStream_t st) {
    const long n = (long)nx * ny;
    const int tiles = n > 0 ? ceil_div(n, kTile) : 1;
    int thr_i = 0;
    if (std::is_same<T, int32_t>::value) {
        const double c = ceil((double)thr);
        thr_i = c > 2147483647.0 ? 2147483647 : (c < -2147483647.0 ? -2147483647 : (int)c);
    }
    int* tile_count = nullptr;
    if (tiles > 1) {
        tile_count = static_cast<int*>(ws);
        hog_status s = launch_pdl(detect_count_kernel<T>, dim3(tiles), dim3(kThreads), 0, st,
                                  static_cast<const T*>(scores), n, thr, thr_i, tile_count);
        if (s != HOG_OK) return s;
    }
    return launch_pdl(detect_scatter_kernel<T>, dim3(tiles), dim3(kThreads), 0, st, static_cast<const T*>(scores),
                      nx > 0 ? nx : 1, n, stride, thr, thr_i, image, level, (const int*)tile_count, out, max_out,
                      d_count);
}

}  // namespace

int detect_tiles(long n_scores) { return n_scores > 0 ? (int)((n_scores + kTile - 1) / kTile) : 0; }

size_t detect_workspace_bytes(int nx, int ny) {
    const long n = (long)nx * ny;
    const long tiles = n > 0 ? (n + kTile - 1) / kTile : 1;
    return (size_t)((tiles * 4 + 255) / 256 * 256);
}

hog_status launch_detect(const void* scores, int score_dtype, int nx, int ny, int stride, float thr, int image,
                         int level, hog_det* out, int max_out, int32_t* d_count, void* ws, cudaStream_t st) {
    if (score_dtype == HOG_I32)
        return launch_t<int32_t>(scores, nx, ny, stride, thr, image, level, out, max_out, d_count, ws, st);
    return launch_t<float>(scores, nx, ny, stride, thr, image, level, out, max_out, d_count, ws, st);
}

}  // namespace fasthog
