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
// A map of a single tile skips the count launch; a map of more than 2048
// tiles scans the tile counts in one CTA between the two launches (the
// scatter then reads its offset instead of summing).  Integer scores compare
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
    pdl_trigger();  // tail of the path: the successor is small, launch it early
    pdl_wait();
    const int c = detect::tile_count<T>(scores, n, blockIdx.x, thr_f, thr_i, red);
    if (threadIdx.x == 0) tile_count[blockIdx.x] = c;
}

template <typename T>
__global__ void __launch_bounds__(kThreads)
    detect_scatter_kernel(const T* __restrict__ scores, int nx, long n, int stride, float thr_f, int thr_i,
                          int image, int level, const int* __restrict__ tile_count,
                          const int* __restrict__ tile_off, hog_det* __restrict__ out, int max_out,
                          int* __restrict__ d_count) {
    __shared__ int red[kThreads / 32];
    __shared__ int wsum[kThreads / 32];
    __shared__ uint32_t stage[kTile * kDetWords];
    pdl_trigger();  // tail of the path: the successor is small, launch it early
    pdl_wait();
    // detections in the tiles before this one: scanned offsets, or the sum of the counts before
    int before = 0;
    if (tile_off != nullptr) {
        before = __ldg(tile_off + blockIdx.x);
    } else {
        if (tile_count != nullptr)
            for (int t = threadIdx.x; t < (int)blockIdx.x; t += kThreads) before += __ldg(tile_count + t);
        before = detect::block_sum(before, red);
    }
    const int tile_total = detect::tile_scatter<T>(scores, nx, n, blockIdx.x, stride, thr_f, thr_i, image, level,
                                                   before, out, max_out, stage, wsum);
    if (blockIdx.x == gridDim.x - 1 && threadIdx.x == 0) *d_count = before + tile_total;
}

// Exclusive scan of the tile counts by one CTA (maps of many tiles, where
// summing the counts before each tile would grow with the square of the
// tile count): each thread sums a contiguous run of tiles, the run totals
// are scanned across the CTA, then each thread writes its run's offsets.
constexpr int kScanThreads = 1024;
constexpr int kScanAbove = 2048;  // tiles

__global__ void __launch_bounds__(kScanThreads)
    detect_scan_kernel(const int* __restrict__ tile_count, int n_tiles, int* __restrict__ tile_off) {
    __shared__ int wsum[kScanThreads / 32];
    pdl_trigger();  // tail of the path: the successor is small, launch it early
    pdl_wait();
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int per = (n_tiles + kScanThreads - 1) / kScanThreads;
    const int t0 = min(tid * per, n_tiles), t1 = min(t0 + per, n_tiles);
    int run = 0;
    for (int t = t0; t < t1; ++t) run += tile_count[t];
    int incl = run;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
        const int u = __shfl_up_sync(0xffffffffu, incl, d);
        if (lane >= d) incl += u;
    }
    if (lane == 31) wsum[warp] = incl;
    __syncthreads();
    if (warp == 0) {
        const int v = wsum[lane];
        int vi = v;
#pragma unroll
        for (int d = 1; d < 32; d <<= 1) {
            const int u = __shfl_up_sync(0xffffffffu, vi, d);
            if (lane >= d) vi += u;
        }
        wsum[lane] = vi - v;
    }
    __syncthreads();
    int off = wsum[warp] + incl - run;
    for (int t = t0; t < t1; ++t) {
        tile_off[t] = off;
        off += tile_count[t];
    }
}

template <typename T>
hog_status launch_t(const void* scores, int nx, int ny, int stride, float thr, int image, int level, hog_det* out,
                    int max_out, int32_t* d_count, void* ws, size_t ws_bytes, cudaStream_t st) {
    const long n = (long)nx * ny;
    const int tiles = n > 0 ? ceil_div(n, kTile) : 1;
    int thr_i = 0;
    if (std::is_same<T, int32_t>::value) {
        const double c = ceil((double)thr);
        thr_i = c > 2147483647.0 ? 2147483647 : (c < -2147483647.0 ? -2147483647 : (int)c);
    }
    int* tile_count = nullptr;
    int* tile_off = nullptr;
    if (tiles > 1) {
        tile_count = static_cast<int*>(ws);
        hog_status s = launch_pdl(detect_count_kernel<T>, dim3(tiles), dim3(kThreads), 0, st,
                                  static_cast<const T*>(scores), n, thr, thr_i, tile_count);
        if (s != HOG_OK) return s;
        if (tiles > kScanAbove && ws_bytes >= (size_t)tiles * 8) {
            tile_off = tile_count + tiles;
            s = launch_pdl(detect_scan_kernel, dim3(1), dim3(kScanThreads), 0, st, (const int*)tile_count, tiles,
                           tile_off);
            if (s != HOG_OK) return s;
        }
    }
    return launch_pdl(detect_scatter_kernel<T>, dim3(tiles), dim3(kThreads), 0, st, static_cast<const T*>(scores),
                      nx > 0 ? nx : 1, n, stride, thr, thr_i, image, level, (const int*)tile_count,
                      (const int*)tile_off, out, max_out, d_count);
}

}  // namespace

int detect_tiles(long n_scores) { return n_scores > 0 ? (int)((n_scores + kTile - 1) / kTile) : 0; }

size_t detect_workspace_bytes(int nx, int ny) {
    const long n = (long)nx * ny;
    const long tiles = n > 0 ? (n + kTile - 1) / kTile : 1;
    const long words = tiles > kScanAbove ? 2 * tiles : tiles;  // counts, and offsets for many tiles
    return (size_t)((words * 4 + 255) / 256 * 256);
}

hog_status launch_detect(const void* scores, int score_dtype, int nx, int ny, int stride, float thr, int image,
                         int level, hog_det* out, int max_out, int32_t* d_count, void* ws, size_t ws_bytes,
                         cudaStream_t st) {
    if (score_dtype == HOG_I32)
        return launch_t<int32_t>(scores, nx, ny, stride, thr, image, level, out, max_out, d_count, ws, ws_bytes, st);
    return launch_t<float>(scores, nx, ny, stride, thr, image, level, out, max_out, d_count, ws, ws_bytes, st);
}

}  // namespace fasthog
