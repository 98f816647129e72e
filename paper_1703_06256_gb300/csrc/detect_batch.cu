// detect_batch.cu -- the detection step (threshold and ordered compaction,
// Sections 1 and 4) over every item of a batch plan, into one list.
//
// Three launches:
//   count    one CTA per detection tile of the batch (2048 scores of one
//            item) writes the tile's number of windows with score >= thr;
//   scan     one CTA turns the tile counts into list offsets (exclusive
//            scan in plan order), each item's count and the total;
//   scatter  one CTA per tile writes its detections at its offset, tagged
//            with its item's image and level.
#include <cmath>

#include "batch_plan.cuh"
#include "detect_core.cuh"
#include "internal.cuh"

namespace fasthog {

namespace {

using detect::kDetWords;
using detect::kThreads;
using detect::kTile;

constexpr int kScanThreads = 1024;

template <typename T>
__global__ void __launch_bounds__(kThreads)
    detect_count_batch_kernel(const PlanItem* __restrict__ items, int n_items, float thr_f, int thr_i,
                              int* __restrict__ tile_count) {
    __shared__ int red[kThreads / 32];
    pdl_trigger();  // tail of the path: the successor is small, launch it early
    pdl_wait();
    const int t = blockIdx.x;
    const PlanItem* it = items + find_item<Stage::kDetect>(items, n_items, t);
    const long n = (long)it->nx * it->ny;
    const int c = detect::tile_count<T>(static_cast<const T*>(it->it.scores), n, t - it->detect_t0, thr_f, thr_i,
                                        red);
    if (threadIdx.x == 0) tile_count[t] = c;
}

// Exclusive scan of the batch's tile counts by one CTA: each thread sums a
// contiguous run of tiles, the run totals are scanned across the CTA, then
// each thread writes its run's offsets.
__global__ void __launch_bounds__(kScanThreads)
    detect_scan_batch_kernel(const PlanItem* __restrict__ items, int n_items, int n_tiles,
                             const int* __restrict__ tile_count, int* __restrict__ tile_off, int* __restrict__ d_count,
                             int* __restrict__ item_counts) {
    __shared__ int wsum[kScanThreads / 32];
    __shared__ int total_s;
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
        int v = wsum[lane];
        int vi = v;
#pragma unroll
        for (int d = 1; d < 32; d <<= 1) {
            const int u = __shfl_up_sync(0xffffffffu, vi, d);
            if (lane >= d) vi += u;
        }
        wsum[lane] = vi - v;  // exclusive prefix of the warp totals
        if (lane == 31) total_s = vi;
    }
    __syncthreads();
    int off = wsum[warp] + incl - run;
    for (int t = t0; t < t1; ++t) {
        tile_off[t] = off;
        off += tile_count[t];
    }
    __syncthreads();  // tile_off complete for the item counts below
    const int total = total_s;
    if (tid == 0) *d_count = total;
    if (item_counts != nullptr) {
        for (int i = tid; i < n_items; i += kScanThreads) {
            const int a = items[i].detect_t0;
            const int b = i + 1 < n_items ? items[i + 1].detect_t0 : n_tiles;
            const int start = a < n_tiles ? tile_off[a] : total;
            const int end = b < n_tiles ? tile_off[b] : total;
            item_counts[i] = end - start;
        }
    }
}

template <typename T>
__global__ void __launch_bounds__(kThreads)
    detect_scatter_batch_kernel(const PlanItem* __restrict__ items, int n_items, int stride, float thr_f, int thr_i,
                                const int* __restrict__ tile_off, hog_det* __restrict__ out, int max_out) {
    __shared__ int wsum[kThreads / 32];
    __shared__ uint32_t stage[kTile * kDetWords];
    pdl_trigger();  // tail of the path: the successor is small, launch it early
    pdl_wait();
    const int t = blockIdx.x;
    const PlanItem* it = items + find_item<Stage::kDetect>(items, n_items, t);
    const int nx = it->nx;
    const long n = (long)nx * it->ny;
    detect::tile_scatter<T>(static_cast<const T*>(it->it.scores), nx, n, t - it->detect_t0, stride, thr_f, thr_i,
                            it->it.image, it->it.level, tile_off[t], out, max_out, stage, wsum);
}

template <typename T>
hog_status launch_t(const PlanHeader& h, const void* plan_dev, float thr, hog_det* out, int max_out,
                    int32_t* d_count, int32_t* item_counts, void* ws, cudaStream_t st) {
    int thr_i = 0;
    if (std::is_same<T, int32_t>::value) {
        const double c = ceil((double)thr);
        thr_i = c > 2147483647.0 ? 2147483647 : (c < -2147483648.0 ? (int)(-2147483647 - 1) : (int)c);
    }
    const PlanItem* items = plan_items(plan_dev);
    const int T_ = h.detect_tiles;
    int* tile_count = static_cast<int*>(ws);
    int* tile_off = tile_count + T_;
    hog_status s = HOG_OK;
    if (T_ > 0)
        s = launch_pdl(detect_count_batch_kernel<T>, dim3(T_), dim3(kThreads), 0, st, items, h.n_items, thr, thr_i,
                       tile_count);
    if (s == HOG_OK)
        s = launch_pdl(detect_scan_batch_kernel, dim3(1), dim3(kScanThreads), 0, st, items, h.n_items, T_,
                       (const int*)tile_count, tile_off, d_count, item_counts);
    if (s == HOG_OK && T_ > 0)
        s = launch_pdl(detect_scatter_batch_kernel<T>, dim3(T_), dim3(kThreads), 0, st, items, h.n_items, h.stride,
                       thr, thr_i, (const int*)tile_off, out, max_out);
    return s;
}

}  // namespace

size_t detect_batch_workspace_bytes(const PlanHeader& h) {
    return (size_t)(((long)h.detect_tiles * 8 + 255) / 256 * 256 + 256);
}

hog_status launch_detect_batch(const PlanHeader& h, const void* plan_dev, int score_dtype, float thr, hog_det* out,
                               int max_out, int32_t* d_count, int32_t* item_counts, void* ws, cudaStream_t st) {
    if (score_dtype == HOG_I32)
        return launch_t<int32_t>(h, plan_dev, thr, out, max_out, d_count, item_counts, ws, st);
    return launch_t<float>(h, plan_dev, thr, out, max_out, d_count, item_counts, ws, st);
}

}  // namespace fasthog
