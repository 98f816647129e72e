// batch_plan.cuh -- layout of a batch plan (include/fasthog_batch.h), shared
// by the batch API and the batch kernels.  The same bytes live in host memory
// (read by the API to size launches) and in device memory (read by kernels).
#pragma once

#include "../../include/fasthog_batch.h"
#include "internal.cuh"

namespace fasthog {

constexpr uint32_t kPlanMagic = 0x4E414C50u;  // "PLAN"
constexpr int kMaxBatchItems = 65536;

struct PlanHeader {
    uint32_t magic;
    int n_items, channels, n_bins, cell, stride, cells_x, cells_y, r;
    int cells_tiles;   // fused-cells tiles over the whole batch
    int score_tc;      // output rows per tensor-core CTA
    int score_ctas;    // tensor-core CTAs over the whole batch
    int detect_tiles;  // detection tiles over the whole batch
    int score_rows;    // 1: the row-GEMM tensor-core score (score_tc = output rows per CTA), 0: banded
    int pad[2];
};

struct PlanItem {
    hog_batch_item it;
    int ncx, ncy, nx, ny;
    int cells_t0, cells_tx;               // first fused tile of the item, fused tiles per tile row
    int score_c0, score_tx, score_bands;  // first tensor-core CTA, 128-window columns, row bands (ranges)
    int detect_t0;                        // first detection tile
    int pad[2];
};

static_assert(sizeof(PlanHeader) == 64, "plan header layout");
static_assert(sizeof(hog_batch_item) == 48, "batch item layout");
static_assert(sizeof(PlanItem) == 96, "plan item layout");

__host__ __device__ inline const PlanHeader* plan_header(const void* p) {
    return static_cast<const PlanHeader*>(p);
}
__host__ __device__ inline const PlanItem* plan_items(const void* p) {
    return reinterpret_cast<const PlanItem*>(static_cast<const char*>(p) + sizeof(PlanHeader));
}

// The item whose stage range holds global index t: the last item whose
// start is <= t (items with an empty range share their successor's start).
enum class Stage { kCells, kScore, kDetect };
template <Stage ST>
__device__ __forceinline__ int plan_start(const PlanItem* items, int i) {
    if constexpr (ST == Stage::kCells) return __ldg(&items[i].cells_t0);
    if constexpr (ST == Stage::kScore) return __ldg(&items[i].score_c0);
    return __ldg(&items[i].detect_t0);
}
template <Stage ST>
__device__ __forceinline__ int find_item(const PlanItem* items, int n, int t) {
    int lo = 0, hi = n - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (plan_start<ST>(items, mid) <= t) lo = mid;
        else hi = mid - 1;
    }
    return lo;
}

// Geometry helpers of the per-stage kernels, used by the planner.
int cells_fused_tiles_x(int ncx, int stride);
int cells_fused_tiles(int ncx, int ncy, int stride);
int score_tc_windows(int n_bins);  // windows per tensor-core CTA

// Batch launchers (kernels in cells_fused.cu, score_tc.cu, detect.cu).
hog_status launch_cells_fused_batch(const PlanHeader& h, const void* plan_dev, const uint8_t* lut, int cell_dtype,
                                    unsigned int* status, cudaStream_t st);
hog_status launch_score_tc_batch(const PlanHeader& h, const void* plan_dev, const void* w, int w_dtype, float bias,
                                 cudaStream_t st);
size_t detect_batch_workspace_bytes(const PlanHeader& h);
hog_status launch_detect_batch(const PlanHeader& h, const void* plan_dev, int score_dtype, float thr, hog_det* out,
                               int max_out, int32_t* d_count, int32_t* item_counts, void* ws, cudaStream_t st);
size_t pyramid_bytes(int W, int H, int channels, int levels);
int score_tc_rows_for(long ctas32);
// The row-GEMM score over a batch: output rows per CTA for strip_rows
// (128-window strips x output rows, summed over the items), and the launch.
int score_rows_batch_rows(long strip_rows);
hog_status launch_score_rows_batch(const PlanHeader& h, const void* plan_dev, const void* w, int w_dtype, float bias,
                                   cudaStream_t st);
hog_status launch_pyramid(const uint8_t* img, int W, int H, int channels, size_t pitch, int levels, uint8_t* out,
                          cudaStream_t st);

}  // namespace fasthog
