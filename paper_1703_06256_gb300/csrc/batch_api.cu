// batch_api.cu -- the extern "C" entry points of include/fasthog_batch.h:
// the host-side planner, argument checks, and one launcher per stage.
#include <cmath>
#include <cstring>

#include "batch_plan.cuh"
#include "internal.cuh"

using namespace fasthog;

namespace {

// The host copy of a plan, if it is one.
const PlanHeader* checked_plan(const void* plan) {
    if (plan == nullptr || reinterpret_cast<uintptr_t>(plan) % 8 != 0) return nullptr;
    const PlanHeader* h = plan_header(plan);
    if (h->magic != kPlanMagic || h->n_items < 1 || h->n_items > kMaxBatchItems) return nullptr;
    return h;
}

bool plan_dev_ok(const void* plan_dev) {
    return plan_dev != nullptr && reinterpret_cast<uintptr_t>(plan_dev) % 16 == 0;
}

}  // namespace

extern "C" {

size_t hog_batch_plan_bytes(int n_items) {
    if (n_items < 1 || n_items > kMaxBatchItems) return 0;
    return sizeof(PlanHeader) + (size_t)n_items * sizeof(PlanItem);
}

hog_status hog_batch_plan(const hog_batch_item* items, int n_items, int channels, int n_bins, int cell, int stride,
                          int cells_x, int cells_y, void* plan, size_t plan_bytes) {
    if (items == nullptr || plan == nullptr || reinterpret_cast<uintptr_t>(plan) % 8 != 0) return HOG_ERR_ARG;
    if (n_items < 1 || n_items > kMaxBatchItems || plan_bytes < hog_batch_plan_bytes(n_items)) return HOG_ERR_ARG;
    if (channels != 1 && channels != 3) return HOG_ERR_ARG;
    if (cells_x < 1 || cells_y < 1 || cells_x > 64 || cells_y > 64) return HOG_ERR_ARG;
    if (cell < 1 || stride < 1 || cell % stride != 0) return HOG_ERR_ARG;
    if (!cells_fused_supported(n_bins, cell, stride)) return HOG_ERR_UNSUPPORTED;
    const int r = cell / stride;
    // 8 bins, 8 x 16 cells: the row-GEMM score (strips of 128 windows by ranges of rows); otherwise the
    // banded tensor-core score (score_tc_windows() windows by Tc rows of one residue class)
    const bool rows = n_bins == 8 && cells_x == 8 && cells_y == 16 && (r == 1 || r == 2 || r == 4);
    const int wpc = rows ? 128 : score_tc_windows(n_bins);
    // first pass: sizes, and the tensor-core row count the whole batch supports
    long ctas32 = 0, strip_rows = 0;
    for (int i = 0; i < n_items; ++i) {
        const hog_batch_item& it = items[i];
        if (it.img == nullptr || it.cells == nullptr) return HOG_ERR_ARG;
        if (it.W < 1 || it.H < 1 || it.W > 65535 || it.H > 65535 || (long)it.W * it.H >= (1L << 31))
            return HOG_ERR_ARG;
        if (it.pitch < (size_t)it.W * channels) return HOG_ERR_ARG;
        const int ncx = n_pos(it.W, cell, stride), ncy = n_pos(it.H, cell, stride);
        const int nx = ncx - (cells_x - 1) * r, ny = ncy - (cells_y - 1) * r;
        if (nx > 0 && ny > 0) {
            if (it.scores == nullptr) return HOG_ERR_ARG;
            ctas32 += (long)((nx + wpc - 1) / wpc) * ((ny + 32 * r - 1) / (32 * r)) * r;
            strip_rows += (long)((nx + wpc - 1) / wpc) * ny;
        }
    }
    const int Tc = rows ? score_rows_batch_rows(strip_rows) : score_tc_rows_for(ctas32);
    const int band_rows = rows ? Tc : Tc * r;  // output rows of one CTA's range (all residues, or one class)
    const int classes = rows ? 1 : r;
    PlanHeader* h = static_cast<PlanHeader*>(plan);
    std::memset(h, 0, sizeof(PlanHeader));
    PlanItem* out = const_cast<PlanItem*>(plan_items(plan));
    long cells_t = 0, score_c = 0, detect_t = 0;
    for (int i = 0; i < n_items; ++i) {
        const hog_batch_item& it = items[i];
        PlanItem& p = out[i];
        std::memset(&p, 0, sizeof(PlanItem));
        p.it = it;
        p.ncx = n_pos(it.W, cell, stride);
        p.ncy = n_pos(it.H, cell, stride);
        const int nx = p.ncx - (cells_x - 1) * r, ny = p.ncy - (cells_y - 1) * r;
        p.nx = nx > 0 && ny > 0 ? nx : 0;
        p.ny = nx > 0 && ny > 0 ? ny : 0;
        p.cells_t0 = (int)cells_t;
        p.cells_tx = p.ncx > 0 ? cells_fused_tiles_x(p.ncx, stride) : 1;
        cells_t += p.ncx > 0 && p.ncy > 0 ? cells_fused_tiles(p.ncx, p.ncy, stride) : 0;
        p.score_c0 = (int)score_c;
        p.score_tx = (p.nx + wpc - 1) / wpc;
        p.score_bands = (p.ny + band_rows - 1) / band_rows;
        score_c += (long)p.score_tx * p.score_bands * classes;
        p.detect_t0 = (int)detect_t;
        detect_t += detect_tiles((long)p.nx * p.ny);
        if (cells_t > 0x7FFFFFFFL || score_c > 0x7FFFFFFFL || detect_t > 0x7FFFFFFFL) return HOG_ERR_ARG;
    }
    h->magic = kPlanMagic;
    h->n_items = n_items;
    h->channels = channels;
    h->n_bins = n_bins;
    h->cell = cell;
    h->stride = stride;
    h->cells_x = cells_x;
    h->cells_y = cells_y;
    h->r = r;
    h->cells_tiles = (int)cells_t;
    h->score_tc = Tc;
    h->score_ctas = (int)score_c;
    h->score_rows = rows ? 1 : 0;
    h->detect_tiles = (int)detect_t;
    return HOG_OK;
}

hog_status hog_cell_hist_fused_batch(const void* plan, const void* plan_dev, const uint8_t* lut, int cell_dtype,
                                     hog_stream_t stream) {
    const PlanHeader* h = checked_plan(plan);
    if (h == nullptr || !plan_dev_ok(plan_dev)) return HOG_ERR_ARG;
    if (lut == nullptr || reinterpret_cast<uintptr_t>(lut) % 16 != 0) return HOG_ERR_ARG;
    if (cell_dtype != HOG_I32 && cell_dtype != HOG_BF16 && cell_dtype != HOG_F32) return HOG_ERR_ARG;
    if (cell_dtype == HOG_BF16 && h->cell > 16) return HOG_ERR_ARG;  // counts above 256 are not exact in bf16
    const PlanItem* items = plan_items(plan);
    const size_t align = cell_dtype == HOG_BF16 ? 2 : 4;
    for (int i = 0; i < h->n_items; ++i)
        if (reinterpret_cast<uintptr_t>(items[i].it.cells) % align != 0) return HOG_ERR_ARG;
    unsigned int* status = nullptr;
    hog_status s = device_status_word(&status);
    if (s != HOG_OK) return s;
    return launch_cells_fused_batch(*h, plan_dev, lut, cell_dtype, status, reinterpret_cast<cudaStream_t>(stream));
}

hog_status hog_window_score_batch(const void* plan, const void* plan_dev, int cell_dtype, const void* w, int w_dtype,
                                  float bias, hog_stream_t stream) {
    const PlanHeader* h = checked_plan(plan);
    if (h == nullptr || !plan_dev_ok(plan_dev) || w == nullptr) return HOG_ERR_ARG;
    if (cell_dtype != HOG_I32 && cell_dtype != HOG_BF16 && cell_dtype != HOG_F32) return HOG_ERR_ARG;
    if (w_dtype != HOG_F32 && w_dtype != HOG_BF16 && w_dtype != HOG_I8) return HOG_ERR_ARG;
    if (!std::isfinite(bias)) return HOG_ERR_ARG;
    const PlanItem* items = plan_items(plan);
    if (w_dtype == HOG_I8 && 127.0 * h->cells_x * h->cells_y * (double)h->cell * h->cell +
                                     std::fabs((double)std::llround((double)bias)) >= 16777216.0)
        return HOG_ERR_UNSUPPORTED;  // int8 scores are exact only below 2^24 (as hog_window_score)
    bool tc = score_tc_supported(cell_dtype, h->n_bins, h->cells_x, h->cells_y, h->r, 0);
    for (int i = 0; i < h->n_items && tc; ++i)
        if (items[i].nx > 0 && reinterpret_cast<uintptr_t>(items[i].it.cells) % 16 != 0) tc = false;
    const cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    if (tc) {
        const float b = w_dtype == HOG_I8 ? (float)std::llround((double)bias) : bias;
        if (h->score_rows) return launch_score_rows_batch(*h, plan_dev, w, w_dtype, b, st);
        return launch_score_tc_batch(*h, plan_dev, w, w_dtype, b, st);
    }
    // other combinations: the per-image call on each item, in plan order
    for (int i = 0; i < h->n_items; ++i) {
        const PlanItem& p = items[i];
        if (p.nx == 0) continue;
        hog_status s = hog_window_score(p.it.cells, cell_dtype, p.ncx, p.ncy, h->n_bins, h->cells_x, h->cells_y,
                                        h->cell, h->stride, w, w_dtype, bias, p.it.scores, stream);
        if (s != HOG_OK) return s;
    }
    return HOG_OK;
}

size_t hog_detect_batch_workspace_bytes(const void* plan) {
    const PlanHeader* h = checked_plan(plan);
    return h == nullptr ? 0 : detect_batch_workspace_bytes(*h);
}

hog_status hog_detect_batch(const void* plan, const void* plan_dev, int score_dtype, float thr, hog_det* out,
                            int max_out, int32_t* d_count, int32_t* item_counts, void* workspace,
                            size_t workspace_bytes, hog_stream_t stream) {
    const PlanHeader* h = checked_plan(plan);
    if (h == nullptr || !plan_dev_ok(plan_dev) || d_count == nullptr || workspace == nullptr) return HOG_ERR_ARG;
    if (max_out < 0 || (out == nullptr && max_out > 0)) return HOG_ERR_ARG;
    if (reinterpret_cast<uintptr_t>(out) % alignof(hog_det) != 0) return HOG_ERR_ARG;
    if (reinterpret_cast<uintptr_t>(workspace) % 16 != 0) return HOG_ERR_ARG;
    if (score_dtype != HOG_F32 && score_dtype != HOG_I32) return HOG_ERR_ARG;
    if (std::isnan(thr)) return HOG_ERR_ARG;
    if (workspace_bytes < detect_batch_workspace_bytes(*h)) return HOG_ERR_ARG;
    return launch_detect_batch(*h, plan_dev, score_dtype, thr, out, max_out, d_count, item_counts, workspace,
                               reinterpret_cast<cudaStream_t>(stream));
}

size_t hog_pyramid_bytes(int W, int H, int channels, int levels) { return pyramid_bytes(W, H, channels, levels); }

hog_status hog_pyramid(const uint8_t* img, int W, int H, int channels, size_t pitch, int levels, uint8_t* out,
                       hog_stream_t stream) {
    if (img == nullptr || (out == nullptr && levels > 1)) return HOG_ERR_ARG;
    if (W < 1 || H < 1 || W > 65535 || H > 65535 || (channels != 1 && channels != 3)) return HOG_ERR_ARG;
    if (pitch < (size_t)W * channels || levels < 1 || levels > 16) return HOG_ERR_ARG;
    return launch_pyramid(img, W, H, channels, pitch, levels, out, reinterpret_cast<cudaStream_t>(stream));
}

}  // extern "C"
