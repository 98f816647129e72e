/*
 * fasthog_batch.h -- the detection path over a batch of images and pyramid
 * levels of uneven sizes, one launch per stage.
 *
 * The paper runs its detector on one image at a time (Section 4) and has no
 * batching or image pyramid; both are additions of this library.  The batch
 * calls run the per-image steps of fasthog.h --
 * hog_cell_hist_fused (bin map, integral images and Eq. 6 cell histograms in
 * one kernel), hog_window_score and hog_detect -- for every item of a batch
 * in one persistent launch per stage, so that small images and small
 * pyramid levels share the GPU instead of each paying for a launch and a
 * partly empty wave.  Each item's results are identical to those of the
 * per-image calls on that item.
 *
 * A batch is described once by a plan.  hog_batch_plan (host only, no CUDA
 * call) writes the items and, for each stage, where its tiles of each item
 * start, into a caller-provided host buffer.  The caller copies those bytes
 * unchanged into device memory (any copy) and passes both copies to the
 * stage calls: the host copy sizes the launches, the device copy is read by
 * the kernels.  A plan stays valid as long as the items' buffers do, so a
 * fixed batch layout is planned once and its stage calls can be captured
 * into a CUDA graph and replayed.
 *
 * Conventions of fasthog.h hold: device pointers owned by the caller, no
 * allocation, no synchronisation, arguments checked before anything is
 * enqueued.
 */
#ifndef FASTHOG_BATCH_H
#define FASTHOG_BATCH_H

#include "fasthog.h"

#ifdef __cplusplus
extern "C" {
#endif

typedef struct {
    const uint8_t* img; /* device: H rows of W * channels bytes, `pitch` bytes apart */
    size_t pitch;
    int W, H;           /* 1..65535 each */
    void* cells;        /* device: [ncy][ncx][N_b] of the batch's cell dtype */
    void* scores;       /* device: [ny][nx], float (int32 for HOG_I8 weights) */
    int image, level;   /* copied into every detection of this item */
} hog_batch_item;

/* Bytes of the plan of an n-item batch (n >= 1; 0 for n < 1). */
size_t hog_batch_plan_bytes(int n_items);

/* Lay out the plan of a batch in host memory `plan` (plan_bytes >=
 * hog_batch_plan_bytes(n_items)).  All items share channels (1 or 3), N_b
 * (8 or 16), the cell side and stride (stride 4 or 8, cell = r * stride,
 * r <= 4) and the window of cells_x x cells_y cells.  Items smaller than a
 * window have no scores and no detections.  At most 65536 items. */
hog_status hog_batch_plan(const hog_batch_item* items, int n_items, int channels, int n_bins, int cell,
                          int stride, int cells_x, int cells_y, void* plan, size_t plan_bytes);

/* hog_cell_hist_fused on every item: cell_dtype HOG_I32, HOG_F32 or HOG_BF16
 * (cell <= 16).  `lut` is the table of hog_build_lut for the plan's N_b. */
hog_status hog_cell_hist_fused_batch(const void* plan, const void* plan_dev, const uint8_t* lut, int cell_dtype,
                                     hog_stream_t stream);

/* hog_window_score on every item's cell map.  Weights as in
 * hog_window_score.  With bf16 cells and bf16 or int8 weights (N_b = 8,
 * window 8 x 16 cells, r = 1, 2 or 4) it is one tensor-core launch over the
 * batch; otherwise the per-image kernel runs once per item. */
hog_status hog_window_score_batch(const void* plan, const void* plan_dev, int cell_dtype, const void* w, int w_dtype,
                                  float bias, hog_stream_t stream);

/* Scratch of hog_detect_batch for this plan. */
size_t hog_detect_batch_workspace_bytes(const void* plan);

/* Threshold and compact every item's scores into ONE list: items in plan
 * order, each item's windows in row-major order, each tagged with the item's
 * image and level.  *d_count (device int32) receives the total;
 * item_counts (device int32[n_items], may be NULL) each item's count.  The
 * list is truncated at max_out, the counts are not.  `out` may be device
 * memory or page-locked host memory mapped into the device's address space. */
hog_status hog_detect_batch(const void* plan, const void* plan_dev, int score_dtype, float thr, hog_det* out,
                            int max_out, int32_t* d_count, int32_t* item_counts, void* workspace,
                            size_t workspace_bytes, hog_stream_t stream);

/* Pyramid levels 1 .. levels-1 of an image by 2:1 decimation: level l is
 * (W >> l) x (H >> l), and its pixel (x, y) is pixel (x << l, y << l) of the
 * image (level l+1 keeps the even rows and columns of level l).  They are
 * written one after the other into `out`, rows contiguous (pitch W_l *
 * channels); hog_pyramid_bytes gives the total.  Plain decimation, no
 * smoothing: every level is exact integer data. */
size_t hog_pyramid_bytes(int W, int H, int channels, int levels);
hog_status hog_pyramid(const uint8_t* img, int W, int H, int channels, size_t pitch, int levels, uint8_t* out,
                       hog_stream_t stream);

#ifdef __cplusplus
}
#endif

#endif /* FASTHOG_BATCH_H */
