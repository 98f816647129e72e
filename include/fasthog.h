/*
 * fasthog.h -- C ABI of the GB300 (sm_103a) fast-HOG detection library.
 *
 * The library implements the detection path of "A Fast HOG Descriptor Using
 * Lookup Table and Integral Image" (Huang & Huang): a 511 x 511 gradient
 * lookup table, a per-pixel orientation-bin map, one integral image per bin,
 * per-cell histograms from four integral-image corners, a linear score per
 * window position, and a threshold that compacts the windows into a list.
 *
 * Conventions shared by every call
 * --------------------------------
 *  - Every pointer argument is a DEVICE pointer, allocated and owned by the
 *    caller, unless its comment says otherwise.  No call allocates device or
 *    host memory, and no call synchronises the stream: work is enqueued on
 *    `stream` (NULL = the legacy default stream) and the call returns.
 *  - Images are W columns (x, to the right) by H rows (y, downwards).
 *  - Every call returns a hog_status.  Arguments are checked on the host
 *    before anything is enqueued; on any error nothing is enqueued and the
 *    outputs are left untouched.  HOG_ERR_CUDA means a launch failed; the CUDA
 *    error code is then available from hog_last_cuda_error().
 *  - Sizes are limited to 1 <= W, H <= 65535 (W * H < 2^31) and 1 <= N_b <= 64.
 *  - The library is thread-safe in the sense that calls on different streams
 *    from different host threads do not share host state, apart from the
 *    last-error slot, which is per thread.
 */
#ifndef FASTHOG_H
#define FASTHOG_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* A cudaStream_t, spelled without the CUDA headers. */
typedef struct CUstream_st* hog_stream_t;

typedef enum {
    HOG_OK = 0,
    HOG_ERR_ARG = 1,          /* null pointer, size, pitch, dtype or N_b out of range,
                                 or a workspace that is too small */
    HOG_ERR_UNSUPPORTED = 2,  /* a valid combination this build does not implement */
    HOG_ERR_CUDA = 3,         /* a CUDA call failed; see hog_last_cuda_error() */
    HOG_ERR_TIMEOUT = 4       /* a bounded device-side wait gave up (see the call) */
} hog_status;

/* Element types named by the dtype arguments. */
typedef enum {
    HOG_U8 = 0,
    HOG_I32 = 1,
    HOG_BF16 = 2,
    HOG_F32 = 3,
    HOG_I8 = 4,
    HOG_U16 = 5
} hog_dtype;

/* The value a bin map holds where a pixel has no orientation bin. */
#define HOG_NO_BIN 0xFF
/* Side of the gradient lookup table: dx and dy both range over [-255, 255]. */
#define HOG_LUT_SIDE 511
/* Row pitch of the table in memory: 511 entries and one pad byte, so that
 * every row half starts on a 16-byte boundary. */
#define HOG_LUT_PITCH 512
/* Offset of the quadrant copy that follows the table: 256 rows of 256 bytes,
 * row dy (0..255), column dx - 1 (dx = 1..256), entry = the table's entry for
 * (dx, dy) (0xFF for dx = 256).  It is a contiguous duplicate of part of the
 * table that the bin-map kernel stages into shared memory in one copy. */
#define HOG_LUT_QUAD_OFFSET (HOG_LUT_SIDE * HOG_LUT_PITCH)
/* Bytes of one table buffer: 511 rows of HOG_LUT_PITCH, then the quadrant. */
#define HOG_LUT_BYTES (HOG_LUT_QUAD_OFFSET + 256 * 256)

/* One detection: window origin (x, y) in pixels, its score, and the image
 * index and pyramid level the caller tagged the call with. */
typedef struct {
    int32_t x;
    int32_t y;
    float score;
    int32_t image;
    int32_t level;
} hog_det;

/* Human-readable name of a status. */
const char* hog_status_string(hog_status s);
/* CUDA error code (cudaError_t as int) of the last HOG_ERR_CUDA on this thread. */
int hog_last_cuda_error(void);
/* Library version, major * 10000 + minor * 100 + patch. */
int hog_version(void);

/* Device-side status of the current device: bit 0 (HOG_STATUS_TIMEOUT) is set
 * when a bounded wait inside a kernel gave up (the kernel then returned
 * without finishing its work, so its outputs are undefined).  `flags` is a
 * host pointer.  With clear != 0 the status is reset to 0.  This call
 * synchronises with the device (it copies one word), unlike every other call. */
#define HOG_STATUS_TIMEOUT 1u
hog_status hog_device_status(uint32_t* flags, int clear);

/*
 * hog_selftest_wait_timeout -- makes one of the library's bounded device-side
 * waits run out, so that the timeout path can be tested without faulting or
 * hanging the GPU.  The paper has no counterpart.
 *
 * One CTA of 32 threads waits, for at most limit_us microseconds
 * (1 .. 1,000,000), on something that nothing will ever provide:
 *   mode 0: phase 0 of a shared-memory mbarrier that no thread arrives at (the
 *           wait of the bin-map, fused-cells and tensor-core kernels), with no
 *           bulk copy or MMA in flight;
 *   mode 1: a flag in device memory that no CTA raises (the wait of the
 *           single-pass integral and detection kernels).
 * The wait gives up, the kernel sets HOG_STATUS_TIMEOUT in the device status
 * word (read it with hog_device_status) and returns; the context stays usable.
 * Other arguments: HOG_ERR_ARG.
 */
hog_status hog_selftest_wait_timeout(int mode, int limit_us, hog_stream_t stream);

/*
 * hog_build_lut -- the 511 x 511 gradient lookup table (paper Section 2).
 *
 * For every (dx, dy) in [-255, 255]^2 (the paper's "-225" is read as -255,
 * since 511 = 2 * 255 + 1) the entry at lut[(dy + 255) * 512 + (dx + 255)]
 * is the orientation bin of the gradient with unit magnitude: the angle phi
 * of (dx, dy), measured from +x towards +y (image y axis pointing down) in
 * [0, 2*pi), falls in the half-open sector [k * 2*pi/N_b, (k+1) * 2*pi/N_b)
 * and the entry is k.  (0, 0) has no angle and gets HOG_NO_BIN.
 * The bin of every entry is decided exactly (no floating-point atan2).
 *
 *   n_bins  N_b, 1..64
 *   lut     out: HOG_LUT_BYTES bytes (uint8), 16-byte aligned; row dy + 255
 *           holds the 511 entries of that dy, then one pad byte (written
 *           0xFF); the quadrant copy follows at HOG_LUT_QUAD_OFFSET
 * Built once per N_b and kept resident; hog_bin_map reads it.
 */
hog_status hog_build_lut(int n_bins, uint8_t* lut, hog_stream_t stream);

/*
 * hog_bin_map -- oriented-gradient map (paper Section 2, Eq. 1).
 *
 * For every pixel with 0 < x < W-1 and 0 < y < H-1:
 *   dx = P[x+1][y] - P[x-1][y],  dy = P[x][y+1] - P[x][y-1]
 * per channel; with 3 channels the channel with the largest dx^2 + dy^2 is
 * used (ties: the lowest channel index).  The pixel's bin is the table entry
 * of its (dx, dy).  Border pixels (where Eq. 1 would read outside the image)
 * and pixels with dx = dy = 0 get HOG_NO_BIN.
 *
 *   img          in: H rows of pitch_bytes; gray pixel img[y*pitch + x],
 *                RGB pixel img[y*pitch + 3*x + c] (interleaved, c = R, G, B)
 *   channels     1 or 3
 *   pitch_bytes  >= W * channels
 *   lut          in: the table from hog_build_lut for this n_bins
 *   bins         out: H * W bytes, row-major, pitch W
 */
hog_status hog_bin_map(const uint8_t* img, int W, int H, int channels, size_t pitch_bytes,
                       const uint8_t* lut, int n_bins, uint8_t* bins, hog_stream_t stream);

/*
 * hog_integral -- one integral image per bin (paper Section 3.2, Eq. 4-5).
 *
 *   ii[n][y][x] = #{ (x', y') : x' <= x, y' <= y, bins[y'][x'] == n }
 *
 * i.e. the inclusive 2-D prefix sum (Eq. 2) of the one-hot image of bin n
 * (Eq. 4).  HOG_NO_BIN pixels count in no plane.
 *
 *   ii_dtype   HOG_I32 (exact), or HOG_U16: every entry modulo 2^16.  Box sums
 *              of the U16 planes taken modulo 2^16 are exact for any box of
 *              fewer than 65536 pixels (the paper's 16-bit integral images,
 *              Section 4), whatever the image size.
 *   ii         out: n_bins planes of H * W entries, [n][y][x]
 *   workspace  scratch of at least hog_integral_workspace_bytes(W, H, n_bins)
 *              bytes, 256-byte aligned, ZERO-FILLED before its first use with
 *              an image size W x H (e.g. cudaMemsetAsync at allocation).  Calls
 *              with that size (any n_bins, ii_dtype or schedule) then reuse it
 *              without clearing: every call leaves it ready for the next.
 *              Zero-fill it again before a call with another W or H (the
 *              single-pass schedule keeps a tag word and one flag per tile at
 *              its start, and where the flags end depends on the size).
 *              Calls that overlap on the device must not share a workspace.
 *              (The cluster schedule, the library's choice for images up to
 *              640 rows and 8 bins, does not touch it.)
 */
size_t hog_integral_workspace_bytes(int W, int H, int n_bins);
/* Kernel launches one hog_integral call of this size enqueues under the
 * current launch-shape knobs (1 or 3 per window of up to 16 bins, 1 per
 * window of up to 8 bins on the cluster schedule); 0 for an invalid size. */
int hog_integral_launches(int W, int H, int n_bins);
hog_status hog_integral(const uint8_t* bins, int W, int H, int n_bins, int ii_dtype, void* ii,
                        void* workspace, size_t workspace_bytes, hog_stream_t stream);

/*
 * hog_cell_hist -- histogram of every cell from its four integral-image
 * corners (paper Section 3.3, Eq. 6 applying Section 3.1, Eq. 3 per bin).
 *
 * Cells are cell x cell pixels with origins (s*i, s*j), s = stride, for
 * i < ncx = (W - cell)/s + 1 and j < ncy = (H - cell)/s + 1.  With
 * x0 = s*i, y0 = s*j, x1 = x0 + cell - 1, y1 = y0 + cell - 1:
 *   cells[j][i][n] = ii_n(x1,y1) + ii_n(x0-1,y0-1) - ii_n(x1,y0-1) - ii_n(x0-1,y1)
 * where an index of -1 reads 0.  These are the area histograms the paper
 * caches so that overlapping windows reuse them.
 *
 *   ii, ii_dtype  the planes written by hog_integral (HOG_I32 or HOG_U16)
 *   cell          cell side in pixels, 1..64 (cell * cell < 65536)
 *   stride        1..cell
 *   cell_dtype    HOG_I32, HOG_F32 (counts are exact in either), or HOG_BF16
 *                 (counts <= cell^2 <= 256 are exact in bf16 for cell <= 16)
 *   cells         out: [ncy][ncx][n_bins], bin innermost
 */
hog_status hog_cell_hist(const void* ii, int W, int H, int n_bins, int ii_dtype, int cell,
                         int stride, int cell_dtype, void* cells, hog_stream_t stream);

/*
 * hog_cell_hist_fused -- the cell map of hog_cell_hist straight from the image
 * (paper Sections 2 and 3 in one kernel).
 *
 * Produces exactly hog_cell_hist(hog_integral(hog_bin_map(img))) for the
 * same arguments, without writing the bin map or the integral planes to
 * memory: each block of stride x stride pixels is binned (Eq. 1 and the
 * table) and counted, a tile-local integral image is formed at the block
 * corners (Eq. 5), and every cell is its four-corner sum (Eq. 6).  Box sums
 * are unchanged by the per-tile offset of a tile-local integral image.
 *
 *   img, W, H, channels, pitch_bytes, lut, n_bins   as for hog_bin_map
 *   cell, stride, cell_dtype, cells                 as for hog_cell_hist
 * Supported: n_bins 8 or 16, stride 4 or 8, cell a multiple of stride with
 * cell / stride <= 4; other valid arguments return HOG_ERR_UNSUPPORTED (use
 * the three separate calls).
 */
hog_status hog_cell_hist_fused(const uint8_t* img, int W, int H, int channels, size_t pitch_bytes,
                               const uint8_t* lut, int n_bins, int cell, int stride, int cell_dtype, void* cells,
                               hog_stream_t stream);

/*
 * hog_window_score -- linear objectness score of every window position
 * (paper Section 1: the cached histograms feed a score at every scan
 * position; Section 4: that score is an inner product of the window feature
 * with a weight vector).
 *
 * A window is cells_x x cells_y cells; its feature is the concatenation of its
 * cell histograms with index (cy * cells_x + cx) * n_bins + b.  With
 * r = cell / stride, the window at pixel (px*s, py*s) uses cell-map entry
 * (px + cx*r, py + cy*r) for its cell (cx, cy), so
 *   scores[py][px] = bias + sum_{cy, cx, b} w[(cy*cells_x + cx)*n_bins + b]
 *                                        * cells[py + cy*r][px + cx*r][b]
 * for px < nx = ncx - (cells_x - 1) r and py < ny = ncy - (cells_y - 1) r.
 *
 *   cells, cell_dtype  from hog_cell_hist (HOG_I32, HOG_F32 or HOG_BF16;
 *                      16-byte aligned for the fast kernels)
 *   cell, stride       as given to hog_cell_hist; stride must divide cell
 *   w, w_dtype         cells_x * cells_y * n_bins weights:
 *                      HOG_F32  -> FP32 arithmetic on CUDA cores, scores f32
 *                      HOG_BF16 -> bf16 x bf16 -> f32, scores f32
 *                      HOG_I8   -> exact; scores int32 (the bias is rounded to
 *                                  the nearest integer).  Exactness needs every
 *                                  partial sum below 2^24, which holds for cells of
 *                                  hard-vote counts (at most cell^2 per cell over
 *                                  its bins) when 127 * cells_x * cells_y * cell^2
 *                                  + |round(bias)| < 2^24; otherwise the call
 *                                  returns HOG_ERR_UNSUPPORTED (e.g. cell = 64
 *                                  with an 8 x 16-cell window)
 *                      All three run on the tensor cores (tcgen05) for
 *                      16-byte-aligned HOG_BF16 cells, n_bins 8 or 16, an
 *                      8 x 16-cell window and r = 1, 2 or 4 (f32 weights as
 *                      three exact bf16 parts accumulated in f32, so the
 *                      products are the f32 products); otherwise on CUDA
 *                      cores with the same accuracy
 *   scores             out: [ny][nx], f32 (F32/BF16 weights) or int32 (I8)
 */
hog_status hog_window_score(const void* cells, int cell_dtype, int ncx, int ncy, int n_bins,
                            int cells_x, int cells_y, int cell, int stride, const void* w,
                            int w_dtype, float bias, void* scores, hog_stream_t stream);

/*
 * Soft votes -- the two-bin vote that Section 2 mentions (OpenCV spreads each
 * pixel over two bins) and the paper sets aside for single-bin unit votes.
 * Each pixel with a gradient (unit magnitude) splits HOG_SOFT_Q vote units
 * between the two bins whose centres c_k = (k + 1/2) 2 pi / N_b flank its
 * angle phi, linearly in angle: with t = phi N_b / (2 pi) - 1/2,
 * k0 = floor(t) mod N_b and alpha = t - floor(t), bin k0 gets q - a and bin
 * k0 + 1 (mod N_b) gets a = round(q alpha).  Integral images and Eq. 6 still
 * apply: they sum vote units instead of counts, exactly.
 *
 * hog_build_soft_lut -- the soft table: 511 rows (dy + 255) of HOG_LUT_PITCH
 *   uint16 entries (dx + 255), entry = k0 | a << 8 (an angle on a bin centre
 *   is (k, 0)), 0xFFFF at (0, 0) and in the pad column.  FP64, fixed
 *   operation order; n_bins 1..64; lut 4-byte aligned, HOG_SOFT_LUT_BYTES.
 * hog_cell_hist_soft -- the cell histograms of the soft votes straight from
 *   the image, in one kernel (as hog_cell_hist_fused): cells[j][i][b] = the
 *   vote units of bin b from the cell's pixels.  n_bins 2..16, stride 4 or 8,
 *   cell = r * stride with r <= 4; cell_dtype HOG_I32 or HOG_F32 (a cell
 *   holds up to cell^2 * HOG_SOFT_Q units).
 */
#define HOG_SOFT_Q 64
#define HOG_SOFT_LUT_BYTES (HOG_LUT_SIDE * HOG_LUT_PITCH * 2)
hog_status hog_build_soft_lut(int n_bins, uint16_t* lut, hog_stream_t stream);
hog_status hog_cell_hist_soft(const uint8_t* img, int W, int H, int channels, size_t pitch_bytes,
                              const uint16_t* soft_lut, int n_bins, int cell, int stride, int cell_dtype,
                              void* cells, hog_stream_t stream);

/*
 * hog_block_norm -- overlapping blocks of 2 x 2 cells, L2-normalised.
 *
 * The paper forms a region's feature from the histograms of four overlapped
 * sub-areas (Section 3, Fig. 4's caption; the figure is missing).  Read here
 * as the classic layout: a block is 2 x 2 cells, blocks step by one cell,
 * and each block's 4 n_bins counts are divided by sqrt(sum of squares +
 * eps^2).  Block (i, j) of the map holds cells (i + cx r, j + cy r) of the
 * cell map, r = cell / stride, in quadrant order q = 2 cy + cx:
 *   blocks[j][i][q * n_bins + b] = cells[j + cy r][i + cx r][b] / norm(i, j)
 * (0 for a block with no binned pixel and eps = 0).
 *
 *   cells, cell_dtype  [ncy][ncx][n_bins] of HOG_I32, HOG_F32 or HOG_BF16
 *   r                  block step in cell-map positions (cell / stride), >= 1
 *   eps                >= 0
 *   blocks             out: float [ncy - r][ncx - r][4 * n_bins]
 *
 * Score the block map with hog_window_score as a map with 4 * n_bins values
 * per entry and a window of 7 x 15 blocks (64 x 128 pixels), with the same
 * cell and stride: ncx, ncy of that call are ncx - r, ncy - r.
 */
hog_status hog_block_norm(const void* cells, int cell_dtype, int ncx, int ncy, int n_bins, int r, float eps,
                          float* blocks, hog_stream_t stream);

/*
 * hog_window_score_multi -- several linear filters over the same windows:
 *   scores[f][py][px] = biases[f] + sum_k w[f][k] * feature_k(px, py),
 * each filter exactly as hog_window_score would score it alone.  The paper
 * scores one filter; several filters (one detector per class or pose) share
 * every cell row the kernel loads, and on the tensor cores they widen the
 * contraction (one MMA per filter per step into its own accumulator block).
 *
 *   w        device [n_filters][cells_y * cells_x * n_bins] of w_dtype
 *   biases   HOST array of n_filters floats, read during the call (rounded to
 *            the nearest integer, halves away from zero, for HOG_I8 weights)
 *   scores   device [n_filters][ny][nx], f32 (int32 for HOG_I8 weights)
 *   n_filters 1..1024; everything else as in hog_window_score.
 */
hog_status hog_window_score_multi(const void* cells, int cell_dtype, int ncx, int ncy, int n_bins, int cells_x,
                                  int cells_y, int cell, int stride, const void* w, int w_dtype, int n_filters,
                                  const float* biases, void* scores, hog_stream_t stream);

/*
 * hog_detect -- threshold and ordered compaction of the score map.
 *
 * Every window with score >= thr is written to out[] in row-major (py, px)
 * order as { x = px*stride, y = py*stride, score, image, level }.  The total
 * number of such windows is written to *d_count (device int32), even when it
 * exceeds max_out; only the first max_out entries are written.
 *
 *   scores, score_dtype  [ny][nx] of HOG_F32 or HOG_I32
 *   image, level         copied into every detection (caller's tags)
 *   out, d_count         device memory, or page-locked host memory mapped into
 *                        the device's address space (the list is written with
 *                        plain coalesced stores, no atomics); out 4-byte aligned
 *   workspace            at least hog_detect_workspace_bytes(nx, ny) bytes of
 *                        scratch, 8-byte aligned, ZERO-FILLED before its first
 *                        use (e.g. cudaMemsetAsync once at allocation); every
 *                        call leaves it ready for the next, so it is never
 *                        cleared again.  The single launch's tiles publish
 *                        their counts in it (a tag word of the last call and one
 *                        status word per 2048 scores).  Calls that overlap on
 *                        the device must not share a workspace.
 */
size_t hog_detect_workspace_bytes(int nx, int ny);
hog_status hog_detect(const void* scores, int score_dtype, int nx, int ny, int stride, float thr,
                      int image, int level, hog_det* out, int max_out, int32_t* d_count,
                      void* workspace, size_t workspace_bytes, hog_stream_t stream);

/*
 * hog_detect_noalloc -- hog_detect without a caller-provided workspace.
 *
 * The paper has no counterpart: this entry point exists for callers that
 * cannot allocate device memory for scratch -- for example a plugin that is
 * handed only its input and output buffers by a host application that owns
 * all device memory, or a latency-critical loop that must not call
 * cudaMalloc.  It computes exactly what hog_detect computes (same arguments
 * minus the workspace) and allocates nothing.
 *
 * Its scratch is a fixed array of 128 KiB + 64 bytes inside the library's
 * device memory, which every GPU that loads the library holds until the
 * process exits.  It is zero-filled when the library is loaded and every
 * call leaves it ready for the next: nothing has to be cleared.
 * Limits and rules:
 *  - nx * ny <= HOG_DETECT_NOALLOC_MAX_SCORES, otherwise HOG_ERR_ARG and
 *    nothing is enqueued;
 *  - the first call on a device looks up the array's device address (a
 *    host-side step, done once per device with that device current); make
 *    that first call before capturing a stream into a graph;
 *  - all calls share the array: calls whose work overlaps on the GPU (on
 *    different streams, or from different host threads without ordering)
 *    race and may return wrong lists.  Serialise them on one stream.
 */
#define HOG_DETECT_NOALLOC_MAX_SCORES (16384 * 2048)
hog_status hog_detect_noalloc(const void* scores, int score_dtype, int nx, int ny, int stride, float thr,
                              int image, int level, hog_det* out, int max_out, int32_t* d_count,
                              hog_stream_t stream);

/*
 * Launch-shape knobs, read by the launches made after they are set (a CUDA
 * graph keeps the shapes it was captured with).  They pick tile shapes,
 * schedules, grid sizes and engines only: integer results (bins, integral
 * images, cells, int8 scores, lists from integer scores) never change;
 * HOG_TUNE_SCORE_PATH changes the order of the f32 additions of float scores
 * (both engines stay within the FP32 bound of hog_window_score), every other
 * knob leaves float scores bit-identical.  0 restores the library's choice.  Process-wide; set them from one thread while no
 * other thread is launching.  The paper has no counterpart: they exist for
 * the autotuner (paper_1703_06256_gb300/autotune.py).
 *
 *   HOG_TUNE_INTEGRAL_BAND_ROWS   rows per tile of the integral-image scan:
 *                                 4, 8, 16 or 32 (hog_integral_workspace_bytes
 *                                 covers every choice); on the single pass 32
 *                                 picks tiles of 32 rows, any other value 16
 *   HOG_TUNE_INTEGRAL_PATH        the integral images' schedule: 1 = three
 *                                 launches (tile reduce, carries, tile scan),
 *                                 2 = one single-pass launch (each tile sums the
 *                                 aggregates of the tiles above and to its left),
 *                                 3 = one launch of thread-block clusters, one
 *                                 cluster of up to 16 CTAs per 128 columns
 *                                 (images up to 1280 rows and 8192 columns;
 *                                 taller or wider ones take three launches).
 *                                 The library's choice: 3 for images up to 640
 *                                 rows with at most 8 bins whose clusters all
 *                                 fit the GPU at once, else 1
 *   HOG_TUNE_INTEGRAL_WARP_ROWS   rows per warp of the cluster schedule: 2, 4
 *                                 or 8 (2 and 4 cover up to 640 rows, 8 up to
 *                                 1280; the library's choice is 2 where every
 *                                 cluster fits the GPU at once, else 4)
 *   HOG_TUNE_BINMAP_CTAS_PER_SM   bin-map grid cap, CTAs per SM: 1..8 (the
 *                                 grid-stride schedule)
 *   HOG_TUNE_BINMAP_SCHEDULE      the bin map's schedule: 1 = a persistent grid
 *                                 striding over quads of 4 pixels, each thread
 *                                 loading its words straight from global memory;
 *                                 2 = one CTA per tile of 128 pixels x 16 rows,
 *                                 the tile's rows (and one above and below)
 *                                 staged in shared memory by 16-byte copies
 *                                 (images whose base address and pitch are
 *                                 multiples of 16, read through the whole table;
 *                                 others take 1).  The library's choice: 2 where
 *                                 it applies and every tile's CTA is resident at
 *                                 once, else 1
 *   HOG_TUNE_FUSED_CTAS_PER_SM    fused-cells grid cap, CTAs per SM: 1 or 2
 *   HOG_TUNE_FUSED_TILE_ROWS      cell rows per tile of hog_cell_hist_fused and
 *                                 hog_cell_hist_soft: 16, 8 or 4 (the library's
 *                                 choice: 8 where tiles of 16 rows would leave
 *                                 SMs without a tile, else 16;
 *                                 hog_cell_hist_soft takes 8 for 4; the batch
 *                                 call keeps 16)
 *   HOG_TUNE_SCORE_TC_ROWS        output rows per tensor-core CTA: 1, 2, 4, 8, 16,
 *                                 32 or 64 for the row-GEMM kernel (8 bins); the
 *                                 banded kernel (16 bins) takes 16 or 32 and its
 *                                 own choice for the other values
 *   HOG_TUNE_CELL_ROWS            cell rows per CTA of the cell-histogram kernel
 *                                 that stages the integral-image samples in
 *                                 shared memory: 4, 8 or 16; 1 = one thread per
 *                                 cell reading its corners directly
 *   HOG_TUNE_SCORE_PATH           the single-image score's engine where more than
 *                                 one applies: 1 = CUDA cores, 2 = tensor cores
 *                                 (8 bins: the row-GEMM kernel, one CTA per block
 *                                 of windows), 3 = tensor cores with each filter's
 *                                 16 rows split over a cluster of 4 CTAs (8 bins;
 *                                 the partial sums meet in shared memory); the
 *                                 library's choice for bf16 cells of 8 bins is 3
 *                                 for maps of at most about 8 x 128 x (number of
 *                                 SMs) window rows x columns, else 2; for other
 *                                 cells the banded tensor-core kernel for bf16
 *                                 and int8 weights, and for f32 weights only
 *                                 when its grid alone gives every SM a CTA
 *   HOG_TUNE_SLIDE_WINDOWS        windows per sequence of the CUDA-core score
 *                                 (8 or 16): fewer gives more CTAs, more shares
 *                                 each staged cell row among more windows
 *   HOG_TUNE_TABLE                where the bin-map and fused-cells kernels read
 *                                 the gradient table: 1 = a quadrant staged in
 *                                 shared memory (N_b a multiple of 4), 2 = the
 *                                 whole table through the read-only cache; the
 *                                 library's choice is 2 for both (measured on
 *                                 natural-image gradients, which cluster in the
 *                                 table)
 *
 * hog_tune_set returns HOG_ERR_ARG for an unknown knob or a value outside its
 * range (nothing changes); hog_tune_get returns the current value (0 = the
 * library's choice), or -1 for an unknown knob.
 */
typedef enum {
    HOG_TUNE_INTEGRAL_BAND_ROWS = 0,
    HOG_TUNE_BINMAP_CTAS_PER_SM = 1,
    HOG_TUNE_FUSED_CTAS_PER_SM = 2,
    HOG_TUNE_SCORE_TC_ROWS = 3,
    HOG_TUNE_TABLE = 4,
    HOG_TUNE_CELL_ROWS = 5,
    HOG_TUNE_SCORE_PATH = 6,
    HOG_TUNE_SLIDE_WINDOWS = 7,
    HOG_TUNE_INTEGRAL_PATH = 8,
    HOG_TUNE_INTEGRAL_WARP_ROWS = 9,
    HOG_TUNE_BINMAP_SCHEDULE = 10,
    HOG_TUNE_FUSED_TILE_ROWS = 11,
    HOG_TUNE_KNOBS = 12
} hog_tune_knob;
hog_status hog_tune_set(int knob, int value);
int hog_tune_get(int knob);

#ifdef __cplusplus
}
#endif

#endif /* FASTHOG_H */
