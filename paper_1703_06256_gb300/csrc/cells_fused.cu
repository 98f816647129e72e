// cells_fused.cu -- image -> cell histograms in one kernel: the bin map
// (Section 2), integral images (Section 3.2, Eq. 4-5) and four-corner cell
// histograms (Section 3.3, Eq. 6) without sending the bin map or the integral
// planes to HBM.
//
// Cells are cell x cell pixels at stride s, cell = r s.  Cut the image into
// blocks of s x s pixels; block (I, J) covers x in [s I, s I + s), y in
// [s J, s J + s), and the cell with origin (s i, s j) is exactly the blocks
// [i, i + r) x [j, j + r).  The integral image sampled at the block corners,
//   G_b(I, J) = ii_b(s I - 1, s J - 1)   (0 for I = 0 or J = 0),
// is all Eq. 6 needs: cell (i, j) = G(i+r, j+r) - G(i, j+r) - G(i+r, j) + G(i, j).
// Box sums do not change when every ii value of a tile is offset by the
// same amount, so each CTA builds G from its own tile only ("tile-local"
// integral image), as a 2-D prefix sum of its block histograms.
//
// Per tile of BX x BY cells (origins), a CTA of 512 threads
//   1. computes the bins of the tile's (BX + r - 1) x (BY + r - 1) blocks with
//      the same quad code and table lookup as the bin-map kernel (the whole
//      table through the read-only cache, or on request a quadrant staged in
//      shared memory), one quad (4 pixels of a row) per task, and adds them into
//      per-block counters (8-bit fields, s^2 <= 64 for s = 4, 8) with
//      shared-memory atomics;
//   2. forms G over those blocks in shared memory (16-bit fields): warp
//      scans along block rows, then running sums down the columns;
//   3. writes each cell's histogram from four corners of G (16-byte stores).
// Tiles overlap by r - 1 blocks, whose bins are computed twice.  The grid is
// persistent, so a staged table quadrant is copied once per CTA.
#include <type_traits>

#include "batch_plan.cuh"
#include "bin_core.cuh"
#include "internal.cuh"
#include "ptx.cuh"

namespace fasthog {

namespace {

constexpr int kThreads = 512;
constexpr int kQuadBytes = 256 * 256;
constexpr int kMaxR = 4;

// Tile of BX x BY cell origins per CTA.  Its blocks span (BX + r - 1) s by
// (BY + r - 1) s pixels, at most 140 x 76 (s = 4) or 152 x 152 (s = 8) for
// r <= 4: below 2^15 pixels, so every corner value of the tile-local integral
// image fits a 16-bit field with a spare bit, and (a + d) - (b + c) of Eq. 6
// never carries or borrows between fields.
template <int S>
struct TileShape {
    static constexpr int BX = S == 4 ? 32 : 16;
    static constexpr int BY = 16;
};

template <int NB, int S>
struct FusedSmem {
    static constexpr int NW8 = NB / 4;                      // 8-bit-field words per block histogram
    static constexpr int NW16 = NB / 2;                     // 16-bit-field words per G entry
    static constexpr int BXB = TileShape<S>::BX + kMaxR - 1;  // blocks per tile row (max)
    static constexpr int BYB = TileShape<S>::BY + kMaxR - 1;
    uint32_t g[BYB + 1][BXB + 1][NW16];                     // corner-sampled tile integral image
    uint32_t bh[BYB][BXB][NW8];                             // block histograms
};

template <typename OutT>
__device__ __forceinline__ OutT as_count(uint32_t v) {
    if constexpr (std::is_same<OutT, uint16_t>::value) {
        return f32_to_bf16_exact_int((float)v);
    } else {
        return (OutT)v;
    }
}

// A count as the 32-bit pattern of a 4-byte OutT (float or int32).
template <typename OutT>
__device__ __forceinline__ uint32_t out_bits(uint32_t v) {
    if constexpr (std::is_same<OutT, float>::value) {
        return __float_as_uint((float)v);
    } else {
        return v;
    }
}

// 1 << n, or 0 when n >= 32 as an unsigned number (PTX clamps the shift amount).
__device__ __forceinline__ uint32_t one_or_zero_shl(uint32_t n) {
    uint32_t r;
    asm("shl.b32 %0, %1, %2;" : "=r"(r) : "r"(1u), "r"(n));
    return r;
}

// The 4 nibbles of the 16-bit half h of x, one per byte.
__device__ __forceinline__ uint32_t nibbles_to_bytes(uint32_t x, int h) {
    uint32_t a = (x >> (16 * h)) & 0xFFFFu;
    a = (a | (a << 8)) & 0x00FF00FFu;
    return (a | (a << 4)) & 0x0F0F0F0Fu;
}

// Stage the shared-memory quadrant of the table (one bulk copy, bounded wait).
__device__ __forceinline__ bool stage_lut(uint8_t* lutq, const uint8_t* __restrict__ lut, uint64_t* bar,
                                          unsigned int* status) {
    const int tid = threadIdx.x;
    if (tid == 0) {
        ptx::mbar_init(bar, 1);
        ptx::fence_mbar_init();
    }
    __syncthreads();
    if (tid == 0) {
        ptx::mbar_arrive_expect_tx(bar, kQuadBytes);
        ptx::bulk_g2s(lutq, lut + kLutQuadOffset, kQuadBytes, bar);
    }
    pdl_wait();
    pdl_trigger();
    const bool ok = ptx::mbar_wait_bounded(bar, 0, kWaitLimitNs);
    if (!ok && tid == 0) atomicOr(status, kStatusTimeout);
    return ok;
}

// One tile of cell origins [bx0, bx0 + BX) x [by0, by0 + BY) of one image:
// steps 1-3 above.  Called by every thread of the CTA.
template <int CH, int NB, int S, typename OutT, bool QUAD, int BYT>
__device__ __forceinline__ void fused_tile(FusedSmem<NB, S>& sm, const uint8_t* lutq, const uint8_t* __restrict__ lut,
                                           const uint8_t* __restrict__ img, int W, int H, size_t pitch, bool aligned,
                                           int r, int ncx, int ncy, OutT* __restrict__ cells, int out_align, int bx0,
                                           int by0) {
    using F = FusedSmem<NB, S>;
    static_assert(BYT <= TileShape<S>::BY, "the shared-memory layout holds tiles of at most TileShape rows");
    constexpr int BX = TileShape<S>::BX, BY = BYT;
    constexpr int QPR = S / 4;  // quads in one block row
    const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
    const int bxn = BX + r - 1, byn = BY + r - 1;  // blocks of a tile
    const long row_bytes = (long)W * CH;
    const int row_tasks = bxn * QPR;               // quads in one pixel row of the tile
    const int n_tasks = byn * S * row_tasks;
    __syncthreads();  // the previous tile's reads of g and bh are done
    for (int k = tid; k < byn * F::BXB * F::NW8; k += kThreads) (&sm.bh[0][0][0])[k] = 0;
    __syncthreads();
    // 1. block histograms: one quad (4 pixels of one row) per task; the
    //    8-bit fields of a block's words collect at most s^2 <= 64 pixels.
    //    A thread's task position (pixel row, quad) steps by kThreads tasks
    //    without a division.
    const int step_rows = kThreads / row_tasks, step_cols = kThreads - step_rows * row_tasks;
    int prow = tid / row_tasks, qc = tid - prow * row_tasks;
    for (int task = tid; task < n_tasks; task += kThreads) {
        const int y = by0 * S + prow, x = bx0 * S + 4 * qc;
        if (y > 0 && y < H - 1 && x < W) {  // else a border row, or outside the image: no bins
            QuadWords<CH> q;
            load_quad<CH>(img, pitch, row_bytes, aligned, x, y, q);
            const uint32_t packed = bins_of_quad<CH, QUAD>(q, x, W, lutq, lut, NB, NB / 4);
            // the quad's one-hot votes in 4-bit fields, bins 8k .. 8k + 7 in word k (at most 4 per
            // field; 0xFF shifts out), then spread to the 8-bit fields of the block histogram
            uint32_t h4[NB / 8];
#pragma unroll
            for (int k = 0; k < NB / 8; ++k) h4[k] = 0;
#pragma unroll
            for (int p = 0; p < 4; ++p) {
                const uint32_t v = __byte_perm(packed, 0u, 0x4440u | (uint32_t)p);
#pragma unroll
                for (int k = 0; k < NB / 8; ++k) h4[k] += one_or_zero_shl(4u * (v - 8u * (uint32_t)k));
            }
            uint32_t* dst = sm.bh[prow / S][qc / QPR];
#pragma unroll
            for (int k = 0; k < NB / 8; ++k) {
                const uint32_t lo = nibbles_to_bytes(h4[k], 0), hi = nibbles_to_bytes(h4[k], 1);
                if (lo) atomicAdd(dst + 2 * k, lo);
                if (hi) atomicAdd(dst + 2 * k + 1, hi);
            }
        }
        prow += step_rows;
        qc += step_cols;
        if (qc >= row_tasks) {
            qc -= row_tasks;
            ++prow;
        }
    }
    __syncthreads();
    // 2. G: exclusive 2-D prefix of the block histograms in 16-bit fields
    //    (bins 2e, 2e+1 in word e).  Along block rows with warp scans (G row
    //    J + 1 holds block row J), then down the columns.
    for (int task = wid; task < byn * F::NW16; task += kThreads / 32) {
        const int J = 1 + task / F::NW16, e = task % F::NW16;
        uint32_t carry = 0;
        for (int I0 = 0; I0 < bxn; I0 += 32) {
            const int I = I0 + lane;
            uint32_t v = 0;
            if (I < bxn) {
                const uint32_t w8 = sm.bh[J - 1][I][e >> 1];
                const uint32_t two = (e & 1) ? (w8 >> 16) : (w8 & 0xFFFFu);  // bins 2e, 2e+1 (8-bit each)
                v = (two & 0xFFu) | ((two >> 8) << 16);
            }
#pragma unroll
            for (int d = 1; d < 32; d <<= 1) {
                const uint32_t u = __shfl_up_sync(0xffffffffu, v, d);
                if (lane >= d) v += u;
            }
            if (I < bxn) sm.g[J][I + 1][e] = v + carry;
            carry += __shfl_sync(0xffffffffu, v, 31);
        }
        if (lane == 0) sm.g[J][0][e] = 0;
    }
    for (int k = tid; k < (bxn + 1) * F::NW16; k += kThreads) sm.g[0][k / F::NW16][k % F::NW16] = 0;
    __syncthreads();
    for (int task = tid; task < (bxn + 1) * F::NW16; task += kThreads) {
        const int I = task / F::NW16, e = task % F::NW16;
        uint32_t v[F::BYB];  // the column's values, all loads in flight before the running sum
#pragma unroll
        for (int J = 0; J < F::BYB; ++J) v[J] = J < byn ? sm.g[J + 1][I][e] : 0u;
        uint32_t run = 0;
#pragma unroll
        for (int J = 0; J < F::BYB; ++J)
            if (J < byn) {
                run += v[J];
                sm.g[J + 1][I][e] = run;
            }
    }
    __syncthreads();
    // 3. cells: Eq. 6 on the corner-sampled integral image
    if (tid < BX * BY) {
        const int ci = tid % BX, cj = tid / BX;
        const int i = bx0 + ci, j = by0 + cj;
        if (i < ncx && j < ncy) {
            // the cell's NB counts as OutT, packed into 32-bit words (bf16: two per word)
            constexpr int NWORDS = NB * (int)sizeof(OutT) / 4;
            uint32_t words[NWORDS];
#pragma unroll
            for (int e = 0; e < F::NW16; ++e) {
                // (a + d) - (b + c) per 16-bit field: no field carries or borrows
                const uint32_t v = (sm.g[cj + r][ci + r][e] + sm.g[cj][ci][e]) -
                                   (sm.g[cj][ci + r][e] + sm.g[cj + r][ci][e]);
                if constexpr (sizeof(OutT) == 2) {
                    words[e] = (uint32_t)as_count<OutT>(v & 0xFFFFu) | ((uint32_t)as_count<OutT>(v >> 16) << 16);
                } else {
                    words[2 * e] = out_bits<OutT>(v & 0xFFFFu);
                    words[2 * e + 1] = out_bits<OutT>(v >> 16);
                }
            }
            OutT* out = cells + ((size_t)j * ncx + i) * NB;
            if (out_align == 16) {
#pragma unroll
                for (int k = 0; k < NWORDS / 4; ++k)
                    reinterpret_cast<uint4*>(out)[k] =
                        make_uint4(words[4 * k], words[4 * k + 1], words[4 * k + 2], words[4 * k + 3]);
            } else if (out_align == 4) {
#pragma unroll
                for (int k = 0; k < NWORDS; ++k) reinterpret_cast<uint32_t*>(out)[k] = words[k];
            } else {  // a 2-byte-aligned bf16 map
#pragma unroll
                for (int k = 0; k < 2 * NWORDS; ++k)
                    reinterpret_cast<uint16_t*>(out)[k] = (uint16_t)(words[k >> 1] >> (16 * (k & 1)));
            }
        }
    }
}

// Output alignment class of a cell map: every cell starts a multiple of 16
// bytes after the map's start.
__host__ __device__ inline int cells_alignment(const void* cells) {
    const uintptr_t c = reinterpret_cast<uintptr_t>(cells);
    return c % 16 == 0 ? 16 : (c % 4 == 0 ? 4 : 2);
}

// The table: QUAD = true stages its quadrant in shared memory (one bulk
// copy per CTA, quarter-turn lookups); QUAD = false reads the whole table
// through the read-only cache (after an L2 prefetch of one slice per CTA)
// and leaves the shared memory to the tile.
template <bool QUAD, int NB, int S>
__device__ __forceinline__ FusedSmem<NB, S>* fused_prologue(uint8_t* smem, const uint8_t* lut, uint64_t* bar,
                                                            unsigned int* status) {
    if constexpr (QUAD) {
        if (!stage_lut(smem, lut, bar, status)) return nullptr;
        return reinterpret_cast<FusedSmem<NB, S>*>(smem + kQuadBytes);
    } else {
        prefetch_table_l2(lut);
        pdl_wait();
        pdl_trigger();
        return reinterpret_cast<FusedSmem<NB, S>*>(smem);
    }
}

template <int CH, int NB, int S, typename OutT, bool QUAD, int BYT>
__global__ void __launch_bounds__(kThreads, 2)
    cells_fused_kernel(const uint8_t* __restrict__ img, int W, int H, size_t pitch, bool aligned,
                       const uint8_t* __restrict__ lut, int r, int ncx, int ncy, OutT* __restrict__ cells,
                       int out_align, unsigned int* status) {
    extern __shared__ __align__(128) uint8_t smem[];
    __shared__ __align__(8) uint64_t lut_bar;
    FusedSmem<NB, S>* sm = fused_prologue<QUAD, NB, S>(smem, lut, &lut_bar, status);
    if (sm == nullptr) return;
    constexpr int BX = TileShape<S>::BX, BY = BYT;
    const int tiles_x = (ncx + BX - 1) / BX, tiles_y = (ncy + BY - 1) / BY;
    for (int t = blockIdx.x; t < tiles_x * tiles_y; t += gridDim.x)
        fused_tile<CH, NB, S, OutT, QUAD, BYT>(*sm, smem, lut, img, W, H, pitch, aligned, r, ncx, ncy, cells,
                                               out_align, (t % tiles_x) * BX, (t / tiles_x) * BY);
}

// The same over every item of a batch plan: the persistent CTAs walk the
// batch's tiles, item by item.
template <int CH, int NB, int S, typename OutT, bool QUAD>
__global__ void __launch_bounds__(kThreads, 2)
    cells_fused_batch_kernel(const PlanItem* __restrict__ items, int n_items, int total_tiles,
                             const uint8_t* __restrict__ lut, int r, unsigned int* status) {
    extern __shared__ __align__(128) uint8_t smem[];
    __shared__ __align__(8) uint64_t lut_bar;
    FusedSmem<NB, S>* sm = fused_prologue<QUAD, NB, S>(smem, lut, &lut_bar, status);
    if (sm == nullptr) return;
    constexpr int BX = TileShape<S>::BX, BY = TileShape<S>::BY;
    for (int t = blockIdx.x; t < total_tiles; t += gridDim.x) {
        const PlanItem* it = items + find_item<Stage::kCells>(items, n_items, t);
        const hog_batch_item item = it->it;
        const int local = t - it->cells_t0, tx = it->cells_tx;
        const uint8_t* img = item.img;
        OutT* cells = static_cast<OutT*>(item.cells);
        const bool aligned = (reinterpret_cast<uintptr_t>(img) % 4 == 0) && (item.pitch % 4 == 0);
        fused_tile<CH, NB, S, OutT, QUAD, BY>(*sm, smem, lut, img, item.W, item.H, item.pitch, aligned, r, it->ncx,
                                              it->ncy, cells, cells_alignment(cells), (local % tx) * BX,
                                              (local / tx) * BY);
    }
}

// Table placement for a launch: the tuned choice, else the whole table
// through the read-only cache.
inline bool use_quad_table() { return tune_get(HOG_TUNE_TABLE) == 1; }

template <int CH, int NB, int S, typename OutT, bool QUAD, int BYT>
hog_status launch_q(const uint8_t* img, int W, int H, size_t pitch, const uint8_t* lut, int r, int ncx, int ncy,
                    void* cells, unsigned int* status, cudaStream_t st) {
    const size_t smem = (QUAD ? kQuadBytes : 0) + sizeof(FusedSmem<NB, S>);
    auto kern = cells_fused_kernel<CH, NB, S, OutT, QUAD, BYT>;
    cudaError_t e = smem_at_least<cells_fused_kernel<CH, NB, S, OutT, QUAD, BYT>>(smem);
    if (e != cudaSuccess) return cuda_fail(e);
    constexpr int BX = TileShape<S>::BX, BY = BYT;
    const int tiles = ((ncx + BX - 1) / BX) * ((ncy + BY - 1) / BY);
    const int per_sm = tune_get(HOG_TUNE_FUSED_CTAS_PER_SM);
    const int cap = (per_sm > 0 ? per_sm : 2) * sm_count();  // two CTAs of this size fit an SM
    const int grid = tiles < cap ? tiles : cap;
    const bool aligned = (reinterpret_cast<uintptr_t>(img) % 4 == 0) && (pitch % 4 == 0);
    const int out_align = cells_alignment(cells);
    return launch_pdl(kern, dim3(grid), dim3(kThreads), smem, st, img, W, H, pitch, aligned, lut, r, ncx, ncy,
                      static_cast<OutT*>(cells), out_align, status);
}

// Tile height in cell rows for one image: the tuned choice (16, 8 or 4), else
// 8 where tiles of 16 rows would leave SMs without one, else 16.  A tile's
// CTA bins its pixels (and its halo's) one quad per thread in turn, so on a
// small image twice as many tiles of half the height finish sooner; the halo
// then adds r - 1 block rows to 8 instead of to 16.  Rows of 4 were measured
// too: slightly faster than 8 at 800 x 600 (27.8-28.3 against 28.5 us for the
// fused step), 2 us slower at 640 x 480, so they are left to the tuner.
template <int S>
int fused_tile_rows(int ncx, int ncy) {
    const int tuned = tune_get(HOG_TUNE_FUSED_TILE_ROWS);
    if (tuned > 0) return tuned;
    constexpr int BX = TileShape<S>::BX, BY = TileShape<S>::BY;
    const long tiles = (long)((ncx + BX - 1) / BX) * ((ncy + BY - 1) / BY);
    return tiles < sm_count() ? BY / 2 : BY;
}

template <int CH, int NB, int S, typename OutT, bool QUAD>
hog_status launch_h(const uint8_t* img, int W, int H, size_t pitch, const uint8_t* lut, int r, int ncx, int ncy,
                    void* cells, unsigned int* status, cudaStream_t st) {
    static_assert(TileShape<S>::BY == 16, "tile heights 16, 8 and 4");
    const int rows = fused_tile_rows<S>(ncx, ncy);
    if (rows == 4) return launch_q<CH, NB, S, OutT, QUAD, 4>(img, W, H, pitch, lut, r, ncx, ncy, cells, status, st);
    if (rows == 8) return launch_q<CH, NB, S, OutT, QUAD, 8>(img, W, H, pitch, lut, r, ncx, ncy, cells, status, st);
    return launch_q<CH, NB, S, OutT, QUAD, 16>(img, W, H, pitch, lut, r, ncx, ncy, cells, status, st);
}

template <int CH, int NB, int S, typename OutT>
hog_status launch_t(const uint8_t* img, int W, int H, size_t pitch, const uint8_t* lut, int r, int ncx, int ncy,
                    void* cells, unsigned int* status, cudaStream_t st) {
    if (use_quad_table())
        return launch_h<CH, NB, S, OutT, true>(img, W, H, pitch, lut, r, ncx, ncy, cells, status, st);
    return launch_h<CH, NB, S, OutT, false>(img, W, H, pitch, lut, r, ncx, ncy, cells, status, st);
}

template <int CH, int NB, int S>
hog_status by_out(const uint8_t* img, int W, int H, size_t pitch, const uint8_t* lut, int r, int ncx, int ncy,
                  int cell_dtype, void* cells, unsigned int* status, cudaStream_t st) {
    if (cell_dtype == HOG_BF16)
        return launch_t<CH, NB, S, uint16_t>(img, W, H, pitch, lut, r, ncx, ncy, cells, status, st);
    if (cell_dtype == HOG_F32)
        return launch_t<CH, NB, S, float>(img, W, H, pitch, lut, r, ncx, ncy, cells, status, st);
    return launch_t<CH, NB, S, int32_t>(img, W, H, pitch, lut, r, ncx, ncy, cells, status, st);
}

template <int CH, int NB>
hog_status by_stride(const uint8_t* img, int W, int H, size_t pitch, const uint8_t* lut, int s, int r, int ncx,
                     int ncy, int cell_dtype, void* cells, unsigned int* status, cudaStream_t st) {
    if (s == 4) return by_out<CH, NB, 4>(img, W, H, pitch, lut, r, ncx, ncy, cell_dtype, cells, status, st);
    return by_out<CH, NB, 8>(img, W, H, pitch, lut, r, ncx, ncy, cell_dtype, cells, status, st);
}

}  // namespace

bool cells_fused_supported(int n_bins, int cell, int stride) {
    // tile shapes keep 16-bit corner sums below 2^15 for strides 4 and 8 with r <= 4
    return (n_bins == 8 || n_bins == 16) && (stride == 4 || stride == 8) && cell % stride == 0 &&
           cell / stride <= kMaxR;
}

hog_status launch_cells_fused(const uint8_t* img, int W, int H, int channels, size_t pitch, const uint8_t* lut,
                              int n_bins, int cell, int stride, int cell_dtype, void* cells, unsigned int* status,
                              cudaStream_t st) {
    const int ncx = W < cell ? 0 : (W - cell) / stride + 1;
    const int ncy = H < cell ? 0 : (H - cell) / stride + 1;
    if (ncx == 0 || ncy == 0) return HOG_OK;
    const int r = cell / stride;
    if (channels == 1)
        return n_bins == 8 ? by_stride<1, 8>(img, W, H, pitch, lut, stride, r, ncx, ncy, cell_dtype, cells, status, st)
                           : by_stride<1, 16>(img, W, H, pitch, lut, stride, r, ncx, ncy, cell_dtype, cells, status, st);
    return n_bins == 8 ? by_stride<3, 8>(img, W, H, pitch, lut, stride, r, ncx, ncy, cell_dtype, cells, status, st)
                       : by_stride<3, 16>(img, W, H, pitch, lut, stride, r, ncx, ncy, cell_dtype, cells, status, st);
}

int cells_fused_tiles_x(int ncx, int stride) {
    const int bx = stride == 4 ? TileShape<4>::BX : TileShape<8>::BX;
    return (ncx + bx - 1) / bx;
}

int cells_fused_tiles(int ncx, int ncy, int stride) {
    const int by = stride == 4 ? TileShape<4>::BY : TileShape<8>::BY;
    return cells_fused_tiles_x(ncx, stride) * ((ncy + by - 1) / by);
}

namespace {

template <int CH, int NB, int S, typename OutT, bool QUAD>
hog_status launch_batch_q(const PlanHeader& h, const void* plan_dev, const uint8_t* lut, unsigned int* status,
                          cudaStream_t st) {
    const size_t smem = (QUAD ? kQuadBytes : 0) + sizeof(FusedSmem<NB, S>);
    auto kern = cells_fused_batch_kernel<CH, NB, S, OutT, QUAD>;
    cudaError_t e = smem_at_least<cells_fused_batch_kernel<CH, NB, S, OutT, QUAD>>(smem);
    if (e != cudaSuccess) return cuda_fail(e);
    const int per_sm = tune_get(HOG_TUNE_FUSED_CTAS_PER_SM);
    const int cap = (per_sm > 0 ? per_sm : 2) * sm_count();
    const int grid = h.cells_tiles < cap ? h.cells_tiles : cap;
    return launch_pdl(kern, dim3(grid), dim3(kThreads), smem, st, plan_items(plan_dev), h.n_items, h.cells_tiles,
                      lut, h.r, status);
}

template <int CH, int NB, int S, typename OutT>
hog_status launch_batch_t(const PlanHeader& h, const void* plan_dev, const uint8_t* lut, unsigned int* status,
                          cudaStream_t st) {
    if (use_quad_table()) return launch_batch_q<CH, NB, S, OutT, true>(h, plan_dev, lut, status, st);
    return launch_batch_q<CH, NB, S, OutT, false>(h, plan_dev, lut, status, st);
}

template <int CH, int NB, int S>
hog_status batch_by_out(const PlanHeader& h, const void* plan_dev, const uint8_t* lut, int cell_dtype,
                        unsigned int* status, cudaStream_t st) {
    if (cell_dtype == HOG_BF16) return launch_batch_t<CH, NB, S, uint16_t>(h, plan_dev, lut, status, st);
    if (cell_dtype == HOG_F32) return launch_batch_t<CH, NB, S, float>(h, plan_dev, lut, status, st);
    return launch_batch_t<CH, NB, S, int32_t>(h, plan_dev, lut, status, st);
}

template <int CH, int NB>
hog_status batch_by_stride(const PlanHeader& h, const void* plan_dev, const uint8_t* lut, int cell_dtype,
                           unsigned int* status, cudaStream_t st) {
    if (h.stride == 4) return batch_by_out<CH, NB, 4>(h, plan_dev, lut, cell_dtype, status, st);
    return batch_by_out<CH, NB, 8>(h, plan_dev, lut, cell_dtype, status, st);
}

}  // namespace

hog_status launch_cells_fused_batch(const PlanHeader& h, const void* plan_dev, const uint8_t* lut, int cell_dtype,
                                    unsigned int* status, cudaStream_t st) {
    if (h.cells_tiles == 0) return HOG_OK;
    if (h.channels == 1)
        return h.n_bins == 8 ? batch_by_stride<1, 8>(h, plan_dev, lut, cell_dtype, status, st)
                             : batch_by_stride<1, 16>(h, plan_dev, lut, cell_dtype, status, st);
    return h.n_bins == 8 ? batch_by_stride<3, 8>(h, plan_dev, lut, cell_dtype, status, st)
                         : batch_by_stride<3, 16>(h, plan_dev, lut, cell_dtype, status, st);
}

}  // namespace fasthog
