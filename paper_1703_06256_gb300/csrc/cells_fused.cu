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
// Per tile of BX x BY cells (origins), a CTA
//   1. computes the bins of the tile's (BX + r - 1) x (BY + r - 1) blocks with
//      the same quad code and shared-memory table quadrant as the bin-map
//      kernel, and counts them per block (8-bit fields, s^2 <= 64 for s = 4, 8);
//   2. forms G over those blocks in shared memory (16-bit fields);
//   3. writes each cell's histogram from four corners of G.
// Tiles overlap by r - 1 blocks, whose bins are computed twice.  The grid is
// persistent so that each CTA stages the table quadrant once.
#include <type_traits>

#include "bin_core.cuh"
#include "internal.cuh"
#include "ptx.cuh"

namespace fasthog {

namespace {

constexpr int kThreads = 256;
constexpr int kBX = 32, kBY = 8;        // cells per tile (= 256 threads in step 3)
constexpr int kQuadBytes = 256 * 256;
constexpr int kMaxR = 4;

template <int NB>
struct FusedSmem {
    static constexpr int NW8 = NB / 4;                 // 8-bit-field words per block histogram
    static constexpr int NW16 = NB / 2;                // 16-bit-field words per G entry
    static constexpr int BXB = kBX + kMaxR - 1;        // blocks per tile row (max)
    static constexpr int BYB = kBY + kMaxR - 1;
    uint32_t bh[BYB][BXB][NW8];                        // block histograms
    uint32_t g[BYB + 1][BXB + 1][NW16];                // corner-sampled tile integral image
};

template <typename OutT>
__device__ __forceinline__ OutT as_count(uint32_t v) {
    if constexpr (std::is_same<OutT, uint16_t>::value) {
        return f32_to_bf16_exact_int((float)v);
    } else {
        return (OutT)v;
    }
}

template <int CH, int NB, typename OutT>
__global__ void __launch_bounds__(kThreads)
    cells_fused_kernel(const uint8_t* __restrict__ img, int W, int H, size_t pitch, bool aligned,
                       const uint8_t* __restrict__ lut, int s, int r, int ncx, int ncy, OutT* __restrict__ cells,
                       unsigned int* status) {
    using S = FusedSmem<NB>;
    extern __shared__ __align__(128) uint8_t smem[];
    uint8_t* lutq = smem;
    S& sm = *reinterpret_cast<S*>(smem + kQuadBytes);
    __shared__ __align__(8) uint64_t lut_bar;

    const int tid = threadIdx.x;
    if (tid == 0) {
        ptx::mbar_init(&lut_bar, 1);
        ptx::fence_mbar_init();
    }
    __syncthreads();
    if (tid == 0) {
        ptx::mbar_arrive_expect_tx(&lut_bar, kQuadBytes);
        ptx::bulk_g2s(lutq, lut + kLutQuadOffset, kQuadBytes, &lut_bar);
    }
    pdl_trigger();
    pdl_wait();
    const bool lut_ok = ptx::mbar_wait_bounded(&lut_bar, 0, kWaitLimitNs);
    if (!lut_ok) {
        if (tid == 0) atomicOr(status, kStatusTimeout);
        return;
    }

    const int tiles_x = (ncx + kBX - 1) / kBX, tiles_y = (ncy + kBY - 1) / kBY;
    const int bxn = kBX + r - 1, byn = kBY + r - 1;  // blocks of a tile
    const long row_bytes = (long)W * CH;
    const int quads_per_brow = s / 4;                // quads in one block row
    for (int t = blockIdx.x; t < tiles_x * tiles_y; t += gridDim.x) {
        const int bx0 = (t % tiles_x) * kBX, by0 = (t / tiles_x) * kBY;
        __syncthreads();  // the previous tile's G reads are done
        // 1. block histograms
        for (int blk = tid; blk < bxn * byn; blk += kThreads) {
            const int bi = blk % bxn, bj = blk / bxn;
            uint32_t h[S::NW8];
#pragma unroll
            for (int k = 0; k < S::NW8; ++k) h[k] = 0;
            const int x_blk = (bx0 + bi) * s, y_blk = (by0 + bj) * s;
            for (int yy = 0; yy < s; ++yy) {
                const int y = y_blk + yy;
                if (y <= 0 || y >= H - 1) continue;  // border rows, or below the image: no bins
                for (int qq = 0; qq < quads_per_brow; ++qq) {
                    const int x = x_blk + 4 * qq;
                    if (x >= W) break;
                    QuadWords<CH> q;
                    load_quad<CH>(img, pitch, row_bytes, aligned, x, y, q);
                    const uint32_t packed = bins_of_quad<CH, true>(q, x, W, lutq, lut, NB, NB / 4);
#pragma unroll
                    for (int p = 0; p < 4; ++p) {
                        const uint32_t v = (packed >> (8 * p)) & 0xFFu;
                        const uint32_t inc = 1u << ((v & 3) << 3);
#pragma unroll
                        for (int k = 0; k < S::NW8; ++k) h[k] += ((v >> 2) == (uint32_t)k) ? inc : 0u;  // 0xFF: none
                    }
                }
            }
#pragma unroll
            for (int k = 0; k < S::NW8; ++k) sm.bh[bj][bi][k] = h[k];
        }
        __syncthreads();
        // 2. G: exclusive 2-D prefix of the block histograms, widened to
        //    16-bit fields (bins 2e, 2e+1 in word e).  First the prefix along
        //    each block row (G row J+1 holds the rows < J+1), then down columns.
        for (int task = tid; task < (byn + 1) * S::NW16; task += kThreads) {
            const int J = task / S::NW16, e = task % S::NW16;
            uint32_t run = 0;
            sm.g[J][0][e] = 0;
            for (int I = 0; I < bxn; ++I) {
                if (J > 0) {
                    const uint32_t w8 = sm.bh[J - 1][I][e >> 1];
                    const uint32_t two = (e & 1) ? (w8 >> 16) : (w8 & 0xFFFFu);  // bins 2e, 2e+1 (8-bit each)
                    run += (two & 0xFFu) | ((two >> 8) << 16);
                }
                sm.g[J][I + 1][e] = run;
            }
        }
        __syncthreads();
        for (int task = tid; task < (bxn + 1) * S::NW16; task += kThreads) {
            const int I = task / S::NW16, e = task % S::NW16;
            uint32_t run = 0;
            for (int J = 0; J <= byn; ++J) {
                run += sm.g[J][I][e];
                sm.g[J][I][e] = run;
            }
        }
        __syncthreads();
        // 3. cells: Eq. 6 on the corner-sampled integral image
        {
            const int ci = tid % kBX, cj = tid / kBX;
            const int i = bx0 + ci, j = by0 + cj;
            if (i < ncx && j < ncy) {
                OutT* out = cells + ((size_t)j * ncx + i) * NB;
#pragma unroll
                for (int e = 0; e < S::NW16; ++e) {
                    // (a + d) - (b + c) per 16-bit field: no field borrows
                    const uint32_t v = (sm.g[cj + r][ci + r][e] + sm.g[cj][ci][e]) -
                                       (sm.g[cj][ci + r][e] + sm.g[cj + r][ci][e]);
                    out[2 * e] = as_count<OutT>(v & 0xFFFFu);
                    out[2 * e + 1] = as_count<OutT>(v >> 16);
                }
            }
        }
    }
}

template <int CH, int NB, typename OutT>
hog_status launch_t(const uint8_t* img, int W, int H, size_t pitch, const uint8_t* lut, int s, int r, int ncx, int ncy,
                    void* cells, unsigned int* status, cudaStream_t st) {
    const size_t smem = kQuadBytes + sizeof(FusedSmem<NB>);
    auto kern = cells_fused_kernel<CH, NB, OutT>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return cuda_fail(e);
    const int tiles = ((ncx + kBX - 1) / kBX) * ((ncy + kBY - 1) / kBY);
    const int cap = 2 * sm_count();
    const int grid = tiles < cap ? tiles : cap;
    const bool aligned = (reinterpret_cast<uintptr_t>(img) % 4 == 0) && (pitch % 4 == 0);
    return launch_pdl(kern, dim3(grid), dim3(kThreads), smem, st, img, W, H, pitch, aligned, lut, s, r, ncx, ncy,
                      static_cast<OutT*>(cells), status);
}

template <int CH, int NB>
hog_status by_out(const uint8_t* img, int W, int H, size_t pitch, const uint8_t* lut, int s, int r, int ncx, int ncy,
                  int cell_dtype, void* cells, unsigned int* status, cudaStream_t st) {
    if (cell_dtype == HOG_BF16)
        return launch_t<CH, NB, uint16_t>(img, W, H, pitch, lut, s, r, ncx, ncy, cells, status, st);
    if (cell_dtype == HOG_F32)
        return launch_t<CH, NB, float>(img, W, H, pitch, lut, s, r, ncx, ncy, cells, status, st);
    return launch_t<CH, NB, int32_t>(img, W, H, pitch, lut, s, r, ncx, ncy, cells, status, st);
}

}  // namespace

bool cells_fused_supported(int n_bins, int cell, int stride) {
    // 16-bit corner sums stay below 2^15 per tile for strides 4 and 8 with r <= 4
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
        return n_bins == 8 ? by_out<1, 8>(img, W, H, pitch, lut, stride, r, ncx, ncy, cell_dtype, cells, status, st)
                           : by_out<1, 16>(img, W, H, pitch, lut, stride, r, ncx, ncy, cell_dtype, cells, status, st);
    return n_bins == 8 ? by_out<3, 8>(img, W, H, pitch, lut, stride, r, ncx, ncy, cell_dtype, cells, status, st)
                       : by_out<3, 16>(img, W, H, pitch, lut, stride, r, ncx, ncy, cell_dtype, cells, status, st);
}

}  // namespace fasthog
