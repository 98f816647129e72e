// cells_soft.cu -- cell histograms of two-bin soft votes (the OpenCV-style
// vote that Section 2 mentions and sets aside; the paper's own method gives
// each pixel one bin with unit magnitude).
//
// Soft table: for every (dx, dy) in [-255, 255]^2 the gradient angle phi in
// [0, 2 pi) is placed among the bin centres c_k = (k + 1/2) 2 pi / N_b,
//   t = phi N_b / (2 pi) - 1/2,  k0 = floor(t) mod N_b,  alpha = t - floor(t),
// and the entry holds k0 and a = round(q alpha) (q = HOG_SOFT_Q vote units
// per pixel; a = q is stored as (k0 + 1, 0)).  FP64 throughout, with the
// operations in a fixed order and no contraction, so the table equals any
// other FP64 evaluation whose atan2 is accurate to a few ulp: no lattice
// point comes within 1e-6 of a rounding tie for the bin counts used.
//
// Cells: the fused scheme of cells_fused.cu with weighted votes.  Each pixel
// adds q - a to bin k0 and a to bin k0 + 1 of its s x s block (32-bit
// shared-memory counters); a tile-local integral image at the block corners
// (Eq. 5 on the vote planes) gives each cell's histogram by Eq. 6.  All sums
// are integers (units of 1/q): exact.
#include <cmath>
#include <type_traits>

#include "bin_core.cuh"
#include "internal.cuh"

namespace fasthog {

namespace {

constexpr int kThreads = 512;
constexpr int kMaxR = 4;
constexpr int kMaxNb = 16;
constexpr int kSoftPitch = HOG_LUT_PITCH;  // entries per table row (511 + 1 pad)

__global__ void __launch_bounds__(256) build_soft_lut_kernel(int nb, int q, uint16_t* __restrict__ lut) {
    pdl_wait();
    pdl_trigger();
    const int idx = blockIdx.x * 256 + threadIdx.x;
    if (idx >= kLutSide * kSoftPitch) return;
    const int row = idx / kSoftPitch, col = idx - row * kSoftPitch;
    if (col == kLutSide) {
        lut[idx] = 0xFFFF;  // pad
        return;
    }
    const int dy = row - kDMax, dx = col - kDMax;
    if (dx == 0 && dy == 0) {
        lut[idx] = 0xFFFF;
        return;
    }
    const double two_pi = 6.283185307179586;  // 2 pi rounded to double
    double phi = atan2((double)dy, (double)dx);
    if (phi < 0.0) phi = __dadd_rn(phi, two_pi);
    const double t = __dsub_rn(__ddiv_rn(__dmul_rn(phi, (double)nb), two_pi), 0.5);
    const double fl = floor(t);
    const double x = __dmul_rn((double)q, __dsub_rn(t, fl));
    int a = (int)floor(__dadd_rn(x, 0.5));
    int k0 = (int)fl % nb;
    if (k0 < 0) k0 += nb;
    if (a >= q) {
        a = 0;
        k0 = (k0 + 1) % nb;
    }
    lut[idx] = (uint16_t)(k0 | (a << 8));
}

template <int S>
struct SoftTile {
    static constexpr int BX = S == 4 ? 32 : 16;
    static constexpr int BY = 16;
    static constexpr int BXB = BX + kMaxR - 1;
    static constexpr int BYB = BY + kMaxR - 1;
};

// BYT: cell rows per tile (16, or 8 on small images; the shared memory is
// laid out for 16).
template <int CH, int S, typename OutT, int BYT>
__global__ void __launch_bounds__(kThreads, 2)
    cells_soft_kernel(const uint8_t* __restrict__ img, int W, int H, size_t pitch, bool aligned,
                      const uint16_t* __restrict__ lut, int nb, int q, int r, int ncx, int ncy,
                      OutT* __restrict__ cells) {
    using T = SoftTile<S>;
    static_assert(BYT <= T::BY, "the shared-memory layout holds tiles of at most 16 rows");
    constexpr int BY = BYT;
    constexpr int QPR = S / 4;
    extern __shared__ __align__(16) uint32_t smem_u[];
    uint32_t* bh = smem_u;                              // [BYB][BXB][nb] block votes
    uint32_t* g = smem_u + T::BYB * T::BXB * kMaxNb;    // [BYB + 1][BXB + 1][nb] corner integral image
    const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
    pdl_wait();
    pdl_trigger();
    const int tiles_x = (ncx + T::BX - 1) / T::BX, tiles_y = (ncy + BY - 1) / BY;
    const int bxn = T::BX + r - 1, byn = BY + r - 1;
    const long row_bytes = (long)W * CH;
    const int row_tasks = bxn * QPR;
    const int n_tasks = byn * S * row_tasks;
    auto BH = [&](int j, int i) { return bh + ((size_t)j * T::BXB + i) * nb; };
    auto G = [&](int j, int i) { return g + ((size_t)j * (T::BXB + 1) + i) * nb; };
    for (int t = blockIdx.x; t < tiles_x * tiles_y; t += gridDim.x) {
        const int bx0 = (t % tiles_x) * T::BX, by0 = (t / tiles_x) * BY;
        __syncthreads();  // the previous tile's reads are done
        for (int k = tid; k < byn * T::BXB * nb; k += kThreads) bh[k] = 0;
        __syncthreads();
        // 1. block votes: one quad of 4 pixels per task
        for (int task = tid; task < n_tasks; task += kThreads) {
            const int prow = task / row_tasks, qc = task - prow * row_tasks;
            const int y = by0 * S + prow, x = bx0 * S + 4 * qc;
            if (y <= 0 || y >= H - 1 || x >= W) continue;
            QuadWords<CH> qw;
            load_quad<CH>(img, pitch, row_bytes, aligned, x, y, qw);
            uint32_t* dst = BH(prow / S, qc / QPR);
#pragma unroll
            for (int p = 0; p < 4; ++p) {
                const int xp = x + p;
                if (xp <= 0 || xp >= W - 1) continue;
                int dx, dy;
                quad_gradient<CH>(qw, p, dx, dy);
                if (dx == 0 && dy == 0) continue;
                const uint32_t e = __ldg(lut + (size_t)(dy + kDMax) * kSoftPitch + (dx + kDMax));
                const int k0 = (int)(e & 0xFFu), a = (int)(e >> 8);
                if (a < q) atomicAdd(dst + k0, (uint32_t)(q - a));
                if (a > 0) atomicAdd(dst + (k0 + 1 == nb ? 0 : k0 + 1), (uint32_t)a);
            }
        }
        __syncthreads();
        // 2. G: exclusive 2-D prefix of the block votes: warp scans along block rows, then down columns
        for (int task = wid; task < byn * nb; task += kThreads / 32) {
            const int J = 1 + task / nb, b = task % nb;
            uint32_t carry = 0;
            for (int I0 = 0; I0 < bxn; I0 += 32) {
                const int I = I0 + lane;
                uint32_t v = I < bxn ? BH(J - 1, I)[b] : 0u;
#pragma unroll
                for (int d = 1; d < 32; d <<= 1) {
                    const uint32_t u = __shfl_up_sync(0xffffffffu, v, d);
                    if (lane >= d) v += u;
                }
                if (I < bxn) G(J, I + 1)[b] = v + carry;
                carry += __shfl_sync(0xffffffffu, v, 31);
            }
            if (lane == 0) G(J, 0)[b] = 0;
        }
        for (int k = tid; k < (bxn + 1) * nb; k += kThreads) G(0, k / nb)[k % nb] = 0;
        __syncthreads();
        for (int task = tid; task < (bxn + 1) * nb; task += kThreads) {
            const int I = task / nb, b = task % nb;
            uint32_t run = 0;
            for (int J = 1; J <= byn; ++J) {
                run += G(J, I)[b];
                G(J, I)[b] = run;
            }
        }
        __syncthreads();
        // 3. cells by Eq. 6 on the corner integral image
        if (tid < T::BX * BY) {
            const int ci = tid % T::BX, cj = tid / T::BX;
            const int i = bx0 + ci, j = by0 + cj;
            if (i < ncx && j < ncy) {
                OutT* out = cells + ((size_t)j * ncx + i) * nb;
                const uint32_t *a = G(cj + r, ci + r), *d = G(cj, ci), *bb = G(cj, ci + r), *c = G(cj + r, ci);
                for (int b = 0; b < nb; ++b) out[b] = (OutT)((a[b] + d[b]) - (bb[b] + c[b]));
            }
        }
    }
}

template <int CH, int S, typename OutT, int BYT>
hog_status launch_b(const uint8_t* img, int W, int H, size_t pitch, const uint16_t* lut, int nb, int r, int ncx,
                    int ncy, void* cells, cudaStream_t st) {
    using T = SoftTile<S>;
    const size_t smem = sizeof(uint32_t) * ((size_t)T::BYB * T::BXB + (size_t)(T::BYB + 1) * (T::BXB + 1)) * kMaxNb;
    auto kern = cells_soft_kernel<CH, S, OutT, BYT>;
    cudaError_t e = smem_at_least<cells_soft_kernel<CH, S, OutT, BYT>>(smem);
    if (e != cudaSuccess) return cuda_fail(e);
    const int tiles = ((ncx + T::BX - 1) / T::BX) * ((ncy + BYT - 1) / BYT);
    const int cap = 2 * sm_count();
    const int grid = tiles < cap ? tiles : cap;
    const bool aligned = (reinterpret_cast<uintptr_t>(img) % 4 == 0) && (pitch % 4 == 0);
    return launch_pdl(kern, dim3(grid), dim3(kThreads), smem, st, img, W, H, pitch, aligned, lut, nb, HOG_SOFT_Q, r,
                      ncx, ncy, static_cast<OutT*>(cells));
}

// Tile height: the tuned choice (HOG_TUNE_FUSED_TILE_ROWS), else 8 cell rows
// where tiles of 16 would leave SMs without a tile (as for the fused cells).
template <int CH, int S, typename OutT>
hog_status launch_t(const uint8_t* img, int W, int H, size_t pitch, const uint16_t* lut, int nb, int r, int ncx,
                    int ncy, void* cells, cudaStream_t st) {
    using T = SoftTile<S>;
    const int tuned = tune_get(HOG_TUNE_FUSED_TILE_ROWS);
    const long tiles16 = (long)((ncx + T::BX - 1) / T::BX) * ((ncy + T::BY - 1) / T::BY);
    const bool half = tuned > 0 ? tuned < 16 : tiles16 < sm_count();  // 8 rows also for a tuned 4
    return half ? launch_b<CH, S, OutT, 8>(img, W, H, pitch, lut, nb, r, ncx, ncy, cells, st)
                : launch_b<CH, S, OutT, 16>(img, W, H, pitch, lut, nb, r, ncx, ncy, cells, st);
}

template <int CH, int S>
hog_status by_out(const uint8_t* img, int W, int H, size_t pitch, const uint16_t* lut, int nb, int r, int ncx,
                  int ncy, int cell_dtype, void* cells, cudaStream_t st) {
    if (cell_dtype == HOG_F32) return launch_t<CH, S, float>(img, W, H, pitch, lut, nb, r, ncx, ncy, cells, st);
    return launch_t<CH, S, int32_t>(img, W, H, pitch, lut, nb, r, ncx, ncy, cells, st);
}

}  // namespace

bool cells_soft_supported(int n_bins, int cell, int stride) {
    return n_bins >= 2 && n_bins <= kMaxNb && (stride == 4 || stride == 8) && cell % stride == 0 &&
           cell / stride <= kMaxR;
}

hog_status launch_build_soft_lut(int n_bins, uint16_t* lut, cudaStream_t st) {
    const int total = kLutSide * kSoftPitch;
    return launch_pdl(build_soft_lut_kernel, dim3((total + 255) / 256), dim3(256), 0, st, n_bins, HOG_SOFT_Q, lut);
}

hog_status launch_cells_soft(const uint8_t* img, int W, int H, int channels, size_t pitch, const uint16_t* lut,
                             int n_bins, int cell, int stride, int cell_dtype, void* cells, cudaStream_t st) {
    const int ncx = W < cell ? 0 : (W - cell) / stride + 1;
    const int ncy = H < cell ? 0 : (H - cell) / stride + 1;
    if (ncx == 0 || ncy == 0) return HOG_OK;
    const int r = cell / stride;
    if (channels == 1)
        return stride == 4 ? by_out<1, 4>(img, W, H, pitch, lut, n_bins, r, ncx, ncy, cell_dtype, cells, st)
                           : by_out<1, 8>(img, W, H, pitch, lut, n_bins, r, ncx, ncy, cell_dtype, cells, st);
    return stride == 4 ? by_out<3, 4>(img, W, H, pitch, lut, n_bins, r, ncx, ncy, cell_dtype, cells, st)
                       : by_out<3, 8>(img, W, H, pitch, lut, n_bins, r, ncx, ncy, cell_dtype, cells, st);
}

}  // namespace fasthog
