// cell_hist.cu -- area histograms from four integral-image corners
// (paper Section 3.3, Eq. 6; Section 3.1, Eq. 3 applied per bin).
//
// One thread per cell.  For each bin the thread reads the four corners
//   ii(x1, y1), ii(x0-1, y0-1), ii(x1, y0-1), ii(x0-1, y1)
// (an index of -1 reads 0) and writes the cell's histogram contiguously,
// bin innermost, as int32 or bf16 (counts <= cell^2 are small integers).
// Consecutive threads take consecutive cells of a row, so the corner loads
// of a warp fall in a few 128-byte lines of the same two ii rows; corners
// shared by neighbouring cells are served by L1.
//
// With uint16 integral images the four-term sum is taken modulo 2^16, which
// is exact because a cell holds fewer than 65536 pixels.
//
// For cells made of whole strides (cell = r * stride) and 8 or 16 bins a
// streaming variant (below) reads only the grid of integral-image samples
// Eq. 6 uses, through shared memory.
#include <type_traits>

#include "internal.cuh"

namespace fasthog {

namespace {

template <typename OutT>
__device__ __forceinline__ OutT count_as(uint32_t v) {
    if constexpr (std::is_same<OutT, uint16_t>::value) {
        return f32_to_bf16_exact_int((float)v);
    } else {
        return (OutT)v;  // int32, or float (counts are exact)
    }
}

// NB > 0: the bin count is a compile-time constant, so all 4 * NB corner
// loads of a cell are issued before any of them is used.  NB == 0: any N_b.
template <typename InT, typename OutT, int NB>
__global__ void __launch_bounds__(128)
    cell_hist_kernel(const InT* __restrict__ ii, int W, int H, int nb_rt, int cell, int stride, int ncx, int ncy,
                     OutT* __restrict__ cells) {
    pdl_wait();
    pdl_trigger();
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    const int j = blockIdx.y;
    if (i >= ncx || j >= ncy) return;
    const int nb = NB > 0 ? NB : nb_rt;
    const int x0 = i * stride, y0 = j * stride;
    const int x1 = x0 + cell - 1, y1 = y0 + cell - 1;
    const bool hx = x0 > 0, hy = y0 > 0;
    const size_t plane = (size_t)W * H;
    const InT* p11 = ii + (size_t)y1 * W + x1;
    const InT* p01 = ii + (size_t)y1 * W + (x0 - 1);
    const InT* p10 = ii + (size_t)(y0 - 1) * W + x1;
    const InT* p00 = ii + (size_t)(y0 - 1) * W + (x0 - 1);
    OutT* out = cells + ((size_t)j * ncx + i) * nb;
    if constexpr (NB > 0) {
        uint32_t v[NB];
#pragma unroll
        for (int b = 0; b < NB; ++b) {
            v[b] = (uint32_t)__ldg(p11 + b * plane);
            if (hx) v[b] -= (uint32_t)__ldg(p01 + b * plane);
            if (hy) v[b] -= (uint32_t)__ldg(p10 + b * plane);
            if (hx && hy) v[b] += (uint32_t)__ldg(p00 + b * plane);
        }
#pragma unroll
        for (int b = 0; b < NB; ++b) {
            if (sizeof(InT) == 2) v[b] &= 0xFFFFu;
            out[b] = count_as<OutT>(v[b]);
        }
    } else {
        for (int b = 0; b < nb; ++b) {
            uint32_t v = (uint32_t)__ldg(p11 + b * plane);
            if (hx) v -= (uint32_t)__ldg(p01 + b * plane);
            if (hy) v -= (uint32_t)__ldg(p10 + b * plane);
            if (hx && hy) v += (uint32_t)__ldg(p00 + b * plane);
            if (sizeof(InT) == 2) v &= 0xFFFFu;
            out[b] = count_as<OutT>(v);
        }
    }
}

// Streaming variant for cell = r * stride.  Eq. 6 only reads the integral
// image on a grid: with S[k][m] = ii(s m - 1, s k - 1) (0 for k = 0 or
// m = 0), cell (i, j) = S[j+r][i+r] - S[j][i+r] - S[j+r][i] + S[j][i].  A CTA
// owns TJ x kTI cells, loads its (TJ + r) x (kTI + r) samples of every bin
// into shared memory (many independent loads in flight; the sample rows of
// neighbouring tiles overlap by r), then forms and writes its cells in
// output order.  Shared rows are padded to NB + 1 words per sample so that
// the loads (consecutive samples of a row) do not collide in banks.
constexpr int kTI = 64;
constexpr int kStreamThreads = 256;

template <typename InT, typename OutT, int NB>
__global__ void __launch_bounds__(kStreamThreads, 4)
    cell_hist_stream_kernel(const InT* __restrict__ ii, int W, int H, int s, int r, int ncx, int ncy, int TJ,
                            OutT* __restrict__ cells) {
    extern __shared__ uint32_t S[];  // [TJ + r][kTI + r][NB + 1]
    pdl_wait();
    pdl_trigger();
    const int i0 = blockIdx.x * kTI, j0 = blockIdx.y * TJ;
    const int rows = TJ + r, cols = kTI + r;
    const int kmax = ncy - 1 + r, mmax = ncx - 1 + r;  // last sample rows / columns any cell reads
    const size_t plane = (size_t)W * H;
    // one warp per (sample row, bin) line, lanes over the line's samples
    // (cols <= kTI + 8 < 3 * 32); a warp issues the loads of kLines lines
    // before it stores any of them, so their latencies overlap
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    constexpr int kWarps = kStreamThreads / 32, kLines = 8, kPerLane = 3;
    for (int l0 = warp * kLines; l0 < rows * NB; l0 += kWarps * kLines) {
        uint32_t v[kLines][kPerLane];
#pragma unroll
        for (int q = 0; q < kLines; ++q) {
            const int line = l0 + q;
            const int kk = line / NB, b = line - kk * NB;
            const int k = j0 + kk;
            const bool row_ok = line < rows * NB && k > 0 && k <= kmax;
            const InT* src = ii + b * plane + (size_t)(s * k - 1) * W - 1;  // sample m at src + s * m
#pragma unroll
            for (int t = 0; t < kPerLane; ++t) {
                const int mm = lane + 32 * t, m = i0 + mm;
                v[q][t] = (row_ok && mm < cols && m > 0 && m <= mmax) ? (uint32_t)__ldg(src + (size_t)s * m) : 0u;
            }
        }
#pragma unroll
        for (int q = 0; q < kLines; ++q) {
            const int line = l0 + q;
            if (line >= rows * NB) break;
            const int kk = line / NB, b = line - kk * NB;
            uint32_t* dst = S + (size_t)kk * cols * (NB + 1) + b;
#pragma unroll
            for (int t = 0; t < kPerLane; ++t) {
                const int mm = lane + 32 * t;
                if (mm < cols) dst[mm * (NB + 1)] = v[q][t];
            }
        }
    }
    __syncthreads();
    const int outs = TJ * kTI * NB;
    for (int e = threadIdx.x; e < outs; e += kStreamThreads) {
        const int b = e % NB, rest = e / NB;
        const int ci = rest % kTI, cj = rest / kTI;
        const int i = i0 + ci, j = j0 + cj;
        if (i >= ncx || j >= ncy) continue;
        const uint32_t a = S[((cj + r) * cols + ci + r) * (NB + 1) + b];
        const uint32_t d = S[(cj * cols + ci) * (NB + 1) + b];
        const uint32_t bb = S[(cj * cols + ci + r) * (NB + 1) + b];
        const uint32_t c = S[((cj + r) * cols + ci) * (NB + 1) + b];
        uint32_t v = (a + d) - (bb + c);
        if (sizeof(InT) == 2) v &= 0xFFFFu;
        cells[((size_t)j * ncx + i) * NB + b] = count_as<OutT>(v);
    }
}

// One cell's NB counts as OutT at `out`: 16-byte stores when the map is 16-byte
// aligned (a cell is 16 or 32 bytes of bf16, 32 or 64 of 4-byte counts), else
// one store per count.
template <typename OutT, int NB>
__device__ __forceinline__ void write_cell(OutT* __restrict__ out, const uint32_t (&val)[NB], bool vec) {
    if (vec) {
        if constexpr (sizeof(OutT) == 2) {
#pragma unroll
            for (int k = 0; k < NB / 8; ++k) {
                uint32_t w[4];
#pragma unroll
                for (int e = 0; e < 4; ++e)
                    w[e] = (uint32_t)count_as<OutT>(val[8 * k + 2 * e]) |
                           ((uint32_t)count_as<OutT>(val[8 * k + 2 * e + 1]) << 16);
                reinterpret_cast<uint4*>(out)[k] = make_uint4(w[0], w[1], w[2], w[3]);
            }
        } else {
#pragma unroll
            for (int k = 0; k < NB / 4; ++k) {
                uint32_t w[4];
#pragma unroll
                for (int e = 0; e < 4; ++e) {
                    const OutT o = count_as<OutT>(val[4 * k + e]);
                    w[e] = *reinterpret_cast<const uint32_t*>(&o);
                }
                reinterpret_cast<uint4*>(out)[k] = make_uint4(w[0], w[1], w[2], w[3]);
            }
        }
    } else {
#pragma unroll
        for (int b = 0; b < NB; ++b) out[b] = count_as<OutT>(val[b]);
    }
}

// Persistent, double-buffered form of the streaming kernel, for tiles whose
// (TJ + r) x N_b sample lines fit one batch of loads per warp (kWarps x
// kLines): a CTA walks tiles with the grid's stride, and while it forms the
// cells of one tile from shared memory, the loads of its next tile are
// already in flight into registers; they are parked in the other buffer
// after the cells are written.  One barrier per tile.
constexpr int kPipeLines = 8;  // lines per warp and tile

template <typename InT, typename OutT, int NB>
__global__ void __launch_bounds__(kStreamThreads, 4)
    cell_hist_pipe_kernel(const InT* __restrict__ ii, int W, int H, int s, int r, int ncx, int ncy, int TJ, int n_tx,
                          int n_tiles, OutT* __restrict__ cells, bool vec_out) {
    extern __shared__ uint32_t S[];  // 2 x [TJ + r][kTI + r][NB + 1]
    pdl_wait();
    pdl_trigger();
    constexpr int kPerLane = 3;
    const int rows = TJ + r, cols = kTI + r, nlines = rows * NB;
    const size_t bufw = (size_t)rows * cols * (NB + 1);
    const int kmax = ncy - 1 + r, mmax = ncx - 1 + r;  // last sample rows / columns any cell reads
    const size_t plane = (size_t)W * H;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    uint32_t v[kPipeLines][kPerLane];
    static_assert((NB & (NB - 1)) == 0 && NB % 8 == 0, "8 or 16 bins: whole 16-byte stores per cell");
    // loads of tile t's samples: warp w takes lines w * kPipeLines .. + kPipeLines - 1,
    // lane l the samples l, l + 32, l + 64 of each line
    auto issue = [&](int t) {
        const int i0 = (t % n_tx) * kTI, j0 = (t / n_tx) * TJ;
        int off[kPerLane];
        bool colok[kPerLane];
#pragma unroll
        for (int u = 0; u < kPerLane; ++u) {
            const int mm = lane + 32 * u, m = i0 + mm;
            colok[u] = mm < cols && m > 0 && m <= mmax;
            off[u] = s * m - 1;
        }
#pragma unroll
        for (int q = 0; q < kPipeLines; ++q) {
            const int line = warp * kPipeLines + q;
            const int kk = line / NB, b = line & (NB - 1);
            const int k = j0 + kk;
            const bool row_ok = line < nlines && k > 0 && k <= kmax;
            const InT* row = ii + (size_t)b * plane + (size_t)(s * k - 1) * W;
#pragma unroll
            for (int u = 0; u < kPerLane; ++u) v[q][u] = (row_ok && colok[u]) ? (uint32_t)__ldg(row + off[u]) : 0u;
        }
    };
    auto park = [&](uint32_t* buf) {
#pragma unroll
        for (int q = 0; q < kPipeLines; ++q) {
            const int line = warp * kPipeLines + q;
            if (line >= nlines) break;
            const int kk = line / NB, b = line & (NB - 1);
            uint32_t* dst = buf + (size_t)kk * cols * (NB + 1) + b;
#pragma unroll
            for (int u = 0; u < kPerLane; ++u) {
                const int mm = lane + 32 * u;
                if (mm < cols) dst[mm * (NB + 1)] = v[q][u];
            }
        }
    };
    int t = blockIdx.x;
    if (t >= n_tiles) return;
    issue(t);
    park(S);
    __syncthreads();
    int cur = 0;
    for (; t < n_tiles; t += gridDim.x) {
        const int tn = t + gridDim.x;
        if (tn < n_tiles) issue(tn);
        const uint32_t* B = S + cur * bufw;
        const int i0 = (t % n_tx) * kTI, j0 = (t / n_tx) * TJ;
        // one cell (all NB bins) per thread and step, cells of the tile in row-major order: a lane's
        // samples are NB + 1 words from its neighbour's (no bank conflicts), and its cell's counts
        // leave in 16-byte stores next to its neighbour's
        const int rstep = cols * (NB + 1);
        for (int cell = threadIdx.x; cell < TJ * kTI; cell += kStreamThreads) {
            const int ci = cell % kTI, cj = cell / kTI;
            const int i = i0 + ci, j = j0 + cj;
            if (i >= ncx || j >= ncy) continue;
            const uint32_t* top = B + (size_t)cj * rstep + (size_t)ci * (NB + 1);  // sample (cj, ci), bin 0
            uint32_t val[NB];
#pragma unroll
            for (int b = 0; b < NB; ++b) {
                // samples (cj, ci), (cj, ci + r), (cj + r, ci), (cj + r, ci + r)
                const uint32_t d = top[b], bb = top[r * (NB + 1) + b];
                const uint32_t c = top[r * rstep + b], a = top[r * rstep + r * (NB + 1) + b];
                uint32_t v = (a + d) - (bb + c);
                if (sizeof(InT) == 2) v &= 0xFFFFu;
                val[b] = v;
            }
            write_cell<OutT, NB>(cells + ((size_t)j * ncx + i) * NB, val, vec_out);
        }
        // the other buffer was last read before the previous barrier
        if (tn < n_tiles) park(S + (cur ^ 1) * bufw);
        __syncthreads();
        cur ^= 1;
    }
}

// Rows of cells per streaming CTA: the tuned value (1 = the per-cell kernel),
// else 4 (measured best or tied among 4, 8 and 16 from 800x600 to 3840x2160).
int stream_rows(int ncx, int ncy) {
    (void)ncx;
    (void)ncy;
    const int tuned = tune_get(HOG_TUNE_CELL_ROWS);
    return tuned > 0 ? tuned : 4;
}

template <typename InT, typename OutT, int NB>
hog_status launch_stream(const void* ii, int W, int H, int stride, int r, int ncx, int ncy, int TJ, void* cells,
                         cudaStream_t st) {
    if ((TJ + r) * NB <= (kStreamThreads / 32) * kPipeLines) {
        const size_t smem = 2 * sizeof(uint32_t) * (size_t)(TJ + r) * (kTI + r) * (NB + 1);
        auto kern = cell_hist_pipe_kernel<InT, OutT, NB>;
        cudaError_t e = smem_at_least<cell_hist_pipe_kernel<InT, OutT, NB>>(smem);
        if (e != cudaSuccess) return cuda_fail(e);
        const int n_tx = ceil_div(ncx, kTI);
        const int n_tiles = n_tx * ceil_div(ncy, TJ);
        const int grid = n_tiles < 4 * sm_count() ? n_tiles : 4 * sm_count();
        const bool vec_out = reinterpret_cast<uintptr_t>(cells) % 16 == 0;
        return launch_pdl(kern, dim3(grid), dim3(kStreamThreads), smem, st, static_cast<const InT*>(ii), W, H, stride,
                          r, ncx, ncy, TJ, n_tx, n_tiles, static_cast<OutT*>(cells), vec_out);
    }
    const size_t smem = sizeof(uint32_t) * (size_t)(TJ + r) * (kTI + r) * (NB + 1);
    auto kern = cell_hist_stream_kernel<InT, OutT, NB>;
    cudaError_t e = smem_at_least<cell_hist_stream_kernel<InT, OutT, NB>>(smem);
    if (e != cudaSuccess) return cuda_fail(e);
    dim3 grid(ceil_div(ncx, kTI), ceil_div(ncy, TJ));
    return launch_pdl(kern, grid, dim3(kStreamThreads), smem, st, static_cast<const InT*>(ii), W, H, stride, r, ncx,
                      ncy, TJ, static_cast<OutT*>(cells));
}

template <typename InT, typename OutT>
hog_status launch_t(const void* ii, int W, int H, int nb, int cell, int stride, int ncx, int ncy, void* cells,
                    cudaStream_t st) {
    if ((nb == 8 || nb == 16) && cell % stride == 0 && cell / stride <= 8) {
        const int TJ = stream_rows(ncx, ncy);
        const int r = cell / stride;
        if (TJ > 1)
            return nb == 8 ? launch_stream<InT, OutT, 8>(ii, W, H, stride, r, ncx, ncy, TJ, cells, st)
                           : launch_stream<InT, OutT, 16>(ii, W, H, stride, r, ncx, ncy, TJ, cells, st);
    }
    dim3 grid(ceil_div(ncx, 128), ncy);
    const InT* src = static_cast<const InT*>(ii);
    OutT* dst = static_cast<OutT*>(cells);
    if (nb == 8)
        return launch_pdl(cell_hist_kernel<InT, OutT, 8>, grid, dim3(128), 0, st, src, W, H, nb, cell, stride, ncx,
                          ncy, dst);
    if (nb == 16)
        return launch_pdl(cell_hist_kernel<InT, OutT, 16>, grid, dim3(128), 0, st, src, W, H, nb, cell, stride, ncx,
                          ncy, dst);
    return launch_pdl(cell_hist_kernel<InT, OutT, 0>, grid, dim3(128), 0, st, src, W, H, nb, cell, stride, ncx, ncy,
                      dst);
}

}  // namespace

hog_status launch_cell_hist(const void* ii, int W, int H, int n_bins, int ii_dtype, int cell, int stride,
                            int cell_dtype, void* cells, cudaStream_t st) {
    const int ncx = W < cell ? 0 : (W - cell) / stride + 1;
    const int ncy = H < cell ? 0 : (H - cell) / stride + 1;
    if (ncx == 0 || ncy == 0) return HOG_OK;
    if (ii_dtype == HOG_U16) {
        if (cell_dtype == HOG_BF16) return launch_t<uint16_t, uint16_t>(ii, W, H, n_bins, cell, stride, ncx, ncy, cells, st);
        if (cell_dtype == HOG_F32) return launch_t<uint16_t, float>(ii, W, H, n_bins, cell, stride, ncx, ncy, cells, st);
        return launch_t<uint16_t, int32_t>(ii, W, H, n_bins, cell, stride, ncx, ncy, cells, st);
    }
    if (cell_dtype == HOG_BF16) return launch_t<int32_t, uint16_t>(ii, W, H, n_bins, cell, stride, ncx, ncy, cells, st);
    if (cell_dtype == HOG_F32) return launch_t<int32_t, float>(ii, W, H, n_bins, cell, stride, ncx, ncy, cells, st);
    return launch_t<int32_t, int32_t>(ii, W, H, n_bins, cell, stride, ncx, ncy, cells, st);
}

}  // namespace fasthog
