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
    pdl_trigger();
    pdl_wait();
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

template <typename InT, typename OutT>
hog_status launch_t(const void* ii, int W, int H, int nb, int cell, int stride, int ncx, int ncy, void* cells,
                    cudaStream_t st) {
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
