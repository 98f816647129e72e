// cell_hist.cu -- area histograms from four integral-image corners
// (paper Section 3.3, Eq. 6; Section 3.1, Eq. 3 applied per bin).
//
// One thread per cell.  For each bin the thread reads the four corners
//   ii(x1, y1), ii(x0-1, y0-1), ii(x1, y0-1), ii(x0-1, y1)
// (an index of -1 reads 0) and writes the cell's histogram contiguously,
// bin innermost, as int32, f32 or bf16 (counts <= cell^2 are small integers).
//
// Fast path (8 or 16 bins): a CTA takes up to 128 consecutive cells of one
// cell row.  All of them read the same two ii rows (y0 - 1 and y0 + cell - 1),
// so the CTA first copies the stretch of those rows it needs, every bin, into
// shared memory with 16-byte vector loads, then each thread forms its cell
// from shared memory.  Generic path: the corners straight from global memory.
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

// Staged fast path.  rows: [2][NB][span] elements of the ii rows y0-1 (row 0)
// and y0+cell-1 (row 1), columns [cb, cb + span).
template <typename InT, typename OutT, int NB>
__global__ void __launch_bounds__(128)
    cell_hist_staged_kernel(const InT* __restrict__ ii, int W, int H, int cell, int stride, int ncx, int cpc, int span,
                            bool vec, OutT* __restrict__ cells) {
    constexpr int VEC = 16 / (int)sizeof(InT);  // elements per 16-byte load
    extern __shared__ __align__(16) uint8_t smem_raw[];
    InT* rows = reinterpret_cast<InT*>(smem_raw);
    const int tid = threadIdx.x;
    const int j = blockIdx.y;
    const int i0 = blockIdx.x * cpc;
    const int y0 = j * stride, y1 = y0 + cell - 1;
    const int cb = max(0, i0 * stride - 1) & ~(VEC - 1);
    const size_t plane = (size_t)W * H;
    const int nv = span / VEC;
    for (int idx = tid; idx < 2 * NB * nv; idx += blockDim.x) {
        const int v = idx % nv, t = idx / nv;
        const int b = t % NB, r = t / NB;
        const int y = r == 0 ? y0 - 1 : y1;
        const int x = cb + v * VEC;
        InT* dst = rows + (size_t)(r * NB + b) * span + v * VEC;
        if (y < 0) continue;  // row y0 - 1 of the first cell row is never read
        const InT* src = ii + (size_t)b * plane + (size_t)y * W + x;
        if (vec && x + VEC <= W) {
            *reinterpret_cast<uint4*>(dst) = __ldg(reinterpret_cast<const uint4*>(src));
        } else {
#pragma unroll
            for (int e = 0; e < VEC; ++e) dst[e] = x + e < W ? __ldg(src + e) : InT(0);
        }
    }
    __syncthreads();
    const int i = i0 + tid;
    if (tid >= cpc || i >= ncx) return;
    const int x0 = i * stride, x1 = x0 + cell - 1;
    const bool hx = x0 > 0, hy = y0 > 0;
    const InT* r0 = rows;
    const InT* r1 = rows + (size_t)NB * span;
    uint32_t v[NB];
#pragma unroll
    for (int b = 0; b < NB; ++b) {
        uint32_t a = (uint32_t)r1[b * span + x1 - cb];
        if (hx) a -= (uint32_t)r1[b * span + x0 - 1 - cb];
        if (hy) a -= (uint32_t)r0[b * span + x1 - cb];
        if (hx && hy) a += (uint32_t)r0[b * span + x0 - 1 - cb];
        if (sizeof(InT) == 2) a &= 0xFFFFu;
        v[b] = a;
    }
    OutT* out = cells + ((size_t)j * ncx + i) * NB;
#pragma unroll
    for (int b = 0; b < NB; ++b) out[b] = count_as<OutT>(v[b]);
}

template <typename InT, typename OutT, int NB>
bool launch_staged(const void* ii, int W, int H, int cell, int stride, int ncx, int ncy, void* cells, cudaStream_t st,
                   hog_status* status) {
    constexpr int VEC = 16 / (int)sizeof(InT);
    int cpc = 128, span = 0;
    size_t smem = 0;
    for (; cpc >= 32; cpc /= 2) {
        span = ((stride * (cpc - 1) + cell + 1 + 2 * VEC) + VEC - 1) / VEC * VEC;
        smem = (size_t)2 * NB * span * sizeof(InT);
        if (smem <= 96 * 1024) break;
    }
    if (cpc < 32) return false;
    auto k = cell_hist_staged_kernel<InT, OutT, NB>;
    cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) {
        *status = cuda_fail(e);
        return true;
    }
    const bool vec = reinterpret_cast<uintptr_t>(ii) % 16 == 0 && ((size_t)W * sizeof(InT)) % 16 == 0;
    dim3 grid(ceil_div(ncx, cpc), ncy);
    k<<<grid, 128, smem, st>>>(static_cast<const InT*>(ii), W, H, cell, stride, ncx, cpc, span, vec,
                               static_cast<OutT*>(cells));
    *status = check_launch();
    return true;
}

template <typename InT, typename OutT>
hog_status launch_t(const void* ii, int W, int H, int nb, int cell, int stride, int ncx, int ncy, void* cells,
                    cudaStream_t st) {
    hog_status s = HOG_OK;
    if (nb == 8 && launch_staged<InT, OutT, 8>(ii, W, H, cell, stride, ncx, ncy, cells, st, &s)) return s;
    if (nb == 16 && launch_staged<InT, OutT, 16>(ii, W, H, cell, stride, ncx, ncy, cells, st, &s)) return s;
    dim3 grid(ceil_div(ncx, 128), ncy);
    const InT* src = static_cast<const InT*>(ii);
    OutT* dst = static_cast<OutT*>(cells);
    if (nb == 8)
        cell_hist_kernel<InT, OutT, 8><<<grid, 128, 0, st>>>(src, W, H, nb, cell, stride, ncx, ncy, dst);
    else if (nb == 16)
        cell_hist_kernel<InT, OutT, 16><<<grid, 128, 0, st>>>(src, W, H, nb, cell, stride, ncx, ncy, dst);
    else
        cell_hist_kernel<InT, OutT, 0><<<grid, 128, 0, st>>>(src, W, H, nb, cell, stride, ncx, ncy, dst);
    return check_launch();
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
