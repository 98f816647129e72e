// block_norm.cu -- overlapping blocks of 2 x 2 cells, L2-normalised (the
// region feature built from four overlapped sub-areas, Section 3, Fig. 4's
// caption; blocks of 2 x 2 cells at a stride of one cell, each divided by
// sqrt(|v|^2 + eps^2)).  One warp per block: the 4 n_bins values are spread
// over the lanes, squared and summed with a shuffle reduction, then written
// back divided by the norm with coalesced stores.  Counts and their squares
// are integers below 2^24, so the sum of squares is exact in FP32; the
// square root and the division are correctly rounded.
#include <cmath>

#include "internal.cuh"

namespace fasthog {

namespace {

constexpr int kWarps = 8;

template <typename CellT>
__device__ __forceinline__ float cell_value(const CellT* p);
template <>
__device__ __forceinline__ float cell_value<int32_t>(const int32_t* p) {
    return (float)__ldg(p);
}
template <>
__device__ __forceinline__ float cell_value<float>(const float* p) {
    return __ldg(p);
}
template <>
__device__ __forceinline__ float cell_value<uint16_t>(const uint16_t* p) {
    return __uint_as_float((uint32_t)__ldg(p) << 16);  // bf16 -> f32
}

template <typename CellT>
__global__ void __launch_bounds__(kWarps * 32)
    block_norm_kernel(const CellT* __restrict__ cells, int ncx, int nb, int r, int nbx, long n_blocks, float eps2,
                      float* __restrict__ blocks) {
    pdl_wait();
    pdl_trigger();
    const long blk = (long)blockIdx.x * kWarps + (threadIdx.x >> 5);
    if (blk >= n_blocks) return;
    const int lane = threadIdx.x & 31;
    const int j = (int)(blk / nbx), i = (int)(blk - (long)j * nbx);
    const int k_total = 4 * nb;  // <= 256: at most 8 values per lane
    float v[8];
    float ss = 0.f;
#pragma unroll
    for (int t = 0; t < 8; ++t) {
        const int k = lane + 32 * t;
        v[t] = 0.f;
        if (k < k_total) {
            const int q = k / nb, b = k - q * nb;
            const int ci = i + (q & 1) * r, cj = j + (q >> 1) * r;
            v[t] = cell_value<CellT>(cells + ((size_t)cj * ncx + ci) * nb + b);
            ss += v[t] * v[t];
        }
    }
#pragma unroll
    for (int d = 16; d > 0; d >>= 1) ss += __shfl_xor_sync(0xffffffffu, ss, d);
    const float norm = sqrtf(ss + eps2);
    float* out = blocks + (size_t)blk * k_total;
#pragma unroll
    for (int t = 0; t < 8; ++t) {
        const int k = lane + 32 * t;
        if (k < k_total) out[k] = norm > 0.f ? v[t] / norm : 0.f;
    }
}

}  // namespace

hog_status launch_block_norm(const void* cells, int cell_dtype, int ncx, int ncy, int nb, int r, float eps,
                             float* blocks, cudaStream_t st) {
    const int nbx = ncx - r, nby = ncy - r;
    if (nbx <= 0 || nby <= 0) return HOG_OK;
    const long n = (long)nbx * nby;
    const dim3 grid((unsigned)((n + kWarps - 1) / kWarps));
    const float eps2 = eps * eps;
    if (cell_dtype == HOG_BF16)
        return launch_pdl(block_norm_kernel<uint16_t>, grid, dim3(kWarps * 32), 0, st,
                          static_cast<const uint16_t*>(cells), ncx, nb, r, nbx, n, eps2, blocks);
    if (cell_dtype == HOG_F32)
        return launch_pdl(block_norm_kernel<float>, grid, dim3(kWarps * 32), 0, st, static_cast<const float*>(cells),
                          ncx, nb, r, nbx, n, eps2, blocks);
    return launch_pdl(block_norm_kernel<int32_t>, grid, dim3(kWarps * 32), 0, st, static_cast<const int32_t*>(cells),
                      ncx, nb, r, nbx, n, eps2, blocks);
}

}  // namespace fasthog
