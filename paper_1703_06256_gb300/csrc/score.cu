// score.cu -- window score on CUDA cores (paper Sections 1 and 4: a linear
// score, the inner product of the window feature with a weight vector, at
// every scan position).
//
//   S[py][px] = bias + sum_{cy, cx, b} w[(cy*cells_x + cx)*nb + b] * C[py + cy*r][px + cx*r][b]
//
// One thread per window; a CTA owns 32 x TY windows, TY = 8, 4, 2 or 1: the
// tallest tile whose staged region fits in shared memory.  It stages the cell-map
// region those windows touch, converted to float, in shared memory as
// [row][bin/4][column] float4 (consecutive threads read consecutive
// float4s: no bank conflicts), and the weights as float4s that every thread
// of a warp reads at the same address (broadcast).  FP32 FMAs into four
// partial sums, added at the end.  Weights may be f32, bf16 or int8; with
// int8 weights every product and partial sum is an integer below 2^24, so
// the float arithmetic is exact and the score is returned as int32.
//
// When even a one-row tile would not fit (strides well below the cell size,
// very long features), the kernel reads the cells from global memory instead.
#include <type_traits>

#include "internal.cuh"

namespace fasthog {

namespace {

constexpr int kTX = 32;
constexpr int kSmemLimit = 200 * 1024;

struct ScoreGeom {
    int nb4;  // bins padded to a multiple of 4, in float4 units
    int rw, rh;
    size_t cells_bytes, w_bytes;
};

ScoreGeom geom(int nb, int cells_x, int cells_y, int r, int ty) {
    ScoreGeom g;
    g.nb4 = (nb + 3) / 4;
    g.rw = kTX + (cells_x - 1) * r;
    g.rh = ty + (cells_y - 1) * r;
    g.cells_bytes = (size_t)g.rh * g.nb4 * g.rw * 16;
    g.w_bytes = (size_t)cells_x * cells_y * g.nb4 * 16;
    return g;
}

template <typename CellT>
__device__ __forceinline__ float cell_val(const CellT* c, size_t idx);
template <>
__device__ __forceinline__ float cell_val<int32_t>(const int32_t* c, size_t idx) {
    return (float)__ldg(c + idx);
}
template <>
__device__ __forceinline__ float cell_val<float>(const float* c, size_t idx) {
    return __ldg(c + idx);
}
template <>
__device__ __forceinline__ float cell_val<uint16_t>(const uint16_t* c, size_t idx) {
    return bf16_to_f32(__ldg(c + idx));
}

template <typename WT>
__device__ __forceinline__ float weight_val(const WT* w, int k);
template <>
__device__ __forceinline__ float weight_val<float>(const float* w, int k) {
    return __ldg(w + k);
}
template <>
__device__ __forceinline__ float weight_val<uint16_t>(const uint16_t* w, int k) {
    return bf16_to_f32(__ldg(w + k));
}
template <>
__device__ __forceinline__ float weight_val<int8_t>(const int8_t* w, int k) {
    return (float)__ldg(w + k);
}

template <typename CellT, typename WT, typename OutT, bool SMEM, int TY>
__global__ void __launch_bounds__(kTX* TY)
    score_kernel(const CellT* __restrict__ cells, int ncx, int ncy, int nb, int cells_x, int cells_y, int r,
                 const WT* __restrict__ w, float bias, int nx, int ny, OutT* __restrict__ scores) {
    extern __shared__ __align__(16) float4 smem4[];
    const int nb4 = (nb + 3) / 4;
    const int rw = kTX + (cells_x - 1) * r;
    const int rh = TY + (cells_y - 1) * r;
    const int K4 = cells_x * cells_y * nb4;
    float4* w_s = smem4;          // [cells_y*cells_x][nb4]
    float4* c_s = smem4 + K4;     // [rh][nb4][rw]
    const int tid = threadIdx.y * kTX + threadIdx.x;
    const int px0 = blockIdx.x * kTX, py0 = blockIdx.y * TY;
    pdl_trigger();  // tail of the path: the successor is small, launch it early
    pdl_wait();

    // weights, padded per cell to nb4 float4s
    for (int i = tid; i < K4 * 4; i += kTX * TY) {
        const int cellk = i / (nb4 * 4), b = i - cellk * nb4 * 4;
        reinterpret_cast<float*>(w_s)[i] = b < nb ? weight_val<WT>(w, cellk * nb + b) : 0.f;
    }
    if (SMEM) {
        for (int i = tid; i < rh * nb4 * rw * 4; i += kTX * TY) {
            // i enumerates [row][b4][col][lane]
            const int lanei = i & 3;
            const int t = i >> 2;
            const int col = t % rw;
            const int t2 = t / rw;
            const int b4 = t2 % nb4;
            const int row = t2 / nb4;
            const int b = b4 * 4 + lanei;
            const int gx = px0 + col, gy = py0 + row;
            float v = 0.f;
            if (b < nb && gx < ncx && gy < ncy) v = cell_val<CellT>(cells, ((size_t)gy * ncx + gx) * nb + b);
            reinterpret_cast<float*>(c_s)[i] = v;
        }
    }
    __syncthreads();

    const int px = px0 + threadIdx.x, py = py0 + threadIdx.y;
    if (px >= nx || py >= ny) return;
    float a0 = 0.f, a1 = 0.f, a2 = 0.f, a3 = 0.f;
    for (int cy = 0; cy < cells_y; ++cy) {
        for (int cx = 0; cx < cells_x; ++cx) {
            const float4* wk = w_s + (cy * cells_x + cx) * nb4;
            if (SMEM) {
                const int row = threadIdx.y + cy * r, col = threadIdx.x + cx * r;
                const float4* ck = c_s + (size_t)row * nb4 * rw + col;
                for (int b4 = 0; b4 < nb4; ++b4) {
                    const float4 c = ck[(size_t)b4 * rw];
                    const float4 ww = wk[b4];
                    a0 = fmaf(ww.x, c.x, a0);
                    a1 = fmaf(ww.y, c.y, a1);
                    a2 = fmaf(ww.z, c.z, a2);
                    a3 = fmaf(ww.w, c.w, a3);
                }
            } else {
                const size_t base = ((size_t)(py + cy * r) * ncx + (px + cx * r)) * nb;
                for (int b4 = 0; b4 < nb4; ++b4) {
                    const float4 ww = wk[b4];
                    const int b = b4 * 4;
                    a0 = fmaf(ww.x, cell_val<CellT>(cells, base + b), a0);
                    if (b + 1 < nb) a1 = fmaf(ww.y, cell_val<CellT>(cells, base + b + 1), a1);
                    if (b + 2 < nb) a2 = fmaf(ww.z, cell_val<CellT>(cells, base + b + 2), a2);
                    if (b + 3 < nb) a3 = fmaf(ww.w, cell_val<CellT>(cells, base + b + 3), a3);
                }
            }
        }
    }
    const float s = ((a0 + a1) + (a2 + a3)) + bias;
    if constexpr (std::is_same<OutT, int32_t>::value) {
        scores[(size_t)py * nx + px] = __float2int_rn(s);  // exact: s is an integer below 2^24
    } else {
        scores[(size_t)py * nx + px] = s;
    }
}

template <typename CellT, typename WT, typename OutT, bool SMEM, int TY>
hog_status launch_ty(const void* cells, int ncx, int ncy, int nb, int cells_x, int cells_y, int r, const void* w,
                     float bias, void* scores, int nx, int ny, size_t smem, cudaStream_t st) {
    auto k = score_kernel<CellT, WT, OutT, SMEM, TY>;
    cudaError_t e = smem_at_least<score_kernel<CellT, WT, OutT, SMEM, TY>>(smem);
    if (e != cudaSuccess) return cuda_fail(e);
    dim3 grid(ceil_div(nx, kTX), ceil_div(ny, TY)), block(kTX, TY);
    return launch_pdl(k, grid, block, smem, st, static_cast<const CellT*>(cells), ncx, ncy, nb, cells_x, cells_y, r,
                      static_cast<const WT*>(w), bias, nx, ny, static_cast<OutT*>(scores));
}

template <typename CellT, typename WT, typename OutT>
hog_status launch_t(const void* cells, int ncx, int ncy, int nb, int cells_x, int cells_y, int r, const void* w,
                    float bias, void* scores, cudaStream_t st) {
    const int nx = ncx - (cells_x - 1) * r, ny = ncy - (cells_y - 1) * r;
    if (nx <= 0 || ny <= 0) return HOG_OK;
    for (int ty : {8, 4, 2, 1}) {
        const ScoreGeom g = geom(nb, cells_x, cells_y, r, ty);
        const size_t smem = g.w_bytes + g.cells_bytes;
        if (smem > (size_t)kSmemLimit) continue;
        switch (ty) {
            case 8: return launch_ty<CellT, WT, OutT, true, 8>(cells, ncx, ncy, nb, cells_x, cells_y, r, w, bias,
                                                               scores, nx, ny, smem, st);
            case 4: return launch_ty<CellT, WT, OutT, true, 4>(cells, ncx, ncy, nb, cells_x, cells_y, r, w, bias,
                                                               scores, nx, ny, smem, st);
            case 2: return launch_ty<CellT, WT, OutT, true, 2>(cells, ncx, ncy, nb, cells_x, cells_y, r, w, bias,
                                                               scores, nx, ny, smem, st);
            default: return launch_ty<CellT, WT, OutT, true, 1>(cells, ncx, ncy, nb, cells_x, cells_y, r, w, bias,
                                                                scores, nx, ny, smem, st);
        }
    }
    const ScoreGeom g = geom(nb, cells_x, cells_y, r, 8);
    if (g.w_bytes > (size_t)kSmemLimit) return HOG_ERR_UNSUPPORTED;
    return launch_ty<CellT, WT, OutT, false, 8>(cells, ncx, ncy, nb, cells_x, cells_y, r, w, bias, scores, nx, ny,
                                                g.w_bytes, st);
}

template <typename CellT>
hog_status by_weight(const void* cells, int ncx, int ncy, int nb, int cells_x, int cells_y, int r, const void* w,
                     int w_dtype, float bias, void* scores, cudaStream_t st) {
    switch (w_dtype) {
        case HOG_F32:
            return launch_t<CellT, float, float>(cells, ncx, ncy, nb, cells_x, cells_y, r, w, bias, scores, st);
        case HOG_BF16:
            return launch_t<CellT, uint16_t, float>(cells, ncx, ncy, nb, cells_x, cells_y, r, w, bias, scores, st);
        case HOG_I8:
            return launch_t<CellT, int8_t, int32_t>(cells, ncx, ncy, nb, cells_x, cells_y, r, w, bias, scores, st);
        default:
            return HOG_ERR_ARG;
    }
}

}  // namespace

hog_status launch_score_cuda_cores(const void* cells, int cell_dtype, int ncx, int ncy, int n_bins, int cells_x,
                                   int cells_y, int r, const void* w, int w_dtype, float bias, void* scores,
                                   cudaStream_t st) {
    if (cell_dtype == HOG_BF16)
        return by_weight<uint16_t>(cells, ncx, ncy, n_bins, cells_x, cells_y, r, w, w_dtype, bias, scores, st);
    if (cell_dtype == HOG_F32)
        return by_weight<float>(cells, ncx, ncy, n_bins, cells_x, cells_y, r, w, w_dtype, bias, scores, st);
    return by_weight<int32_t>(cells, ncx, ncy, n_bins, cells_x, cells_y, r, w, w_dtype, bias, scores, st);
}

}  // namespace fasthog
