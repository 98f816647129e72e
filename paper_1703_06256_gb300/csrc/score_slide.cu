// score_slide.cu -- window score on CUDA cores, FP32 arithmetic, for the
// window of 8 x 16 cells with 8 bins per cell (the paper's linear score,
// Sections 1 and 4, at the workloads' shape).
//
//   S[py][px] = bias + sum_{j<16} sum_{i<8} sum_{b<8} w[j][i][b] * C[py + j r][px + i r][b]
//
// Sixteen lanes share a window.  Lane j keeps filter row j (8 cells x 8 bins
// = 64 weights) in registers and forms that row's partial sum; a 4-step
// xor-shuffle adds the sixteen partials.  Each half-warp then slides along
// its scan row: the windows px, px + r, px + 2r, ... reuse 7 of their 8
// cells, so a lane keeps the last 8 cells of its cell row in a register ring
// and loads a single new cell (8 values) per window.  The ring index
// (t + i) mod 8 is a compile-time constant because the loop over windows is
// unrolled by 8.  The two half-warps take the two residues px mod r = 0, 1
// (for r = 2) of the same segment, so they read interleaved cells of the
// same rows.  Each lane accumulates in eight independent partial sums (one
// per cell) to keep the FMA pipe busy.
//
// Work item ("sequence"): output row py, residue rho, segment s of T windows
// px = rho + r * (s*T + t), t < T.
#include <type_traits>

#include "internal.cuh"

namespace fasthog {

namespace {

constexpr int kNB = 8, kCX = 8, kCY = 16;
constexpr int kThreads = 128;

template <typename CellT>
__device__ __forceinline__ void load_cell(const CellT* __restrict__ p, bool ok, float (&c)[kNB]);

template <>
__device__ __forceinline__ void load_cell<float>(const float* __restrict__ p, bool ok, float (&c)[kNB]) {
    float4 a = make_float4(0.f, 0.f, 0.f, 0.f), b = a;
    if (ok) {
        a = __ldg(reinterpret_cast<const float4*>(p));
        b = __ldg(reinterpret_cast<const float4*>(p) + 1);
    }
    c[0] = a.x; c[1] = a.y; c[2] = a.z; c[3] = a.w;
    c[4] = b.x; c[5] = b.y; c[6] = b.z; c[7] = b.w;
}

template <>
__device__ __forceinline__ void load_cell<int32_t>(const int32_t* __restrict__ p, bool ok, float (&c)[kNB]) {
    int4 a = make_int4(0, 0, 0, 0), b = a;
    if (ok) {
        a = __ldg(reinterpret_cast<const int4*>(p));
        b = __ldg(reinterpret_cast<const int4*>(p) + 1);
    }
    c[0] = (float)a.x; c[1] = (float)a.y; c[2] = (float)a.z; c[3] = (float)a.w;
    c[4] = (float)b.x; c[5] = (float)b.y; c[6] = (float)b.z; c[7] = (float)b.w;
}

template <>
__device__ __forceinline__ void load_cell<uint16_t>(const uint16_t* __restrict__ p, bool ok, float (&c)[kNB]) {
    uint4 a = make_uint4(0, 0, 0, 0);
    if (ok) a = __ldg(reinterpret_cast<const uint4*>(p));
    const uint32_t v[4] = {a.x, a.y, a.z, a.w};
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        c[2 * k] = __uint_as_float(v[k] << 16);
        c[2 * k + 1] = __uint_as_float(v[k] & 0xFFFF0000u);
    }
}

template <typename WT>
__device__ __forceinline__ float wval(const WT* w, int k);
template <>
__device__ __forceinline__ float wval<float>(const float* w, int k) { return __ldg(w + k); }
template <>
__device__ __forceinline__ float wval<uint16_t>(const uint16_t* w, int k) { return bf16_to_f32(__ldg(w + k)); }
template <>
__device__ __forceinline__ float wval<int8_t>(const int8_t* w, int k) { return (float)__ldg(w + k); }

// Shared-memory block of cells for one work item: cell rows py0 .. py0 + RB - 1 + 15 r
// (RB = 8 / r output rows) and the cell columns of one segment of T windows
// for all r residues.  Rows are stored grouped by residue class (row % r), so
// the 16 rows a half-warp reads (py + j r, j < 16) are consecutive; the row
// stride is an odd number of 16-byte slots, so 8 consecutive rows fall in 8
// different bank groups.
struct SlideGeom {
    int r, rb, T, rows, cols, rpc, stride4;  // stride4: float4 slots per smem row
    __host__ __device__ SlideGeom(int r_, int T_) : r(r_), rb(8 / r_), T(T_) {
        rows = rb + (kCY - 1) * r;
        cols = r * (T + kCX - 1);
        rpc = (rows + r - 1) / r;
        stride4 = 2 * cols + 1;
    }
    __host__ __device__ size_t smem_bytes() const { return (size_t)r * rpc * stride4 * 16; }
    __host__ __device__ int ridx(int row) const { return (row % r) * rpc + row / r; }
};

template <typename CellT, typename WT, typename OutT>
__global__ void __launch_bounds__(kThreads, 3)
    score_slide_kernel(const CellT* __restrict__ cells, int ncx, int ncy, int r, int T, const WT* __restrict__ w,
                       float bias, int nx, int ny, int S, int n_items, OutT* __restrict__ scores) {
    extern __shared__ __align__(16) float4 blk[];
    const SlideGeom G(r, T);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int j = lane & 15;
    const int seq = warp * 2 + (lane >> 4);  // 0..7: (output row offset, residue)
    const int dpy = seq / r, rho = seq % r;
    float wr[kCX][kNB];
#pragma unroll
    for (int i = 0; i < kCX; ++i)
#pragma unroll
        for (int b = 0; b < kNB; ++b) wr[i][b] = wval<WT>(w, (j * kCX + i) * kNB + b);
    pdl_trigger();  // tail of the path: the successor is small, launch it early
    pdl_wait();  // the weights above are inputs of the call, not of a predecessor

    for (int item = blockIdx.x; item < n_items; item += gridDim.x) {
        const int s = item % S, rblk = item / S;
        const int py0 = rblk * G.rb, u0 = s * T;
        const int cx0 = r * u0;  // first cell column of the block
        __syncthreads();          // the previous item's reads are done
        for (int idx = threadIdx.x; idx < G.rows * G.cols; idx += kThreads) {
            const int row = idx / G.cols, col = idx - row * G.cols;
            const int gy = py0 + row, gx = cx0 + col;
            float c[kNB];
            load_cell<CellT>(cells + ((size_t)gy * ncx + gx) * kNB, gy < ncy && gx < ncx, c);
            float4* d = blk + (size_t)G.ridx(row) * G.stride4 + 2 * col;
            d[0] = make_float4(c[0], c[1], c[2], c[3]);
            d[1] = make_float4(c[4], c[5], c[6], c[7]);
        }
        __syncthreads();
        const int py = py0 + dpy;
        const bool seq_ok = py < ny;
        // smem row of filter row j for this sequence, and the first cell column
        const float4* rowp = blk + (size_t)G.ridx(dpy + j * r) * G.stride4 + 2 * rho;
        float ring[kCX][kNB];
#pragma unroll
        for (int i = 0; i < kCX - 1; ++i) {
            const float4 a = rowp[2 * r * i], b2 = rowp[2 * r * i + 1];
            ring[i][0] = a.x; ring[i][1] = a.y; ring[i][2] = a.z; ring[i][3] = a.w;
            ring[i][4] = b2.x; ring[i][5] = b2.y; ring[i][6] = b2.z; ring[i][7] = b2.w;
        }
        for (int blk8 = 0; blk8 < T; blk8 += kCX) {
#pragma unroll
            for (int t = 0; t < kCX; ++t) {
                const int tt = blk8 + t;
                {
                    const int slot = (t + kCX - 1) % kCX;
                    const float4 a = rowp[2 * r * (tt + kCX - 1)], b2 = rowp[2 * r * (tt + kCX - 1) + 1];
                    ring[slot][0] = a.x; ring[slot][1] = a.y; ring[slot][2] = a.z; ring[slot][3] = a.w;
                    ring[slot][4] = b2.x; ring[slot][5] = b2.y; ring[slot][6] = b2.z; ring[slot][7] = b2.w;
                }
                float part[kCX];
#pragma unroll
                for (int i = 0; i < kCX; ++i) {
                    const float* c = ring[(t + i) % kCX];
                    float acc = wr[i][0] * c[0];
#pragma unroll
                    for (int b = 1; b < kNB; ++b) acc = fmaf(wr[i][b], c[b], acc);
                    part[i] = acc;
                }
                float p = ((part[0] + part[1]) + (part[2] + part[3])) + ((part[4] + part[5]) + (part[6] + part[7]));
#pragma unroll
                for (int off = 8; off > 0; off >>= 1) p += __shfl_xor_sync(0xffffffffu, p, off);
                const int px = rho + r * (u0 + tt);
                if (j == 0 && seq_ok && px < nx) {
                    const float sc = p + bias;
                    if constexpr (std::is_same<OutT, int32_t>::value) {
                        scores[(size_t)py * nx + px] = __float2int_rn(sc);  // exact: an integer below 2^24
                    } else {
                        scores[(size_t)py * nx + px] = sc;
                    }
                }
            }
        }
    }
}

template <typename CellT, typename WT, typename OutT>
hog_status launch_t(const void* cells, int ncx, int ncy, int r, const void* w, float bias, void* scores,
                    cudaStream_t st) {
    const int nx = ncx - (kCX - 1) * r, ny = ncy - (kCY - 1) * r;
    if (nx <= 0 || ny <= 0) return HOG_OK;
    const int tuned = tune_get(HOG_TUNE_SLIDE_WINDOWS);
    const int T = tuned > 0 ? tuned : (r <= 2 ? 16 : 8);  // windows per sequence
    const SlideGeom G(r, T);
    const int per_class = (nx + r - 1) / r;
    const int S = (per_class + T - 1) / T;
    const int n_items = ((ny + G.rb - 1) / G.rb) * S;
    const size_t smem = G.smem_bytes();
    auto kern = score_slide_kernel<CellT, WT, OutT>;
    cudaError_t e = smem_at_least<score_slide_kernel<CellT, WT, OutT>>(smem);
    if (e != cudaSuccess) return cuda_fail(e);
    const int per_sm = smem <= 70 * 1024 ? 3 : (smem <= 110 * 1024 ? 2 : 1);
    const int cap = per_sm * sm_count();
    const int grid = n_items < cap ? n_items : cap;
    return launch_pdl(kern, dim3(grid), dim3(kThreads), smem, st, static_cast<const CellT*>(cells), ncx, ncy, r, T,
                      static_cast<const WT*>(w), bias, nx, ny, S, n_items, static_cast<OutT*>(scores));
}

template <typename CellT>
hog_status by_weight(const void* cells, int ncx, int ncy, int r, const void* w, int w_dtype, float bias, void* scores,
                     cudaStream_t st) {
    switch (w_dtype) {
        case HOG_F32: return launch_t<CellT, float, float>(cells, ncx, ncy, r, w, bias, scores, st);
        case HOG_BF16: return launch_t<CellT, uint16_t, float>(cells, ncx, ncy, r, w, bias, scores, st);
        case HOG_I8: return launch_t<CellT, int8_t, int32_t>(cells, ncx, ncy, r, w, bias, scores, st);
        default: return HOG_ERR_ARG;
    }
}

}  // namespace

bool score_slide_supported(const void* cells, int n_bins, int cells_x, int cells_y, int r) {
    return n_bins == kNB && cells_x == kCX && cells_y == kCY && reinterpret_cast<uintptr_t>(cells) % 16 == 0 &&
           (r == 1 || r == 2 || r == 4);
}

hog_status launch_score_slide(const void* cells, int cell_dtype, int ncx, int ncy, int r, const void* w, int w_dtype,
                              float bias, void* scores, cudaStream_t st) {
    if (cell_dtype == HOG_F32) return by_weight<float>(cells, ncx, ncy, r, w, w_dtype, bias, scores, st);
    if (cell_dtype == HOG_BF16) return by_weight<uint16_t>(cells, ncx, ncy, r, w, w_dtype, bias, scores, st);
    return by_weight<int32_t>(cells, ncx, ncy, r, w, w_dtype, bias, scores, st);
}

}  // namespace fasthog
