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

template <typename CellT, typename WT, typename OutT>
__global__ void __launch_bounds__(kThreads, 3)
    score_slide_kernel(const CellT* __restrict__ cells, int ncx, int r, const WT* __restrict__ w, float bias, int nx,
                       int ny, int T, int S, long Q, OutT* __restrict__ scores) {
    const int lane = threadIdx.x & 31;
    const int j = lane & 15, half = lane >> 4;
    float wr[kCX][kNB];
#pragma unroll
    for (int i = 0; i < kCX; ++i)
#pragma unroll
        for (int b = 0; b < kNB; ++b) wr[i][b] = wval<WT>(w, (j * kCX + i) * kNB + b);

    const long warps_total = (long)gridDim.x * (kThreads / 32);
    const long warp0 = (long)blockIdx.x * (kThreads / 32) + (threadIdx.x >> 5);
    for (long pair = warp0; 2 * pair < Q; pair += warps_total) {
        const long q = 2 * pair + half;
        const bool seq_ok = q < Q;
        // q = (py * S + s) * r + rho
        const long qq = seq_ok ? q : 0;
        const int rho = (int)(qq % r);
        const long t2 = qq / r;
        const int s = (int)(t2 % S);
        const int py = (int)(t2 / S);
        const int row = py + j * r;
        const CellT* rowp = cells + (size_t)row * ncx * kNB;
        const int u0 = s * T;
        float ring[kCX][kNB];
#pragma unroll
        for (int i = 0; i < kCX - 1; ++i) {
            const int pos = rho + r * (u0 + i);
            load_cell<CellT>(rowp + (size_t)pos * kNB, seq_ok && pos < ncx, ring[i]);
        }
        for (int blk = 0; blk < T; blk += kCX) {
#pragma unroll
            for (int t = 0; t < kCX; ++t) {
                const int u = u0 + blk + t;
                const int pos_new = rho + r * (u + kCX - 1);
                load_cell<CellT>(rowp + (size_t)pos_new * kNB, seq_ok && pos_new < ncx, ring[(t + kCX - 1) % kCX]);
                float part[kCX];
#pragma unroll
                for (int i = 0; i < kCX; ++i) {
                    const float* c = ring[(t + i) % kCX];
                    float a = wr[i][0] * c[0];
#pragma unroll
                    for (int b = 1; b < kNB; ++b) a = fmaf(wr[i][b], c[b], a);
                    part[i] = a;
                }
                float p = ((part[0] + part[1]) + (part[2] + part[3])) + ((part[4] + part[5]) + (part[6] + part[7]));
#pragma unroll
                for (int off = 8; off > 0; off >>= 1) p += __shfl_xor_sync(0xffffffffu, p, off);
                const int px = rho + r * u;
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
    const int per_class = (nx + r - 1) / r;
    // segments of 16 windows when that still gives every SM several warps
    int T = 16;
    long Q = (long)ny * r * ((per_class + T - 1) / T);
    if (Q / 2 < 4L * sm_count() * 4) T = 8;
    const int S = (per_class + T - 1) / T;
    Q = (long)ny * r * S;
    const long warps = (Q + 1) / 2;
    const long blocks_needed = (warps + kThreads / 32 - 1) / (kThreads / 32);
    const long cap = 3L * sm_count() * 4;
    const int grid = (int)(blocks_needed < cap ? blocks_needed : cap);
    score_slide_kernel<CellT, WT, OutT><<<grid, kThreads, 0, st>>>(static_cast<const CellT*>(cells), ncx, r,
                                                                    static_cast<const WT*>(w), bias, nx, ny, T, S, Q,
                                                                    static_cast<OutT*>(scores));
    return check_launch();
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

bool score_slide_supported(const void* cells, int n_bins, int cells_x, int cells_y) {
    return n_bins == kNB && cells_x == kCX && cells_y == kCY && reinterpret_cast<uintptr_t>(cells) % 16 == 0;
}

hog_status launch_score_slide(const void* cells, int cell_dtype, int ncx, int ncy, int r, const void* w, int w_dtype,
                              float bias, void* scores, cudaStream_t st) {
    if (cell_dtype == HOG_F32) return by_weight<float>(cells, ncx, ncy, r, w, w_dtype, bias, scores, st);
    if (cell_dtype == HOG_BF16) return by_weight<uint16_t>(cells, ncx, ncy, r, w, w_dtype, bias, scores, st);
    return by_weight<int32_t>(cells, ncx, ncy, r, w, w_dtype, bias, scores, st);
}

}  // namespace fasthog
