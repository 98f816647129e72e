// detect_core.cuh -- the per-tile pieces of the detection step (threshold
// and ordered compaction, Sections 1 and 4), shared by the per-image kernels
// (detect.cu) and the batch kernels (detect_batch.cu).
#pragma once

#include <type_traits>

#include "internal.cuh"

namespace fasthog {
namespace detect {

constexpr int kThreads = 256;
constexpr int kPer = 8;
constexpr int kTile = kThreads * kPer;
constexpr int kDetWords = sizeof(hog_det) / 4;  // x, y, score, image, level
static_assert(sizeof(hog_det) == 20, "hog_det is five 32-bit words");

template <typename T>
__device__ __forceinline__ bool pass(T v, float thr_f, int thr_i);
template <>
__device__ __forceinline__ bool pass<float>(float v, float thr_f, int) {
    return v >= thr_f;
}
// Integer scores: v >= thr  <=>  v >= ceil(thr).  The caller clamps ceil(thr)
// into the int32 range; a threshold of 2^31 or more (thr_f) passes nothing.
template <>
__device__ __forceinline__ bool pass<int32_t>(int32_t v, float thr_f, int thr_i) {
    return v >= thr_i && thr_f < 2147483648.0f;
}

__device__ __forceinline__ int block_sum(int v, int* red) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int d = 16; d > 0; d >>= 1) v += __shfl_xor_sync(0xffffffffu, v, d);
    __syncthreads();
    if (lane == 0) red[warp] = v;
    __syncthreads();
    int t = 0;
#pragma unroll
    for (int w = 0; w < kThreads / 32; ++w) t += red[w];
    return t;
}

// Windows of tile `tile` (scores [tile * kTile, + kTile) of [0, n)) that pass.
template <typename T>
__device__ __forceinline__ int tile_count(const T* __restrict__ scores, long n, int tile, float thr_f, int thr_i,
                                          int* red) {
    const long base = (long)tile * kTile + (long)threadIdx.x * kPer;
    int c = 0;
#pragma unroll
    for (int e = 0; e < kPer; ++e) {
        const long i = base + e;
        if (i < n) c += pass<T>(__ldg(scores + i), thr_f, thr_i);
    }
    return block_sum(c, red);
}

// The scores of this thread in tile `tile` (kPer consecutive ones) and the
// bit mask of those that pass.
template <typename T>
__device__ __forceinline__ unsigned tile_load(const T* __restrict__ scores, long n, int tile, float thr_f, int thr_i,
                                              T (&v)[kPer]) {
    static_assert(sizeof(T) == 4 && kPer == 8, "two 16-byte loads per thread");
    const long base = (long)tile * kTile + (long)threadIdx.x * kPer;
    if (base + kPer <= n && (reinterpret_cast<uintptr_t>(scores + base) & 15) == 0) {
        // the thread's 8 scores as two 16-byte loads (a warp reads 1 KB in one go)
        const uint4 a = __ldg(reinterpret_cast<const uint4*>(scores + base));
        const uint4 b = __ldg(reinterpret_cast<const uint4*>(scores + base) + 1);
        const uint32_t w[8] = {a.x, a.y, a.z, a.w, b.x, b.y, b.z, b.w};
#pragma unroll
        for (int e = 0; e < kPer; ++e) {
            if constexpr (std::is_same<T, float>::value) {
                v[e] = __uint_as_float(w[e]);
            } else {
                v[e] = (T)w[e];
            }
        }
        unsigned flags = 0;
#pragma unroll
        for (int e = 0; e < kPer; ++e)
            if (pass<T>(v[e], thr_f, thr_i)) flags |= 1u << e;
        return flags;
    }
    unsigned flags = 0;
#pragma unroll
    for (int e = 0; e < kPer; ++e) {
        const long i = base + e;
        v[e] = i < n ? __ldg(scores + i) : T(0);
        if (i < n && pass<T>(v[e], thr_f, thr_i)) flags |= 1u << e;
    }
    return flags;
}

// Position of this thread's first detection in the tile's run of the list
// (exclusive scan of the per-thread counts over the CTA); `total` gets the
// tile's count.  Contains one barrier.
__device__ __forceinline__ int tile_rank(unsigned flags, int* wsum, int& total) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int mine = __popc(flags);
    int incl = mine;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
        const int t = __shfl_up_sync(0xffffffffu, incl, d);
        if (lane >= d) incl += t;
    }
    if (lane == 31) wsum[warp] = incl;
    __syncthreads();
    int loc = incl - mine;
    total = 0;
#pragma unroll
    for (int w = 0; w < kThreads / 32; ++w) {
        if (w < warp) loc += wsum[w];
        total += wsum[w];
    }
    return loc;
}

// Build this thread's records of the tile's run of the list in shared
// memory (stage: kTile * kDetWords words), from run position loc on.
template <typename T>
__device__ __forceinline__ void tile_stage(const T (&v)[kPer], unsigned flags, int loc, int nx, int tile, int stride,
                                           int image, int level, uint32_t* stage) {
    const long base = (long)tile * kTile + (long)threadIdx.x * kPer;
#pragma unroll
    for (int e = 0; e < kPer; ++e) {
        if (flags & (1u << e)) {
            const long i = base + e;
            // a map holds fewer than 2^31 scores (every caller checks the size), so 32-bit division
            const int py = (int)((uint32_t)i / (uint32_t)nx), px = (int)i - py * nx;
            uint32_t* d = stage + loc * kDetWords;
            d[0] = (uint32_t)(px * stride);
            d[1] = (uint32_t)(py * stride);
            d[2] = __float_as_uint((float)v[e]);
            d[3] = (uint32_t)image;
            d[4] = (uint32_t)level;
            ++loc;
        }
    }
}

// Copy the tile's staged run (tile_total records) to list positions
// before, before + 1, ... (those below max_out) with coalesced word stores
// (full 128-byte lines, whether `out` is device or mapped host memory).
// The stage must be complete (a barrier after tile_stage).
__device__ __forceinline__ void tile_write(const uint32_t* stage, int tile_total, int before,
                                           hog_det* __restrict__ out, int max_out) {
    const int room = max_out - before;
    const int keep = tile_total < room ? tile_total : (room > 0 ? room : 0);
    uint32_t* dst = reinterpret_cast<uint32_t*>(out + (room > 0 ? before : 0));
    for (int j = threadIdx.x; j < keep * kDetWords; j += kThreads) dst[j] = stage[j];
}

// Write the detections of tile `tile` at list positions before, before + 1,
// ... (those below max_out); returns the tile's number of detections.
template <typename T>
__device__ __forceinline__ int tile_scatter(const T* __restrict__ scores, int nx, long n, int tile, int stride,
                                            float thr_f, int thr_i, int image, int level, int before,
                                            hog_det* __restrict__ out, int max_out, uint32_t* stage, int* wsum) {
    T v[kPer];
    const unsigned flags = tile_load<T>(scores, n, tile, thr_f, thr_i, v);
    int tile_total = 0;
    const int loc = tile_rank(flags, wsum, tile_total);
    tile_stage<T>(v, flags, loc, nx, tile, stride, image, level, stage);
    __syncthreads();
    tile_write(stage, tile_total, before, out, max_out);
    return tile_total;
}

}  // namespace detect
}  // namespace fasthog
