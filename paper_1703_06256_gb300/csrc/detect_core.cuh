// detect_core.cuh -- the per-tile pieces of the detection step (threshold
// and ordered compaction, Sections 1 and 4), shared by the per-image kernels
// (detect.cu) and the batch kernels (detect_batch.cu).
#pragma once

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
template <>
__device__ __forceinline__ bool pass<int32_t>(int32_t v, float, int thr_i) {
    return v >= thr_i;
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

// Write the detections of tile `tile` at list positions before, before + 1,
// ... (those below max_out); returns the tile's number of detections.  The
// tile's run of the list is built in shared memory (stage: kTile * kDetWords
// words) and written with coalesced word stores.
template <typename T>
__device__ __forceinline__ int tile_scatter(const T* __restrict__ scores, int nx, long n, int tile, int stride,
                                            float thr_f, int thr_i, int image, int level, int before,
                                            hog_det* __restrict__ out, int max_out, uint32_t* stage, int* wsum) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const long base = (long)tile * kTile + (long)threadIdx.x * kPer;
    T v[kPer];
    unsigned flags = 0;
#pragma unroll
    for (int e = 0; e < kPer; ++e) {
        const long i = base + e;
        v[e] = i < n ? __ldg(scores + i) : T(0);
        if (i < n && pass<T>(v[e], thr_f, thr_i)) flags |= 1u << e;
    }
    const int mine = __popc(flags);
    int incl = mine;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
        const int t = __shfl_up_sync(0xffffffffu, incl, d);
        if (lane >= d) incl += t;
    }
    if (lane == 31) wsum[warp] = incl;
    __syncthreads();
    int loc = incl - mine;  // this thread's first slot in the tile's list
    int tile_total = 0;
#pragma unroll
    for (int w = 0; w < kThreads / 32; ++w) {
        if (w < warp) loc += wsum[w];
        tile_total += wsum[w];
    }
    // The tile's detections are contiguous in the output: build them in
    // shared memory, then write the whole run with coalesced word stores
    // (full 128-byte lines, whether `out` is device or mapped host memory).
#pragma unroll
    for (int e = 0; e < kPer; ++e) {
        if (flags & (1u << e)) {
            const long i = base + e;
            const int py = (int)(i / nx), px = (int)(i - (long)py * nx);
            uint32_t* d = stage + loc * kDetWords;
            d[0] = (uint32_t)(px * stride);
            d[1] = (uint32_t)(py * stride);
            d[2] = __float_as_uint((float)v[e]);
            d[3] = (uint32_t)image;
            d[4] = (uint32_t)level;
            ++loc;
        }
    }
    __syncthreads();
    const int room = max_out - before;
    const int keep = tile_total < room ? tile_total : (room > 0 ? room : 0);
    uint32_t* dst = reinterpret_cast<uint32_t*>(out + (room > 0 ? before : 0));
    for (int j = threadIdx.x; j < keep * kDetWords; j += kThreads) dst[j] = stage[j];
    return tile_total;
}

}  // namespace detect
}  // namespace fasthog
