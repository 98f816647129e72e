// detect.cu -- threshold the score map and compact the windows that pass
// into a list in row-major order (the detection step the paper's pipeline
// ends with, Sections 1 and 4).
//
// Two launches, no waiting between CTAs:
//   count    one CTA per tile of 2048 scores writes the tile's number of
//            windows with score >= thr to the workspace;
//   scatter  one CTA per tile sums the counts of the tiles before it (a block
//            reduction over at most a few thousand ints), scans its own flags
//            (warp shuffles + one cross-warp step), builds its run of the
//            list in shared memory and writes it with coalesced stores.  The
//            last tile writes the total.
// A map of a single tile skips the count launch.  Integer scores compare
// against ceil(thr), which for integers is the same test as >= thr.
#include <cmath>
#include <type_traits>

#include "internal.cuh"

namespace fasthog {

namespace {

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

template <typename T>
__global__ void __launch_bounds__(kThreads)
    detect_count_kernel(const T* __restrict__ scores, long n, float thr_f, int thr_i, int* __restrict__ tile_count) {
    __shared__ int red[kThreads / 32];
    pdl_trigger();
    pdl_wait();
    const long base = (long)blockIdx.x * kTile + (long)threadIdx.x * kPer;
    int c = 0;
#pragma unroll
    for (int e = 0; e < kPer; ++e) {
        const long i = base + e;
        if (i < n) c += pass<T>(__ldg(scores + i), thr_f, thr_i);
    }
    c = block_sum(c, red);
    if (threadIdx.x == 0) tile_count[blockIdx.x] = c;
}

template <typename T>
__global__ void __launch_bounds__(kThreads)
    detect_scatter_kernel(const T* __restrict__ scores, int nx, long n, int stride, float thr_f, int thr_i,
                          int image, int level, const int* __restrict__ tile_count, hog_det* __restrict__ out,
                          int max_out, int* __restrict__ d_count) {
    __shared__ int red[kThreads / 32];
    __shared__ int wsum[kThreads / 32];
    __shared__ uint32_t stage[kTile * kDetWords];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    pdl_trigger();
    pdl_wait();
    // detections in the tiles before this one
    int before = 0;
    if (tile_count != nullptr)
        for (int t = threadIdx.x; t < (int)blockIdx.x; t += kThreads) before += __ldg(tile_count + t);
    before = block_sum(before, red);

    const long base = (long)blockIdx.x * kTile + (long)threadIdx.x * kPer;
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
    if (blockIdx.x == gridDim.x - 1 && threadIdx.x == 0) *d_count = before + tile_total;
}

template <typename T>
hog_status launch_t(const void* scores, int nx, int ny, int stride, float thr, int image, int level, hog_det* out,
                    int max_out, int32_t* d_count, void* ws, cudaStream_t st) {
    const long n = (long)nx * ny;
    const int tiles = n > 0 ? ceil_div(n, kTile) : 1;
    int thr_i = 0;
    if (std::is_same<T, int32_t>::value) {
        const double c = ceil((double)thr);
        thr_i = c > 2147483647.0 ? 2147483647 : (c < -2147483647.0 ? -2147483647 : (int)c);
    }
    int* tile_count = nullptr;
    if (tiles > 1) {
        tile_count = static_cast<int*>(ws);
        hog_status s = launch_pdl(detect_count_kernel<T>, dim3(tiles), dim3(kThreads), 0, st,
                                  static_cast<const T*>(scores), n, thr, thr_i, tile_count);
        if (s != HOG_OK) return s;
    }
    return launch_pdl(detect_scatter_kernel<T>, dim3(tiles), dim3(kThreads), 0, st, static_cast<const T*>(scores),
                      nx > 0 ? nx : 1, n, stride, thr, thr_i, image, level, (const int*)tile_count, out, max_out,
                      d_count);
}

}  // namespace

size_t detect_workspace_bytes(int nx, int ny) {
    const long n = (long)nx * ny;
    const long tiles = n > 0 ? (n + kTile - 1) / kTile : 1;
    return (size_t)((tiles * 4 + 255) / 256 * 256);
}

hog_status launch_detect(const void* scores, int score_dtype, int nx, int ny, int stride, float thr, int image,
                         int level, hog_det* out, int max_out, int32_t* d_count, void* ws, cudaStream_t st) {
    if (score_dtype == HOG_I32)
        return launch_t<int32_t>(scores, nx, ny, stride, thr, image, level, out, max_out, d_count, ws, st);
    return launch_t<float>(scores, nx, ny, stride, thr, image, level, out, max_out, d_count, ws, st);
}

}  // namespace fasthog
