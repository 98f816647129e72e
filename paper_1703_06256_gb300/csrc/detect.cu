// detect.cu -- threshold the score map and compact the windows that pass
// into a list in row-major order (the detection step the paper's pipeline
// ends with, Sections 1 and 4).
//
// One launch, one CTA per tile of 2048 scores, single pass (decoupled
// look-back, onepass.cuh): a CTA loads its scores, ranks the ones that pass
// inside the tile (warp shuffles + one cross-warp step) and publishes the
// tile's count; it builds its run of the list in shared memory while its
// first warp adds up the counts of the tiles before it -- 32 predecessors
// per step, stopping at the nearest one that has already published its
// inclusive prefix -- then publishes its own inclusive prefix and writes
// its run with coalesced stores at the offset found.  The last tile writes
// the total.  Integer scores compare against ceil(thr), which for integers
// is the same test as >= thr.
#include <cmath>
#include <type_traits>

#include "detect_core.cuh"
#include "internal.cuh"
#include "onepass.cuh"

namespace fasthog {

namespace {

using detect::kDetWords;
using detect::kPer;
using detect::kThreads;
using detect::kTile;

// Detections in tiles 0 .. t-1, by warp 0 of tile t > 0.  `ok` turns false
// if a wait ran out (the sum is then incomplete).
__device__ __forceinline__ int look_back(const unsigned long long* st, int t, uint32_t tag, bool& ok) {
    const int lane = threadIdx.x & 31;
    int before = 0;
    for (int hi = t - 1;; hi -= 32) {
        const int p = hi - lane;  // lane 0 the nearest predecessor
        bool incl = true;         // before tile 0: an inclusive prefix of 0
        uint32_t v = 0;
        if (p >= 0 && !onepass::wait_status(st + p, tag, incl, v)) {
            ok = false;
            incl = true;
            v = 0;
        }
        const unsigned m = __ballot_sync(0xffffffffu, incl);
        const int first = __ffs(m) - 1;  // nearest predecessor with an inclusive prefix, or -1
        int take = (first < 0 || lane <= first) ? (int)v : 0;
#pragma unroll
        for (int d = 16; d > 0; d >>= 1) take += __shfl_xor_sync(0xffffffffu, take, d);
        before += take;
        if (first >= 0) break;
    }
    return before;
}

template <typename T>
__global__ void __launch_bounds__(kThreads)
    detect_kernel(const T* __restrict__ scores, int nx, long n, int stride, float thr_f, int thr_i, int image,
                  int level, void* ws, hog_det* __restrict__ out, int max_out, int* __restrict__ d_count,
                  unsigned int* status) {
    __shared__ int wsum[kThreads / 32];
    __shared__ int before_s;
    __shared__ uint32_t stage[kTile * kDetWords];
    pdl_trigger();  // tail of the path: the successor is small, launch it early
    pdl_wait();
    const int tile = blockIdx.x, tiles = gridDim.x;
    unsigned long long* st = reinterpret_cast<unsigned long long*>(static_cast<uint8_t*>(ws) + onepass::kHeaderBytes);
    uint32_t tag = 0;
    if (tiles > 1 && threadIdx.x < 32) tag = onepass::launch_tag(ws);

    T v[kPer];
    const unsigned flags = detect::tile_load<T>(scores, n, tile, thr_f, thr_i, v);
    int total = 0;
    const int loc = detect::tile_rank(flags, wsum, total);
    // the tile's count (tile 0: already its inclusive prefix)
    if (tiles > 1 && threadIdx.x == 0) onepass::st_relaxed(st + tile, onepass::status_word(tag, tile == 0, total));
    detect::tile_stage<T>(v, flags, loc, nx, tile, stride, image, level, stage);
    if (threadIdx.x < 32) {
        int before = 0;
        if (tile > 0) {
            bool ok = true;
            before = look_back(st, tile, tag, ok);
            if (threadIdx.x == 0) {
                if (!ok) atomicOr(status, kStatusTimeout);
                onepass::st_relaxed(st + tile, onepass::status_word(tag, true, (uint32_t)(before + total)));
            }
        }
        if (threadIdx.x == 0) {
            before_s = before;
            if (tile == tiles - 1) {
                *d_count = before + total;
                // every tile has published (the look-back reached tile 0 through inclusive prefixes),
                // so every tile has read the old tag
                if (tiles > 1) onepass::end_launch(ws, tag);
            }
        }
    }
    __syncthreads();
    detect::tile_write(stage, total, before_s, out, max_out);
}

template <typename T>
hog_status launch_t(const void* scores, int nx, int ny, int stride, float thr, int image, int level, hog_det* out,
                    int max_out, int32_t* d_count, void* ws, cudaStream_t st) {
    const long n = (long)nx * ny;
    const int tiles = n > 0 ? ceil_div(n, kTile) : 1;
    int thr_i = 0;
    if (std::is_same<T, int32_t>::value) {
        const double c = ceil((double)thr);
        thr_i = c > 2147483647.0 ? 2147483647 : (c < -2147483648.0 ? (int)(-2147483647 - 1) : (int)c);
    }
    unsigned int* status = nullptr;
    hog_status s = device_status_word(&status);
    if (s != HOG_OK) return s;
    return launch_pdl(detect_kernel<T>, dim3(tiles), dim3(kThreads), 0, st, static_cast<const T*>(scores),
                      nx > 0 ? nx : 1, n, stride, thr, thr_i, image, level, ws, out, max_out, d_count, status);
}

}  // namespace

int detect_tiles(long n_scores) { return n_scores > 0 ? (int)((n_scores + kTile - 1) / kTile) : 0; }

size_t detect_workspace_bytes(int nx, int ny) {
    const long n = (long)nx * ny;
    const long tiles = n > 0 ? (n + kTile - 1) / kTile : 1;
    return (size_t)((onepass::kHeaderBytes + tiles * 8 + 255) / 256 * 256);
}

hog_status launch_detect(const void* scores, int score_dtype, int nx, int ny, int stride, float thr, int image,
                         int level, hog_det* out, int max_out, int32_t* d_count, void* ws, cudaStream_t st) {
    if (score_dtype == HOG_I32)
        return launch_t<int32_t>(scores, nx, ny, stride, thr, image, level, out, max_out, d_count, ws, st);
    return launch_t<float>(scores, nx, ny, stride, thr, image, level, out, max_out, d_count, ws, st);
}

}  // namespace fasthog
