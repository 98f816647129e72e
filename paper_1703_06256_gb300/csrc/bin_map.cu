// bin_map.cu -- oriented-gradient map (paper Section 2, Eq. 1 + table lookup).
//
// Work unit: a quad of 4 consecutive pixels of one row, written as one
// 32-bit word.  A thread loads the 32-bit words that hold its quad and the
// one-pixel halo straight from global memory (through L1: neighbouring
// quads share their edge words): for RGB, 5 words of the centre row and 3
// of the rows above and below; for gray, 3 + 1 + 1.  Interior quads of
// 4-byte aligned images load without bounds tests; edge quads and unaligned
// images take a guarded byte path.
//
// Every byte position inside the loaded words is a compile-time constant, so
// Eq. 1 for the 4 x C channel values is register arithmetic: byte
// extraction, differences, dx^2 + dy^2 per channel and the strongest
// channel (ties to the lowest index).  A thread takes two quads per
// iteration and issues both quads' loads before using either.
//
// The table lives in shared memory.  The full 511 x 511 table (255.5 KiB)
// does not fit, so when 4 divides N_b the CTA holds one quadrant only:
// (dx, dy) with dx in 1..255, dy in 0..255, 255 x 256 entries, 64 KiB.  A
// quarter turn (dx, dy) -> (-dy, dx) adds pi/2 to the angle and, because
// the sectors are half-open and N_b/4 of them span pi/2, adds exactly N_b/4
// to the bin.  So any gradient is turned into that quadrant by q quarter
// turns and its bin is (quadrant entry + q * N_b/4) mod N_b.  The quadrant
// (stored contiguously after the table by hog_build_lut) arrives by one
// 64 KiB bulk async copy that completes on an mbarrier, while the first
// quads' pixels are loaded.  For other N_b the kernel reads the table
// through the read-only cache.
//
// The grid is persistent (a few CTAs per SM, grid-stride over quads) so
// that each CTA stages the table once.
#include "internal.cuh"
#include "ptx.cuh"

namespace fasthog {

namespace {

constexpr int kThreads = 256;
constexpr int kQuadBytes = 256 * 256;  // 256 rows (dy 0..255) x 256 columns (dx 1..256)

// The 32-bit word at byte offset `off` of a row of `row_bytes` bytes; bytes
// outside the row read as 0.
__device__ __forceinline__ uint32_t row_word(const uint8_t* __restrict__ row, long off, long row_bytes, bool aligned) {
    if (aligned && off >= 0 && off + 4 <= row_bytes) return __ldg(reinterpret_cast<const uint32_t*>(row + off));
    uint32_t w = 0;
#pragma unroll
    for (int b = 0; b < 4; ++b)
        if (off + b >= 0 && off + b < row_bytes) w |= (uint32_t)__ldg(row + off + b) << (8 * b);
    return w;
}

// Byte i of a little-endian word array, i a compile-time constant.
template <int N>
__device__ __forceinline__ int byte_of(const uint32_t (&w)[N], int i) {
    return (int)((w[i >> 2] >> (8 * (i & 3))) & 0xFFu);
}

template <int CH>
struct QuadWords {
    static constexpr int NC = CH == 3 ? 5 : 3;  // centre-row words, from byte CH*x - 4
    static constexpr int NV = CH == 3 ? 3 : 1;  // rows above / below: the quad's own bytes
    uint32_t wc[NC], wu[NV], wd[NV];
};

// Load the words of quad (x, y), 0 < y < H-1.  Interior quads of aligned
// images load without bounds tests.
template <int CH>
__device__ __forceinline__ void load_quad(const uint8_t* __restrict__ img, size_t pitch, long row_bytes, bool aligned,
                                          int x, int y, QuadWords<CH>& q) {
    using Q = QuadWords<CH>;
    const uint8_t* mid = img + (size_t)y * pitch;
    const uint8_t* up = mid - pitch;
    const uint8_t* dn = mid + pitch;
    const long o = (long)x * CH;
    if (aligned && x >= 4 && o + 4 * Q::NC - 4 <= row_bytes) {
        const uint32_t* m4 = reinterpret_cast<const uint32_t*>(mid + o - 4);
        const uint32_t* u4 = reinterpret_cast<const uint32_t*>(up + o);
        const uint32_t* d4 = reinterpret_cast<const uint32_t*>(dn + o);
#pragma unroll
        for (int k = 0; k < Q::NC; ++k) q.wc[k] = __ldg(m4 + k);
#pragma unroll
        for (int k = 0; k < Q::NV; ++k) {
            q.wu[k] = __ldg(u4 + k);
            q.wd[k] = __ldg(d4 + k);
        }
    } else {
#pragma unroll
        for (int k = 0; k < Q::NC; ++k) q.wc[k] = row_word(mid, o - 4 + 4 * k, row_bytes, aligned);
#pragma unroll
        for (int k = 0; k < Q::NV; ++k) {
            q.wu[k] = row_word(up, o + 4 * k, row_bytes, aligned);
            q.wd[k] = row_word(dn, o + 4 * k, row_bytes, aligned);
        }
    }
}

// Eq. 1 and the table lookup for the 4 pixels of quad x (row loaded in q).
// Channel c of pixel x + p: right neighbour at byte 4 + (p+1)*CH + c of wc,
// left at 4 + (p-1)*CH + c, below / above at byte p*CH + c of wd / wu.
template <int CH, bool QUAD>
__device__ __forceinline__ uint32_t bins_of_quad(const QuadWords<CH>& q, int x, int W, const uint8_t* __restrict__ lutq,
                                                 const uint8_t* __restrict__ lut, int nb, int nb4) {
    uint32_t packed = 0;
#pragma unroll
    for (int p = 0; p < 4; ++p) {
        uint32_t bin = kNoBin;
        const int xp = x + p;
        if (xp > 0 && xp < W - 1) {
            int dx = byte_of(q.wc, 4 + (p + 1) * CH) - byte_of(q.wc, 4 + (p - 1) * CH);
            int dy = byte_of(q.wd, p * CH) - byte_of(q.wu, p * CH);
            if (CH == 3) {
                int best = dx * dx + dy * dy;
#pragma unroll
                for (int c = 1; c < 3; ++c) {
                    const int ddx = byte_of(q.wc, 4 + (p + 1) * CH + c) - byte_of(q.wc, 4 + (p - 1) * CH + c);
                    const int ddy = byte_of(q.wd, p * CH + c) - byte_of(q.wu, p * CH + c);
                    const int m = ddx * ddx + ddy * ddy;
                    if (m > best) {  // strict: ties keep the lower channel
                        best = m;
                        dx = ddx;
                        dy = ddy;
                    }
                }
            }
            if (dx != 0 || dy != 0) {
                if (QUAD) {
                    int qd, u, v;  // quadrant and quadrant-0 coordinates
                    if (dx > 0 && dy >= 0) { qd = 0; u = dx; v = dy; }
                    else if (dx <= 0 && dy > 0) { qd = 1; u = dy; v = -dx; }
                    else if (dx < 0 && dy <= 0) { qd = 2; u = -dx; v = -dy; }
                    else { qd = 3; u = -dy; v = dx; }
                    const int t = lutq[v * 256 + u - 1] + qd * nb4;
                    bin = t >= nb ? t - nb : t;
                } else {
                    bin = __ldg(lut + (size_t)(dy + kDMax) * kLutPitch + (dx + kDMax));
                }
            }
        }
        packed |= bin << (8 * p);
    }
    return packed;
}

__device__ __forceinline__ void store_quad(uint8_t* __restrict__ bins, int W, int x, int y, uint32_t packed,
                                           bool word_stores) {
    uint8_t* out = bins + (size_t)y * W + x;
    if (word_stores && x + 3 < W) {
        *reinterpret_cast<uint32_t*>(out) = packed;
    } else {
#pragma unroll
        for (int e = 0; e < 4; ++e)
            if (x + e < W) out[e] = (uint8_t)(packed >> (8 * e));
    }
}

template <int CH, bool QUAD>
__global__ void __launch_bounds__(kThreads)
    bin_map_kernel(const uint8_t* __restrict__ img, int W, int H, size_t pitch, bool aligned,
                   const uint8_t* __restrict__ lut, int nb, uint8_t* __restrict__ bins, bool word_stores,
                   unsigned int* status) {
    extern __shared__ __align__(128) uint8_t lutq[];
    __shared__ __align__(8) uint64_t lut_bar;

    const int tid = threadIdx.x;
    const int nb4 = nb >> 2;
    if (QUAD) {
        if (tid == 0) {
            ptx::mbar_init(&lut_bar, 1);
            ptx::fence_mbar_init();
        }
        __syncthreads();
        if (tid == 0) {
            // the contiguous quadrant copy that follows the table: one bulk copy
            ptx::mbar_arrive_expect_tx(&lut_bar, kQuadBytes);
            ptx::bulk_g2s(lutq, lut + kLutQuadOffset, kQuadBytes, &lut_bar);
        }
    }
    bool lut_ready = !QUAD;
    pdl_trigger();
    pdl_wait();  // the table copy above reads only the table, built before the path runs

    const int qpr = (W + 3) >> 2;  // quads per row
    const long n_quads = (long)qpr * H;
    const long row_bytes = (long)W * CH;
    const long step = (long)gridDim.x * kThreads;
    // two quads per iteration (q and q + step): both loads are in flight together
    for (long q0 = (long)blockIdx.x * kThreads + tid; q0 < n_quads; q0 += 2 * step) {
        const long q1 = q0 + step;
        const int y0 = (int)(q0 / qpr), x0 = (int)(q0 - (long)y0 * qpr) * 4;
        const bool has1 = q1 < n_quads;
        const int y1 = has1 ? (int)(q1 / qpr) : 0, x1 = has1 ? (int)(q1 - (long)y1 * qpr) * 4 : 0;
        const bool in0 = y0 > 0 && y0 < H - 1, in1 = has1 && y1 > 0 && y1 < H - 1;
        QuadWords<CH> a, b;
        if (in0) load_quad<CH>(img, pitch, row_bytes, aligned, x0, y0, a);
        if (in1) load_quad<CH>(img, pitch, row_bytes, aligned, x1, y1, b);
        if (!lut_ready && (in0 || in1)) {
            if (!ptx::mbar_wait_bounded(&lut_bar, 0, kWaitLimitNs)) {
                atomicOr(status, kStatusTimeout);
                return;  // nothing else of this CTA is in flight
            }
            lut_ready = true;
        }
        // border rows hold no bins
        store_quad(bins, W, x0, y0, in0 ? bins_of_quad<CH, QUAD>(a, x0, W, lutq, lut, nb, nb4) : 0xFFFFFFFFu,
                   word_stores);
        if (has1)
            store_quad(bins, W, x1, y1, in1 ? bins_of_quad<CH, QUAD>(b, x1, W, lutq, lut, nb, nb4) : 0xFFFFFFFFu,
                       word_stores);
    }
    if (QUAD && !lut_ready) {
        // This thread never needed the table: still let the copy land before
        // the CTA exits.
        if (!ptx::mbar_wait_bounded(&lut_bar, 0, kWaitLimitNs)) atomicOr(status, kStatusTimeout);
    }
}

template <int CH, bool QUAD>
hog_status launch_t(const uint8_t* img, int W, int H, size_t pitch, const uint8_t* lut, int nb, uint8_t* bins,
                    unsigned int* status, cudaStream_t st) {
    const size_t smem = QUAD ? kQuadBytes : 0;
    auto kern = bin_map_kernel<CH, QUAD>;
    if (QUAD) {
        cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return cuda_fail(e);
    }
    const long n_quads = (long)((W + 3) / 4) * H;
    // at least 4 quads per thread, so each staged table copy serves a fair share of pixels
    const long need = (n_quads + 4 * kThreads - 1) / (4 * kThreads);
    const long cap = (long)sm_count() * (QUAD ? 3 : 8);
    const int grid = (int)(need < cap ? need : cap);
    const bool aligned = (reinterpret_cast<uintptr_t>(img) % 4 == 0) && (pitch % 4 == 0);
    const bool word_stores = (reinterpret_cast<uintptr_t>(bins) % 4 == 0) && (W % 4 == 0);
    return launch_pdl(kern, dim3(grid), dim3(kThreads), smem, st, img, W, H, pitch, aligned, lut, nb, bins, word_stores,
                      status);
}

}  // namespace

hog_status launch_bin_map(const uint8_t* img, int W, int H, int channels, size_t pitch, const uint8_t* lut,
                          int n_bins, uint8_t* bins, unsigned int* status, cudaStream_t st) {
    const bool quad = (n_bins % 4 == 0);
    if (channels == 1)
        return quad ? launch_t<1, true>(img, W, H, pitch, lut, n_bins, bins, status, st)
                    : launch_t<1, false>(img, W, H, pitch, lut, n_bins, bins, status, st);
    return quad ? launch_t<3, true>(img, W, H, pitch, lut, n_bins, bins, status, st)
                : launch_t<3, false>(img, W, H, pitch, lut, n_bins, bins, status, st);
}

}  // namespace fasthog
