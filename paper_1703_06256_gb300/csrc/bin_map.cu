// bin_map.cu -- oriented-gradient map (paper Section 2, Eq. 1 + table lookup).
//
// Work unit: a quad of 4 consecutive pixels of one row, written as one
// 32-bit word.  A thread loads the 32-bit words that hold its quad and the
// one-pixel halo straight from global memory (through L1: neighbouring
// quads share their edge words): for RGB, 5 words of the centre row and 3
// of the rows above and below; for gray, 3 + 1 + 1.  Every byte position
// inside those words is a compile-time constant, so Eq. 1 for the 4 x C
// channel values needs only register shifts, no shared-memory traffic.
// Rows start at arbitrary addresses; unaligned images take a byte path.
//
// The table lives in shared memory.  The full 511 x 511 table (255.5 KiB)
// does not fit, so when 4 divides N_b the CTA holds one quadrant only:
// (dx, dy) with dx in 1..255, dy in 0..255, 255 x 256 entries, 64 KiB.  A
// quarter turn (dx, dy) -> (-dy, dx) adds pi/2 to the angle and, because
// the sectors are half-open and N_b/4 of them span pi/2, adds exactly N_b/4
// to the bin.  So any gradient is turned into that quadrant by q quarter
// turns and its bin is (quadrant entry + q * N_b/4) mod N_b.  The quadrant
// (rows 255..510, columns 256..511 of the table, each row 16-byte aligned
// thanks to the 512-byte pitch) arrives by 256 bulk async copies that
// complete on one mbarrier, while the first quads' pixels are loaded.
// For other N_b the kernel reads the table through the read-only cache.
//
// The grid is persistent (a few CTAs per SM, grid-stride over quads) so
// that each CTA stages the table once.
#include "internal.cuh"
#include "ptx.cuh"

namespace fasthog {

namespace {

constexpr int kThreads = 256;
constexpr int kQuadBytes = 256 * 256;  // 256 rows (dy 0..255) x 256 columns (dx 1..256)

// Load the 32-bit word at byte offset `off` of a row of `row_bytes` bytes;
// bytes outside the row read as 0.
__device__ __forceinline__ uint32_t row_word(const uint8_t* __restrict__ row, long off, long row_bytes, bool aligned) {
    if (aligned && off >= 0 && off + 4 <= row_bytes) return __ldg(reinterpret_cast<const uint32_t*>(row + off));
    uint32_t w = 0;
#pragma unroll
    for (int b = 0; b < 4; ++b)
        if (off + b >= 0 && off + b < row_bytes) w |= (uint32_t)__ldg(row + off + b) << (8 * b);
    return w;
}

template <int N>
__device__ __forceinline__ int byte_at(const uint32_t (&w)[N], int i) {
    return (int)((w[i >> 2] >> (8 * (i & 3))) & 0xFFu);
}

template <int CH, bool QUAD>
__global__ void __launch_bounds__(kThreads)
    bin_map_kernel(const uint8_t* __restrict__ img, int W, int H, size_t pitch, bool aligned,
                   const uint8_t* __restrict__ lut, int nb, uint8_t* __restrict__ bins, bool word_stores,
                   unsigned int* status) {
    // centre-row words: bytes [4*CH*k - 4, ...) hold pixels x-1 .. x+4
    constexpr int NC = CH == 3 ? 5 : 3;
    constexpr int NV = CH == 3 ? 3 : 1;  // rows above / below: the quad's own bytes
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
        if (tid < 32) {
            if (tid == 0) ptx::mbar_arrive_expect_tx(&lut_bar, kQuadBytes);
            __syncwarp();
            // table row dy + 255, columns 256..511 -> quadrant row dy
            for (int row = tid; row < 256; row += 32)
                ptx::bulk_g2s(lutq + row * 256, lut + (size_t)(row + kDMax) * kLutPitch + 256, 256, &lut_bar);
        }
    }
    bool lut_ready = !QUAD;

    const int qpr = (W + 3) >> 2;  // quads per row
    const long n_quads = (long)qpr * H;
    const long row_bytes = (long)W * CH;
    for (long q = (long)blockIdx.x * kThreads + tid; q < n_quads; q += (long)gridDim.x * kThreads) {
        const int y = (int)(q / qpr);
        const int x = (int)(q - (long)y * qpr) * 4;
        uint32_t packed = 0xFFFFFFFFu;  // border rows: no bins
        if (y > 0 && y < H - 1) {
            const uint8_t* mid = img + (size_t)y * pitch;
            const uint8_t* up = mid - pitch;
            const uint8_t* dn = mid + pitch;
            const long o = (long)x * CH;
            uint32_t wc[NC], wu[NV], wd[NV];
#pragma unroll
            for (int k = 0; k < NC; ++k) wc[k] = row_word(mid, o - 4 + 4 * k, row_bytes, aligned);
#pragma unroll
            for (int k = 0; k < NV; ++k) {
                wu[k] = row_word(up, o + 4 * k, row_bytes, aligned);
                wd[k] = row_word(dn, o + 4 * k, row_bytes, aligned);
            }
            if (!lut_ready) {
                if (!ptx::mbar_wait_bounded(&lut_bar, 0, kWaitLimitNs)) {
                    atomicOr(status, kStatusTimeout);
                    return;  // nothing else of this CTA is in flight
                }
                lut_ready = true;
            }
            packed = 0;
#pragma unroll
            for (int e = 0; e < 4; ++e) {
                uint32_t bin = kNoBin;
                const int xe = x + e;
                if (xe > 0 && xe < W - 1) {
                    // byte of pixel xe+d, channel c in wc: 4 + (e + d) * CH + c
                    int dx = byte_at(wc, 4 + (e + 1) * CH) - byte_at(wc, 4 + (e - 1) * CH);
                    int dy = byte_at(wd, e * CH) - byte_at(wu, e * CH);
                    if (CH == 3) {
                        int best = dx * dx + dy * dy;
#pragma unroll
                        for (int c = 1; c < 3; ++c) {
                            const int ddx = byte_at(wc, 4 + (e + 1) * CH + c) - byte_at(wc, 4 + (e - 1) * CH + c);
                            const int ddy = byte_at(wd, e * CH + c) - byte_at(wu, e * CH + c);
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
                            int qd, ax, ay;
                            if (dx > 0 && dy >= 0) { qd = 0; ax = dx; ay = dy; }
                            else if (dx <= 0 && dy > 0) { qd = 1; ax = dy; ay = -dx; }
                            else if (dx < 0 && dy <= 0) { qd = 2; ax = -dx; ay = -dy; }
                            else { qd = 3; ax = -dy; ay = dx; }
                            const int v = lutq[ay * 256 + ax - 1] + qd * nb4;
                            bin = v >= nb ? v - nb : v;
                        } else {
                            bin = __ldg(lut + (size_t)(dy + kDMax) * kLutPitch + (dx + kDMax));
                        }
                    }
                }
                packed = (packed & ~(0xFFu << (8 * e))) | (bin << (8 * e));
            }
        }
        uint8_t* out = bins + (size_t)y * W + x;
        if (word_stores && x + 3 < W) {
            *reinterpret_cast<uint32_t*>(out) = packed;
        } else {
#pragma unroll
            for (int e = 0; e < 4; ++e)
                if (x + e < W) out[e] = (uint8_t)(packed >> (8 * e));
        }
    }
    if (QUAD && !lut_ready) {
        // This thread never needed the table: still let the copies land
        // before the CTA exits.
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
    const long need = (n_quads + kThreads - 1) / kThreads;
    const long cap = (long)sm_count() * (QUAD ? 3 : 8);
    const int grid = (int)(need < cap ? need : cap);
    const bool aligned = (reinterpret_cast<uintptr_t>(img) % 4 == 0) && (pitch % 4 == 0);
    const bool word_stores = (reinterpret_cast<uintptr_t>(bins) % 4 == 0) && (W % 4 == 0);
    kern<<<grid, kThreads, smem, st>>>(img, W, H, pitch, aligned, lut, nb, bins, word_stores, status);
    return check_launch();
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
