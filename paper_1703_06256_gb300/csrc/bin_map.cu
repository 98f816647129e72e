// bin_map.cu -- oriented-gradient map (paper Section 2, Eq. 1 + table lookup).
//
// Work unit: a tile of 128 x 16 pixels.  The CTA stages the tile plus a
// one-pixel halo (rows y0-1 .. y0+16, bytes of columns x0-1 .. x0+128) in
// shared memory with 32-bit loads, then every thread forms Eq. 1 for 4 x 2
// pixels, picks the strongest channel and looks the bin up.
//
// The table lives in shared memory.  The full 511 x 511 table (255.5 KiB)
// does not fit, so when 4 divides N_b the CTA holds one quadrant only:
// (dx, dy) with dx in 1..255, dy in 0..255, 255 x 256 entries, 64 KiB.  A
// quarter turn (dx, dy) -> (-dy, dx) adds pi/2 to the angle and, because
// the sectors are half-open and N_b/4 of them span pi/2, adds exactly N_b/4
// to the bin.  So any gradient is turned into that quadrant by q quarter
// turns and its bin is (quadrant entry + q * N_b/4) mod N_b.  The quadrant
// (rows 255..510, columns 256..511 of the table, each row 16-byte aligned
// thanks to the 512-byte pitch) is pulled in by 256 bulk async copies that
// complete on one mbarrier, while the first tile's pixels are loaded.
//
// For other N_b the kernel reads the table from global memory through the
// read-only cache.
//
// The grid is persistent (a multiple of the SM count, at most one CTA per
// tile) so that each CTA stages the table once.
#include "internal.cuh"
#include "ptx.cuh"

namespace fasthog {

namespace {

constexpr int kTileW = 128;
constexpr int kTileH = 16;
constexpr int kThreads = 256;
constexpr int kQuadBytes = 256 * 256;  // 256 rows (dy 0..255) x 256 columns (dx 1..256)

template <int CH>
struct TileGeom {
    // Bytes of one staged row: columns x0-1 .. x0+kTileW, starting at the
    // word-aligned byte x0*CH - 4.
    static constexpr int kWords = (kTileW * CH + CH + 4 + 3) / 4;
    static constexpr int kRowBytes = kWords * 4;
    static constexpr int kRows = kTileH + 2;
};

template <int CH, bool QUAD>
__global__ void __launch_bounds__(kThreads)
    bin_map_kernel(const uint8_t* __restrict__ img, int W, int H, size_t pitch, bool word_loads,
                   const uint8_t* __restrict__ lut, int nb, uint8_t* __restrict__ bins, bool word_stores,
                   unsigned int* status) {
    using G = TileGeom<CH>;
    extern __shared__ __align__(128) uint8_t smem[];
    __shared__ __align__(8) uint64_t lut_bar;
    uint8_t* lutq = smem;                                  // kQuadBytes when QUAD
    uint8_t* tile = smem + (QUAD ? kQuadBytes : 0);        // kRows x kRowBytes

    const int tid = threadIdx.x;
    const int tiles_x = (W + kTileW - 1) / kTileW;
    const int tiles_y = (H + kTileH - 1) / kTileH;
    const int n_tiles = tiles_x * tiles_y;
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

    for (int t = blockIdx.x; t < n_tiles; t += gridDim.x) {
        const int x0 = (t % tiles_x) * kTileW;
        const int y0 = (t / tiles_x) * kTileH;
        const long g0 = (long)x0 * CH - 4;     // byte of the row held at tile[r][0]
        const long row_bytes = (long)W * CH;

        __syncthreads();  // previous tile fully consumed
        for (int i = tid; i < G::kRows * G::kWords; i += kThreads) {
            const int r = i / G::kWords;
            const int k = i - r * G::kWords;
            const int y = y0 - 1 + r;
            uint32_t word = 0;
            if (y >= 0 && y < H) {
                const long g = g0 + 4L * k;
                const uint8_t* rowp = img + (size_t)y * pitch;
                if (word_loads && g >= 0 && g + 4 <= row_bytes) {
                    word = __ldg(reinterpret_cast<const uint32_t*>(rowp + g));
                } else {
#pragma unroll
                    for (int b = 0; b < 4; ++b) {
                        const long gb = g + b;
                        if (gb >= 0 && gb < row_bytes) word |= (uint32_t)__ldg(rowp + gb) << (8 * b);
                    }
                }
            }
            *reinterpret_cast<uint32_t*>(tile + r * G::kRowBytes + 4 * k) = word;
        }
        __syncthreads();

        if (!lut_ready) {
            if (!ptx::mbar_wait_bounded(&lut_bar, 0, kWaitLimitNs)) {
                atomicOr(status, kStatusTimeout);
                return;  // the copies are bounded by the table size; nothing else is in flight
            }
            lut_ready = true;
        }

        // 16 rows x 32 quads of 4 pixels
        for (int qd = tid; qd < kTileH * (kTileW / 4); qd += kThreads) {
            const int r = qd / (kTileW / 4);
            const int c = (qd - r * (kTileW / 4)) * 4;
            const int y = y0 + r;
            if (y >= H) continue;
            uint32_t packed = 0;
#pragma unroll
            for (int e = 0; e < 4; ++e) {
                const int x = x0 + c + e;
                uint32_t bin = kNoBin;
                if (x > 0 && x < W - 1 && y > 0 && y < H - 1) {
                    const uint8_t* mid = tile + (r + 1) * G::kRowBytes + 4;
                    const uint8_t* up = tile + r * G::kRowBytes + 4;
                    const uint8_t* dn = tile + (r + 2) * G::kRowBytes + 4;
                    const int lc = (c + e - 1) * CH, cc = (c + e) * CH, rc = (c + e + 1) * CH;
                    int dx = (int)mid[rc] - (int)mid[lc];
                    int dy = (int)dn[cc] - (int)up[cc];
                    if (CH == 3) {
                        int best = dx * dx + dy * dy;
#pragma unroll
                        for (int ch = 1; ch < 3; ++ch) {
                            const int ddx = (int)mid[rc + ch] - (int)mid[lc + ch];
                            const int ddy = (int)dn[cc + ch] - (int)up[cc + ch];
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
                            int q, ax, ay;
                            if (dx > 0 && dy >= 0) { q = 0; ax = dx; ay = dy; }
                            else if (dx <= 0 && dy > 0) { q = 1; ax = dy; ay = -dx; }
                            else if (dx < 0 && dy <= 0) { q = 2; ax = -dx; ay = -dy; }
                            else { q = 3; ax = -dy; ay = dx; }
                            int v = lutq[ay * 256 + ax - 1] + q * nb4;
                            bin = v >= nb ? v - nb : v;
                        } else {
                            bin = __ldg(lut + (size_t)(dy + kDMax) * kLutPitch + (dx + kDMax));
                        }
                    }
                }
                packed |= bin << (8 * e);
            }
            const int x = x0 + c;
            uint8_t* out = bins + (size_t)y * W + x;
            if (word_stores && x + 3 < W) {
                *reinterpret_cast<uint32_t*>(out) = packed;
            } else {
#pragma unroll
                for (int e = 0; e < 4; ++e)
                    if (x + e < W) out[e] = (uint8_t)(packed >> (8 * e));
            }
        }
    }
    if (QUAD && !lut_ready) {
        // This CTA had no tile: still let its copies land before exiting.
        if (!ptx::mbar_wait_bounded(&lut_bar, 0, kWaitLimitNs)) atomicOr(status, kStatusTimeout);
    }
}

template <int CH, bool QUAD>
hog_status launch_t(const uint8_t* img, int W, int H, size_t pitch, const uint8_t* lut, int nb,
                    uint8_t* bins, unsigned int* status, cudaStream_t st) {
    using G = TileGeom<CH>;
    const size_t smem = (QUAD ? kQuadBytes : 0) + (size_t)G::kRows * G::kRowBytes;
    auto kern = bin_map_kernel<CH, QUAD>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return cuda_fail(e);
    const int n_tiles = ceil_div(W, kTileW) * ceil_div(H, kTileH);
    const int per_sm = QUAD ? 3 : 8;
    const int grid = n_tiles < sm_count() * per_sm ? n_tiles : sm_count() * per_sm;
    const bool word_loads = (reinterpret_cast<uintptr_t>(img) % 4 == 0) && (pitch % 4 == 0);
    const bool word_stores = (reinterpret_cast<uintptr_t>(bins) % 4 == 0) && (W % 4 == 0);
    kern<<<grid, kThreads, smem, st>>>(img, W, H, pitch, word_loads, lut, nb, bins, word_stores, status);
    return check_launch();
}

}  // namespace

hog_status launch_bin_map(const uint8_t* img, int W, int H, int channels, size_t pitch,
                          const uint8_t* lut, int n_bins, uint8_t* bins, unsigned int* status,
                          cudaStream_t st) {
    const bool quad = (n_bins % 4 == 0);
    if (channels == 1)
        return quad ? launch_t<1, true>(img, W, H, pitch, lut, n_bins, bins, status, st)
                    : launch_t<1, false>(img, W, H, pitch, lut, n_bins, bins, status, st);
    return quad ? launch_t<3, true>(img, W, H, pitch, lut, n_bins, bins, status, st)
                : launch_t<3, false>(img, W, H, pitch, lut, n_bins, bins, status, st);
}

}  // namespace fasthog
