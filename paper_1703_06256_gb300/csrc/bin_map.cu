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
// channel (ties to the lowest index).  A thread takes two quads per step
// and issues the next step's loads before computing the current pair, so
// four quads of loads are in flight per thread.
//
// The table is read through the read-only cache by default: gradients of
// natural images cluster near (0, 0), so the lines they touch stay in L1,
// and one lookup is a multiply-add and a load.  Each CTA first asks L2 for
// its slice of the table, so that a table evicted by other work arrives
// while the image loads are in flight.  On request (and when 4
// divides N_b) the CTA instead stages one quadrant in shared memory -- the
// full 511 x 511 table (255.5 KiB) does not fit:
// (dx, dy) with dx in 1..255, dy in 0..255, 255 x 256 entries, 64 KiB.  A
// quarter turn (dx, dy) -> (-dy, dx) adds pi/2 to the angle and, because
// the sectors are half-open and N_b/4 of them span pi/2, adds exactly N_b/4
// to the bin.  So any gradient is turned into that quadrant by q quarter
// turns and its bin is (quadrant entry + q * N_b/4) mod N_b.  The quadrant
// (stored contiguously after the table by hog_build_lut) arrives by one
// 64 KiB bulk async copy that completes on an mbarrier, while the first
// quads' pixels are loaded.  That costs a dozen more instructions per pixel
// (the turn and the wrap-around) than the direct lookup.
//
// The grid is persistent (a few CTAs per SM, grid-stride over quads) so
// that each CTA stages the table once.
//
// Small images take a second schedule (bit-identical): one CTA per tile of
// 128 pixels x 16 rows.  The CTA first copies the tile's rows and the rows
// above and below it, with 16 bytes of halo on each side, into shared memory
// by 16-byte asynchronous copies (bytes outside the image arrive as zeros,
// like the guarded loads above), then warp w computes tile rows w and w + 8,
// lane L the quad at column 4L, reading the same words from shared memory
// (consecutive lanes read words 3 apart for RGB: no bank conflicts).  One
// 16-byte copy per 16 bytes of a row replaces about three 4-byte loads per
// quad, and every tile's copies are in flight at once; when all tiles are
// resident in one wave that is shorter than the grid-stride schedule (at
// 800 x 600 RGB: 266 tiles, 3.88 -> 3.41 us per call in a chain of calls).
// With more tiles than resident CTAs the grid-stride schedule, whose threads
// keep four quads of loads in flight while they compute, is faster.
#include <atomic>

#include "bin_core.cuh"
#include "internal.cuh"
#include "ptx.cuh"

namespace fasthog {

namespace {

constexpr int kThreads = 256;
constexpr int kQuadBytes = 256 * 256;  // 256 rows (dy 0..255) x 256 columns (dx 1..256)

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
__global__ void __launch_bounds__(kThreads, 3)
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
    if (!QUAD) prefetch_table_l2(lut);
    pdl_wait();  // the table copy or prefetch above reads only the table, built before the path runs
    pdl_trigger();

    const int qpr = (W + 3) >> 2;  // quads per row
    const long row_bytes = (long)W * CH;
    // grid-stride over quads in row-major order; the (row, quad) position
    // advances by the stride without dividing
    const long step = (long)gridDim.x * kThreads;
    const int sy = (int)(step / qpr), sxq = (int)(step - (long)sy * qpr);
    auto advance = [&](int& y, int& xq) {
        y += sy;
        xq += sxq;
        if (xq >= qpr) {
            xq -= qpr;
            ++y;
        }
    };
    auto interior = [&](int y) { return y > 0 && y < H - 1; };
    // Two quads per step (a, and b one stride later), software-pipelined:
    // the loads of the next step's pair are issued before this pair is
    // computed, so every thread keeps four quads of loads in flight.
    const long qs = (long)blockIdx.x * kThreads + tid;
    int ya = (int)(qs / qpr), xqa = (int)(qs - (long)ya * qpr);
    int yb = ya, xqb = xqa;
    advance(yb, xqb);
    QuadWords<CH> a, b;
    if (ya < H && interior(ya)) load_quad<CH>(img, pitch, row_bytes, aligned, 4 * xqa, ya, a);
    if (yb < H && interior(yb)) load_quad<CH>(img, pitch, row_bytes, aligned, 4 * xqb, yb, b);
    while (ya < H) {
        int yc = yb, xqc = xqb;
        advance(yc, xqc);
        int yd = yc, xqd = xqc;
        advance(yd, xqd);
        QuadWords<CH> c, d;
        if (yc < H && interior(yc)) load_quad<CH>(img, pitch, row_bytes, aligned, 4 * xqc, yc, c);
        if (yd < H && interior(yd)) load_quad<CH>(img, pitch, row_bytes, aligned, 4 * xqd, yd, d);
        const bool in0 = interior(ya), has1 = yb < H, in1 = has1 && interior(yb);
        if (!lut_ready && (in0 || in1)) {
            if (!ptx::mbar_wait_bounded(&lut_bar, 0, kWaitLimitNs)) {
                atomicOr(status, kStatusTimeout);
                return;  // nothing else of this CTA is in flight
            }
            lut_ready = true;
        }
        // border rows hold no bins
        const int x0 = 4 * xqa, x1 = 4 * xqb;
        store_quad(bins, W, x0, ya, in0 ? bins_of_quad<CH, QUAD>(a, x0, W, lutq, lut, nb, nb4) : 0xFFFFFFFFu,
                   word_stores);
        if (has1)
            store_quad(bins, W, x1, yb, in1 ? bins_of_quad<CH, QUAD>(b, x1, W, lutq, lut, nb, nb4) : 0xFFFFFFFFu,
                       word_stores);
        a = c;
        b = d;
        ya = yc;
        xqa = xqc;
        yb = yd;
        xqb = xqd;
    }
    if (QUAD && !lut_ready) {
        // This thread never needed the table: still let the copy land before
        // the CTA exits.
        if (!ptx::mbar_wait_bounded(&lut_bar, 0, kWaitLimitNs)) atomicOr(status, kStatusTimeout);
    }
}

// ---- staged schedule
constexpr int kTileW = 128, kTileH = 16;  // pixels x rows per CTA; 8 warps x 2 rows
template <int CH>
struct StagedRow {
    static constexpr int kBytes = CH * kTileW + 32;  // 16 bytes of halo on each side
    static constexpr int kWords = kBytes / 4;
    static constexpr int kChunks = kBytes / 16;
};

template <int CH>
__global__ void __launch_bounds__(kThreads, 4)
    bin_map_staged_kernel(const uint8_t* __restrict__ img, int W, int H, size_t pitch,
                          const uint8_t* __restrict__ lut, int nb, uint8_t* __restrict__ bins, bool word_stores) {
    using R = StagedRow<CH>;
    __shared__ __align__(16) uint32_t rows[(kTileH + 2) * R::kWords];
    prefetch_table_l2(lut);
    const int tiles_x = (W + kTileW - 1) / kTileW;
    const int ty = blockIdx.x / tiles_x, tx = blockIdx.x - ty * tiles_x;
    const int x0 = kTileW * tx, y0 = kTileH * ty;
    const long row_bytes = (long)W * CH;
    pdl_wait();  // the prefetch above reads only the table
    pdl_trigger();
    // staged row r holds image row y0 - 1 + r, bytes CH x0 - 16 .. CH (x0 + 128) + 15;
    // the image base and pitch are multiples of 16, so is every chunk's address
    for (int c = threadIdx.x; c < (kTileH + 2) * R::kChunks; c += kThreads) {
        const int r = c / R::kChunks, j = c - r * R::kChunks;
        const int y = y0 - 1 + r;
        const long off = (long)CH * x0 - 16 + 16L * j;
        const uint8_t* src = img;  // nothing is read when n = 0
        int n = 0;
        if (y >= 0 && y < H && off >= 0 && off < row_bytes) {
            src = img + (size_t)y * pitch + off;
            n = (int)(row_bytes - off < 16 ? row_bytes - off : 16);
        }
        ptx::cp_async16_zfill(rows + r * R::kWords + 4 * j, src, n);
    }
    ptx::cp_async_wait_all();
    __syncthreads();
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int x = x0 + 4 * lane;
#pragma unroll
    for (int i = 0; i < kTileH / 8; ++i) {
        const int r = warp + 8 * i, y = y0 + r;
        if (y >= H || x >= W) continue;
        uint32_t packed = 0xFFFFFFFFu;  // border rows hold no bins
        if (y > 0 && y < H - 1) {
            // the words load_quad would read: centre row from byte CH x - 4, the
            // rows above and below from byte CH x
            using Q = QuadWords<CH>;
            Q q;
            const uint32_t* mid = rows + (r + 1) * R::kWords + CH * lane;
#pragma unroll
            for (int k = 0; k < Q::NC; ++k) q.wc[k] = mid[3 + k];
#pragma unroll
            for (int k = 0; k < Q::NV; ++k) {
                q.wu[k] = mid[4 + k - R::kWords];
                q.wd[k] = mid[4 + k + R::kWords];
            }
            packed = bins_of_quad<CH, false>(q, x, W, nullptr, lut, nb, nb >> 2);
        }
        store_quad(bins, W, x, y, packed, word_stores);
    }
}

// Resident CTAs of the staged kernel on the current device (cached per device).
template <int CH>
long staged_capacity() {
    constexpr int kDevices = 64;
    static std::atomic<int> per_sm[kDevices];
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kDevices) return 0;
    int n = per_sm[dev].load(std::memory_order_relaxed);
    if (n == 0) {
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, bin_map_staged_kernel<CH>, kThreads, 0) != cudaSuccess)
            return 0;
        per_sm[dev].store(n > 0 ? n : -1, std::memory_order_relaxed);
    }
    return n > 0 ? (long)n * sm_count() : 0;
}

template <int CH>
bool use_staged(const uint8_t* img, int W, int H, size_t pitch) {
    const int sched = tune_get(HOG_TUNE_BINMAP_SCHEDULE);
    if (sched == 1) return false;
    if (reinterpret_cast<uintptr_t>(img) % 16 != 0 || pitch % 16 != 0) return false;
    const long tiles = (long)((W + kTileW - 1) / kTileW) * ((H + kTileH - 1) / kTileH);
    if (tiles > 0x7FFFFFFFL) return false;
    if (sched == 2) return true;
    return tiles <= staged_capacity<CH>();
}

template <int CH>
hog_status launch_staged(const uint8_t* img, int W, int H, size_t pitch, const uint8_t* lut, int nb, uint8_t* bins,
                         cudaStream_t st) {
    const long tiles = (long)((W + kTileW - 1) / kTileW) * ((H + kTileH - 1) / kTileH);
    const bool word_stores = (reinterpret_cast<uintptr_t>(bins) % 4 == 0) && (W % 4 == 0);
    return launch_pdl(bin_map_staged_kernel<CH>, dim3((unsigned)tiles), dim3(kThreads), 0, st, img, W, H, pitch, lut,
                      nb, bins, word_stores);
}

template <int CH, bool QUAD>
hog_status launch_t(const uint8_t* img, int W, int H, size_t pitch, const uint8_t* lut, int nb, uint8_t* bins,
                    unsigned int* status, cudaStream_t st) {
    const size_t smem = QUAD ? kQuadBytes : 0;
    auto kern = bin_map_kernel<CH, QUAD>;
    if (QUAD) {
        cudaError_t e = smem_at_least<bin_map_kernel<CH, QUAD>>(smem);
        if (e != cudaSuccess) return cuda_fail(e);
    }
    const long n_quads = (long)((W + 3) / 4) * H;
    // at least one step (2 quads) per thread; with a staged table copy, 4 quads,
    // so that each copy serves a fair share of pixels
    const int qpt = QUAD ? 4 : 2;
    const long need = (n_quads + qpt * kThreads - 1) / (qpt * kThreads);
    const int per_sm = tune_get(HOG_TUNE_BINMAP_CTAS_PER_SM);
    // three CTAs per SM are resident (registers; with the quadrant, shared memory too)
    const long cap = (long)sm_count() * (per_sm > 0 ? per_sm : 3);
    const int grid = (int)(need < cap ? need : cap);
    const bool aligned = (reinterpret_cast<uintptr_t>(img) % 4 == 0) && (pitch % 4 == 0);
    const bool word_stores = (reinterpret_cast<uintptr_t>(bins) % 4 == 0) && (W % 4 == 0);
    return launch_pdl(kern, dim3(grid), dim3(kThreads), smem, st, img, W, H, pitch, aligned, lut, nb, bins, word_stores,
                      status);
}

}  // namespace

hog_status launch_bin_map(const uint8_t* img, int W, int H, int channels, size_t pitch, const uint8_t* lut,
                          int n_bins, uint8_t* bins, unsigned int* status, cudaStream_t st) {
    // the shared-memory quadrant needs 4 | N_b and is taken on request; the
    // whole table through the read-only cache is the default
    const bool quad = (n_bins % 4 == 0) && tune_get(HOG_TUNE_TABLE) == 1;
    if (!quad) {
        if (channels == 1 && use_staged<1>(img, W, H, pitch)) return launch_staged<1>(img, W, H, pitch, lut, n_bins, bins, st);
        if (channels == 3 && use_staged<3>(img, W, H, pitch)) return launch_staged<3>(img, W, H, pitch, lut, n_bins, bins, st);
    }
    if (channels == 1)
        return quad ? launch_t<1, true>(img, W, H, pitch, lut, n_bins, bins, status, st)
                    : launch_t<1, false>(img, W, H, pitch, lut, n_bins, bins, status, st);
    return quad ? launch_t<3, true>(img, W, H, pitch, lut, n_bins, bins, status, st)
                : launch_t<3, false>(img, W, H, pitch, lut, n_bins, bins, status, st);
}

}  // namespace fasthog
