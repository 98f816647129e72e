// integral.cu -- one integral image per bin (paper Section 3.2, Eq. 4-5).
//
//   ii_n(x, y) = #{ (x', y') : x' <= x, y' <= y, bin(x', y') = n }
//
// The one-hot images of Eq. 4 are never stored: every phase tests the bin
// map on the fly.  The planes are written exactly once, which is the bulk of
// the work (4 * N_b bytes per pixel for int32, 2 * N_b for uint16).
//
// Tiling.  One warp owns a tile of h rows (a band) by G columns (a group).
// Lane L holds the columns 4L..4L+3 of every 128-column slice of the group
// (one slice, G = 128, in the current tiling), so that a warp's 16-byte
// stores cover whole sectors.  A tile's values need three carries from
// outside it:
//   V(x, top-1)   per column and bin, the count above the band;
//   RL(y)         per row and bin, the count left of the group;
//   corner        per bin, ii(group_left - 1, top - 1).
// With those, ii(x, y) = ii(x, y-1) + RL(y) + (row prefix inside the group),
// starting from ii(x, top-1) = corner + (prefix of V over the group's
// columns up to x).  V is a whole row vector per band, too large to pass
// along a look-back chain, so the carries come from a reduce-then-scan in
// which no warp ever waits for another:
//
//   A  tile reduce  per tile: per-column counts over the band (8-bit fields,
//                   4 bins per word), per-row counts over the group (a warp
//                   reduction per row), and the tile's total per bin.
//   B  carries      (a) per column: the exclusive prefix of the column counts
//                   over bands = V at every band top; (b) per group and bin:
//                   the exclusive prefix of the tile totals over bands (in
//                   place); (c) per row: the exclusive prefix of the row
//                   counts over groups = RL (in place, a warp per row).
//   C  tile scan    per tile: corner = the sum of (b) over the groups to the
//                   left; acc = corner + prefix of V over the columns;
//                   then per row the one-hot row's prefix inside each chunk
//                   (8-bit fields), warp shuffle scans of the chunk totals,
//                   and acc += RL + those prefixes; each lane stores its
//                   chunks of every plane.  No barrier inside a row.
//
// The one-hot counts come from variable shifts: bin b of a window starting
// at lo sets byte b - lo - 4m of word m (bins lo + 4m .. lo + 4m + 3) through
// 1 << 8 (b - lo - 4m); every other bin, and 0xFF, gives a shift outside
// 0..31, which shl clamps to a zero result.
//
// Bins are handled in windows of at most 16; larger N_b runs the phases once
// per window.  Limits: W, H < 65536 (16-bit row counts and carries).
//
// Three schedules compute the same planes: the three launches above (large
// images), a single pass (small images, where three launches cost more in
// latency than the planes take to write) and a cluster pass (images up to
// 640 rows; see "cluster pass" below).
//
// Single pass.  One CTA per tile of R = 16 or 32
// rows by 128 columns, tiles numbered row-major; warp w owns 2 rows of the
// tile.  A CTA loads its rows, publishes the tile's aggregates -- its
// per-column counts over the R rows, its per-row counts over the 128
// columns and its totals -- and raises its flag (onepass.cuh).  It then
// waits for the flags of the tiles above and to the left (all of lower
// number, each raised right after its own loads: no chain of waits), and
// forms its carries directly from their aggregates:
//   V(x, tile top - 1) = sum over the tiles above of their column counts;
//   RL(y)              = sum over the tiles to the left of their row counts;
//   corner             = sum over the tiles above-left of their totals.
// Inside the tile the warps' carries come from shared memory (the column
// counts of the warps above, the RL of the rows above), and each warp runs
// the scan of phase C on its rows.
#include <map>
#include <mutex>
#include <tuple>

#include "internal.cuh"
#include "onepass.cuh"

namespace fasthog {

namespace {

constexpr int kMaxBand = 32;        // rows per tile at most (8-bit column counts)
constexpr int kCarryThreads = 512;
constexpr int kSegments = kCarryThreads / 32;  // phase B(a): band segments per column
constexpr int kSlice = 128;         // columns per slice: 4 per lane

template <int WIN>
struct Cfg {
    static constexpr int NCH = 1;                  // 4-column chunks per lane
    static constexpr int G = kSlice * NCH;         // columns per tile
    static constexpr int NM = (WIN + 3) / 4;       // 8-bit-field words, 4 bins each
};

struct Plan {
    int W, H, h, n_bands, n_groups, win, n_windows, G;
    size_t colcnt_bytes, rowcnt_bytes, bt_bytes, carry_bytes;
};

inline size_t align256(size_t b) { return (b + 255) & ~size_t(255); }

// Band height h (rows per tile): the tuned value if one is set (force > 0
// overrides both), else the tallest band that still gives every SM 16 tiles
// (one warp each).
Plan make_plan(int W, int H, int n_bins, int force = 0) {
    Plan p{};
    p.W = W;
    p.H = H;
    p.win = n_bins <= 4 ? 4 : (n_bins <= 8 ? 8 : 16);
    p.n_windows = ceil_div(n_bins, p.win);
    p.G = p.win == 16 ? Cfg<16>::G : Cfg<8>::G;
    p.n_groups = ceil_div(W, p.G);
    const int tuned = force > 0 ? force : tune_get(HOG_TUNE_INTEGRAL_BAND_ROWS);
    if (tuned > 0) {
        p.h = tuned;
    } else {
        const long target = 16L * sm_count();
        p.h = 4;
        for (int h : {32, 16, 8})
            if ((long)ceil_div(H, h) * p.n_groups >= target) {
                p.h = h;
                break;
            }
    }
    p.n_bands = ceil_div(H, p.h);
    const int nm = (p.win + 3) / 4;
    p.colcnt_bytes = align256((size_t)p.n_bands * nm * W * 4);
    p.rowcnt_bytes = align256((size_t)H * p.n_groups * p.win * 2);
    p.bt_bytes = align256((size_t)p.n_bands * p.n_groups * p.win * 4);
    p.carry_bytes = align256((size_t)p.n_bands * W * p.win * 2);
    return p;
}

struct Ws {
    uint32_t* colcnt;  // [band][NM][W]        8-bit column counts over the band, 4 bins per word
    uint16_t* rowcnt;  // [y][group][WIN]      row counts inside the group, then RL (in place)
    uint32_t* bt;      // [band][group][WIN]   tile totals, then their prefix over bands (in place)
    uint16_t* carry;   // [band][W][WIN]       V(x, band_top - 1)
};

Ws carve(const Plan& p, void* base) {
    uint8_t* b = static_cast<uint8_t*>(base);
    Ws w;
    w.colcnt = reinterpret_cast<uint32_t*>(b);
    b += p.colcnt_bytes;
    w.rowcnt = reinterpret_cast<uint16_t*>(b);
    b += p.rowcnt_bytes;
    w.bt = reinterpret_cast<uint32_t*>(b);
    b += p.bt_bytes;
    w.carry = reinterpret_cast<uint16_t*>(b);
    return w;
}

// 1 << n, or 0 when n >= 32 as an unsigned number (PTX clamps the shift amount).
__device__ __forceinline__ uint32_t bit_or_zero(uint32_t n) {
    uint32_t r;
    asm("shl.b32 %0, %1, %2;" : "=r"(r) : "r"(1u), "r"(n));
    return r;
}

// Byte k of x, zero-extended.
__device__ __forceinline__ uint32_t byte_at(uint32_t x, int k) { return __byte_perm(x, 0u, 0x4440u | (uint32_t)k); }

__device__ __forceinline__ uint32_t warp_incl_scan(uint32_t v, int lane) {
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
        const uint32_t t = __shfl_up_sync(0xffffffffu, v, d);
        if (lane >= d) v += t;
    }
    return v;
}

// The bins of the 4 columns at p (0xFF past the ncol valid ones).
__device__ __forceinline__ uint32_t load_chunk(const uint8_t* __restrict__ p, int ncol, bool vec) {
    if (vec && ncol == 4) return __ldg(reinterpret_cast<const uint32_t*>(p));
    uint32_t w = 0;
#pragma unroll
    for (int k = 0; k < 4; ++k) w |= (k < ncol ? (uint32_t)__ldg(p + k) : 0xFFu) << (8 * k);
    return w;
}

// Column geometry of this lane's chunks in tile group g.
template <int NCH>
struct Chunks {
    int x[NCH];     // first column of each chunk
    int ncol[NCH];  // valid columns of each chunk (0..4)
    __device__ __forceinline__ Chunks(int g, int G, int W) {
#pragma unroll
        for (int j = 0; j < NCH; ++j) {
            x[j] = g * G + kSlice * j + 4 * (int)threadIdx.x;
            ncol[j] = max(0, min(4, W - x[j]));
        }
    }
};

// Park this lane's chunks of rows y0 .. y0 + nrows - 1 in shared memory; the
// loads of up to 16 rows are issued before any of them is stored.
template <int NCH>
__device__ __forceinline__ void stage_rows(const uint8_t* __restrict__ bins, int W, int y0, int nrows,
                                           const Chunks<NCH>& ch, bool vec, uint32_t (*st)[32][NCH]) {
    const int lane = threadIdx.x;
    for (int r0 = 0; r0 < nrows; r0 += 16) {
        uint32_t v[16][NCH];
#pragma unroll
        for (int k = 0; k < 16; ++k) {
            const uint8_t* row = bins + (size_t)(y0 + r0 + k) * W;
#pragma unroll
            for (int j = 0; j < NCH; ++j) v[k][j] = r0 + k < nrows ? load_chunk(row + ch.x[j], ch.ncol[j], vec) : 0u;
        }
#pragma unroll
        for (int k = 0; k < 16; ++k)
            if (r0 + k < nrows)
#pragma unroll
                for (int j = 0; j < NCH; ++j) st[r0 + k][lane][j] = v[k][j];
    }
}

// ---------------------------------------------------------------- phase A
template <int WIN>
__global__ void __launch_bounds__(32, 16)
    ii_tile_reduce_kernel(const uint8_t* __restrict__ bins, int W, int H, int h, int n_bands, int n_groups, int lo,
                          bool vec, Ws ws) {
    using C = Cfg<WIN>;
    constexpr int NCH = C::NCH, NM = C::NM;
    static_assert(4 * NCH * 32 < 256, "a group row's count of a bin must fit a byte");
    const int tile = blockIdx.x;
    const int band = tile / n_groups, g = tile - band * n_groups;
    const int lane = threadIdx.x;
    const Chunks<NCH> ch(g, C::G, W);
    const int y0 = band * h, nrows = min(h, H - y0);

    pdl_wait();
    pdl_trigger();

    // col[j][k][m]: counts over the band of bins lo+4m .. lo+4m+3 in column k
    // of chunk j (8-bit fields: a band has at most 32 rows)
    uint32_t col[NCH][4][NM];
#pragma unroll
    for (int j = 0; j < NCH; ++j)
#pragma unroll
        for (int k = 0; k < 4; ++k)
#pragma unroll
            for (int m = 0; m < NM; ++m) col[j][k][m] = 0;
    // rc: lane r keeps row r's counts over the group, 8-bit fields, word m = bins lo+4m .. lo+4m+3
    uint32_t rc[NM];
#pragma unroll
    for (int m = 0; m < NM; ++m) rc[m] = 0;

    for (int r0 = 0; r0 < nrows; r0 += 16) {
        // the loads of 16 rows are in flight together
        uint32_t v[16][NCH];
#pragma unroll
        for (int k = 0; k < 16; ++k) {
            const uint8_t* row = bins + (size_t)(y0 + r0 + k) * W;
#pragma unroll
            for (int j = 0; j < NCH; ++j)
                v[k][j] = r0 + k < nrows ? load_chunk(row + ch.x[j], ch.ncol[j], vec) : 0xFFFFFFFFu;
        }
#pragma unroll
        for (int k = 0; k < 16; ++k) {
            if (r0 + k >= nrows) break;
            uint32_t rowt[NM];
#pragma unroll
            for (int m = 0; m < NM; ++m) rowt[m] = 0;
#pragma unroll
            for (int j = 0; j < NCH; ++j) {
#pragma unroll
                for (int c = 0; c < 4; ++c) {
                    const int t = 8 * ((int)byte_at(v[k][j], c) - lo);
#pragma unroll
                    for (int m = 0; m < NM; ++m) {
                        const uint32_t oh = bit_or_zero((uint32_t)(t - 32 * m));
                        col[j][c][m] += oh;
                        rowt[m] += oh;
                    }
                }
            }
            // sum over the warp (a group row holds at most 4 * NCH * 32 < 256 of a bin)
#pragma unroll
            for (int m = 0; m < NM; ++m) {
                const uint32_t sum = __reduce_add_sync(0xffffffffu, rowt[m]);
                if (lane == r0 + k) rc[m] = sum;
            }
        }
    }

    // per-column counts of the band
#pragma unroll
    for (int j = 0; j < NCH; ++j) {
#pragma unroll
        for (int m = 0; m < NM; ++m) {
            uint32_t* dst = ws.colcnt + ((size_t)band * NM + m) * W + ch.x[j];
            if (vec && ch.ncol[j] == 4) {
                *reinterpret_cast<uint4*>(dst) = make_uint4(col[j][0][m], col[j][1][m], col[j][2][m], col[j][3][m]);
            } else {
#pragma unroll
                for (int k = 0; k < 4; ++k)
                    if (k < ch.ncol[j]) dst[k] = col[j][k][m];
            }
        }
    }
    // per-row counts of the group: WIN consecutive uint16 per row; rcw word i = bins lo+2i, lo+2i+1
    uint32_t rcw[2 * NM];
#pragma unroll
    for (int m = 0; m < NM; ++m) {
        rcw[2 * m] = __byte_perm(rc[m], 0u, 0x4140u);
        rcw[2 * m + 1] = __byte_perm(rc[m], 0u, 0x4342u);
    }
    if (lane < nrows) {
        uint16_t* dst = ws.rowcnt + ((size_t)(y0 + lane) * n_groups + g) * WIN;
        if (NM == 1) {
            *reinterpret_cast<uint2*>(dst) = make_uint2(rcw[0], rcw[1 % (2 * NM)]);
        } else {
#pragma unroll
            for (int k = 0; k < NM / 2; ++k)
                reinterpret_cast<uint4*>(dst)[k] = make_uint4(rcw[4 * k], rcw[(4 * k + 1) % (2 * NM)],
                                                              rcw[(4 * k + 2) % (2 * NM)], rcw[(4 * k + 3) % (2 * NM)]);
        }
    }
    // tile totals (at most 32 * 256 per bin)
    uint32_t tot[2 * NM];
#pragma unroll
    for (int i = 0; i < 2 * NM; ++i) tot[i] = __reduce_add_sync(0xffffffffu, lane < nrows ? rcw[i] : 0u);
    if (lane < WIN) {
        uint32_t v = 0;
#pragma unroll
        for (int i = 0; i < 2 * NM; ++i)
            if (i == (lane >> 1)) v = tot[i];
        v = (lane & 1) ? (v >> 16) : (v & 0xFFFFu);
        ws.bt[((size_t)band * n_groups + g) * WIN + lane] = v;
    }
}

// ---------------------------------------------------------------- phase B
// Blocks [0, na): (a) column carries; block = 32 columns, all bins; threads
//   (lane = column, warp = segment of bands).
// Blocks [na, na + nbb): (b) tile-total prefixes; block = 32 (group, bin)
//   pairs; threads (lane = pair, warp = segment of bands).
// Blocks [na + nbb, ...): (c) RL; one warp per row, lanes = groups.
template <int WIN>
__global__ void __launch_bounds__(kCarryThreads)
    ii_carry_kernel(int W, int H, int n_bands, int n_groups, int na, int nbb, Ws ws) {
    constexpr int NM = Cfg<WIN>::NM;
    constexpr int kWarps = kCarryThreads / 32;
    constexpr int kPF = 8;  // bands of loads in flight per thread
    static_assert(kSegments == 16, "the segment scans take half a warp per column");
    __shared__ uint32_t seg_sum[4][32][kSegments + 1];  // [bin of 4][column][segment]
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    pdl_wait();
    pdl_trigger();

    if ((int)blockIdx.x >= na + nbb) {
        // (c) RL(y) = exclusive prefix over groups of the row counts, in place;
        // 16-bit fields never carry: a row holds at most W < 65536 of a bin
        const int y = (blockIdx.x - na - nbb) * kWarps + warp;
        if (y >= H) return;
        uint16_t* row = ws.rowcnt + (size_t)y * n_groups * WIN;
        uint32_t before[WIN / 2];
#pragma unroll
        for (int i = 0; i < WIN / 2; ++i) before[i] = 0;
        for (int g0 = 0; g0 < n_groups; g0 += 32) {
            const int g = g0 + lane;
            uint32_t u[WIN / 2];
#pragma unroll
            for (int i = 0; i < WIN / 2; ++i) u[i] = 0;
            uint16_t* src = row + (size_t)g * WIN;
            if (g < n_groups) {
                if (WIN == 4) {
                    const uint2 a = __ldcg(reinterpret_cast<const uint2*>(src));
                    u[0] = a.x;
                    u[1 % (WIN / 2)] = a.y;
                } else {
#pragma unroll
                    for (int q = 0; q < WIN / 8; ++q) {
                        const uint4 a = __ldcg(reinterpret_cast<const uint4*>(src) + q);
                        u[4 * q] = a.x;
                        u[(4 * q + 1) % (WIN / 2)] = a.y;
                        u[(4 * q + 2) % (WIN / 2)] = a.z;
                        u[(4 * q + 3) % (WIN / 2)] = a.w;
                    }
                }
            }
#pragma unroll
            for (int i = 0; i < WIN / 2; ++i) {
                const uint32_t incl = warp_incl_scan(u[i], lane);
                const uint32_t excl = before[i] + incl - u[i];
                before[i] += __shfl_sync(0xffffffffu, incl, 31);
                u[i] = excl;
            }
            if (g < n_groups) {
                if (WIN == 4) {
                    *reinterpret_cast<uint2*>(src) = make_uint2(u[0], u[1 % (WIN / 2)]);
                } else {
#pragma unroll
                    for (int q = 0; q < WIN / 8; ++q)
                        reinterpret_cast<uint4*>(src)[q] = make_uint4(u[4 * q], u[(4 * q + 1) % (WIN / 2)],
                                                                      u[(4 * q + 2) % (WIN / 2)],
                                                                      u[(4 * q + 3) % (WIN / 2)]);
                }
            }
        }
        return;
    }

    const int seg = warp;
    const int per = (n_bands + kSegments - 1) / kSegments;
    const int b0 = min(n_bands, seg * per), b1 = min(n_bands, b0 + per);
    // exclusive scan over the segments of the 4 values in s, for the 32
    // columns of the block: the two halves of warp w scan columns w and w + 16
    auto segment_scan = [&](const uint32_t (&s)[4], uint32_t (&run)[4]) {
#pragma unroll
        for (int e = 0; e < 4; ++e) seg_sum[e][lane][seg] = s[e];
        __syncthreads();
        const int cx = warp + 16 * (lane >> 4), sg = lane & 15;
#pragma unroll
        for (int e = 0; e < 4; ++e) {
            const uint32_t v = seg_sum[e][cx][sg];
            uint32_t incl = v;
#pragma unroll
            for (int d = 1; d < 16; d <<= 1) {
                const uint32_t t = __shfl_up_sync(0xffffffffu, incl, d, 16);
                if (sg >= d) incl += t;
            }
            seg_sum[e][cx][sg] = incl - v;
        }
        __syncthreads();
#pragma unroll
        for (int e = 0; e < 4; ++e) run[e] = seg_sum[e][lane][seg];
        __syncthreads();
    };

    if ((int)blockIdx.x >= na) {
        // (b) per (group, bin) pair: exclusive prefix over bands of the tile totals, in place
        const int np = n_groups * WIN;
        const int pi = (blockIdx.x - na) * 32 + lane;
        uint32_t* t = ws.bt + pi;  // band k at t[k * np]
        uint32_t s[4] = {0, 0, 0, 0}, run[4];
        for (int b = b0; b < b1; b += kPF) {
            uint32_t v[kPF];
#pragma unroll
            for (int k = 0; k < kPF; ++k) v[k] = (pi < np && b + k < b1) ? __ldcg(t + (size_t)(b + k) * np) : 0u;
#pragma unroll
            for (int k = 0; k < kPF; ++k) s[0] += v[k];
        }
        segment_scan(s, run);
        if (pi >= np) return;
        for (int b = b0; b < b1; b += kPF) {
            uint32_t v[kPF];
#pragma unroll
            for (int k = 0; k < kPF; ++k) v[k] = b + k < b1 ? __ldcg(t + (size_t)(b + k) * np) : 0u;
#pragma unroll
            for (int k = 0; k < kPF; ++k)
                if (b + k < b1) {
                    t[(size_t)(b + k) * np] = run[0];
                    run[0] += v[k];
                }
        }
        return;
    }

    // (a) V at every band top: exclusive prefix over bands of the column counts
    const int x = blockIdx.x * 32 + lane;
    uint32_t s[4 * NM];
#pragma unroll
    for (int i = 0; i < 4 * NM; ++i) s[i] = 0;
    for (int b = b0; b < b1; b += kPF) {
        uint32_t wv[kPF][NM];
#pragma unroll
        for (int k = 0; k < kPF; ++k)
#pragma unroll
            for (int m = 0; m < NM; ++m)
                wv[k][m] = (x < W && b + k < b1) ? __ldcg(ws.colcnt + ((size_t)(b + k) * NM + m) * W + x) : 0u;
#pragma unroll
        for (int k = 0; k < kPF; ++k)
#pragma unroll
            for (int m = 0; m < NM; ++m)
#pragma unroll
                for (int e = 0; e < 4; ++e) s[4 * m + e] += byte_at(wv[k][m], e);
    }
    uint32_t run[4 * NM];
#pragma unroll
    for (int m = 0; m < NM; ++m) {
        uint32_t s4[4] = {s[4 * m], s[4 * m + 1], s[4 * m + 2], s[4 * m + 3]}, r4[4];
        segment_scan(s4, r4);
#pragma unroll
        for (int e = 0; e < 4; ++e) run[4 * m + e] = r4[e];
    }
    if (x >= W) return;
    for (int b = b0; b < b1; b += kPF) {
        uint32_t wv[kPF][NM];
#pragma unroll
        for (int k = 0; k < kPF; ++k)
#pragma unroll
            for (int m = 0; m < NM; ++m)
                wv[k][m] = b + k < b1 ? __ldcg(ws.colcnt + ((size_t)(b + k) * NM + m) * W + x) : 0u;
#pragma unroll
        for (int k = 0; k < kPF; ++k) {
            if (b + k < b1) {
                // V of this column at the top of band b + k, WIN uint16 (bins lo .. lo + WIN - 1)
                uint32_t u[WIN / 2];
#pragma unroll
                for (int i = 0; i < WIN / 2; ++i) u[i] = (run[2 * i] & 0xFFFFu) | (run[2 * i + 1] << 16);
                uint16_t* dst = ws.carry + ((size_t)(b + k) * W + x) * WIN;
                if (WIN == 4) {
                    *reinterpret_cast<uint2*>(dst) = make_uint2(u[0], u[1 % (WIN / 2)]);
                } else {
#pragma unroll
                    for (int q = 0; q < WIN / 8; ++q)
                        reinterpret_cast<uint4*>(dst)[q] = make_uint4(u[4 * q], u[(4 * q + 1) % (WIN / 2)],
                                                                      u[(4 * q + 2) % (WIN / 2)],
                                                                      u[(4 * q + 3) % (WIN / 2)]);
                }
#pragma unroll
                for (int m = 0; m < NM; ++m)
#pragma unroll
                    for (int e = 0; e < 4; ++e) run[4 * m + e] += byte_at(wv[k][m], e);
            }
        }
    }
}

// ---------------------------------------------------------------- phase C
template <typename OutT>
__device__ __forceinline__ void store_chunk(OutT* p, const int* v, int n, bool vec) {
    if (vec && n == 4) {
        if (sizeof(OutT) == 4) {
            *reinterpret_cast<int4*>(p) = make_int4(v[0], v[1], v[2], v[3]);
        } else {
            *reinterpret_cast<uint2*>(p) = make_uint2(__byte_perm((uint32_t)v[0], (uint32_t)v[1], 0x5410u),
                                                      __byte_perm((uint32_t)v[2], (uint32_t)v[3], 0x5410u));
        }
    } else {
#pragma unroll
        for (int k = 0; k < 4; ++k)
            if (k < n) p[k] = (OutT)v[k];
    }
}

template <int WIN, typename OutT>
__global__ void __launch_bounds__(32)
    ii_tile_scan_kernel(const uint8_t* __restrict__ bins, int W, int H, int h, int n_groups, int lo, int n_bins,
                        bool vec, Ws ws, OutT* __restrict__ ii) {
    using C = Cfg<WIN>;
    constexpr int NCH = C::NCH, NM = C::NM;
    __shared__ uint32_t st[kMaxBand][32][NCH];
    __shared__ __align__(16) uint32_t rl_s[kMaxBand][WIN];
    const int tile = blockIdx.x;
    const int band = tile / n_groups, g = tile - band * n_groups;
    const int lane = threadIdx.x;
    const Chunks<NCH> ch(g, C::G, W);
    const int y0 = band * h, nrows = min(h, H - y0);
    const int wins = min(WIN, n_bins - lo);

    pdl_wait();
    pdl_trigger();
    stage_rows<NCH>(bins, W, y0, nrows, ch, vec, st);
    // RL of the band's rows: lane r fetches row r
    if (lane < nrows) {
        const uint16_t* src = ws.rowcnt + ((size_t)(y0 + lane) * n_groups + g) * WIN;
        uint32_t u[WIN / 2];
        if (WIN == 4) {
            const uint2 a = __ldcg(reinterpret_cast<const uint2*>(src));
            u[0] = a.x;
            u[1 % (WIN / 2)] = a.y;
        } else {
#pragma unroll
            for (int k = 0; k < WIN / 8; ++k) {
                const uint4 a = __ldcg(reinterpret_cast<const uint4*>(src) + k);
                u[4 * k] = a.x;
                u[(4 * k + 1) % (WIN / 2)] = a.y;
                u[(4 * k + 2) % (WIN / 2)] = a.z;
                u[(4 * k + 3) % (WIN / 2)] = a.w;
            }
        }
#pragma unroll
        for (int k = 0; k < WIN / 2; ++k) {
            rl_s[lane][2 * k] = u[k] & 0xFFFFu;
            rl_s[lane][2 * k + 1] = u[k] >> 16;
        }
    }
    // corner = ii(group_left - 1, y0 - 1): the sum over the groups to the left
    // of their counts above the band; lanes split the groups, then combine
    uint32_t corner = 0;
    {
        constexpr int kSlots = 32 / WIN;
        const uint32_t* src = ws.bt + (size_t)band * n_groups * WIN + (lane % WIN);
        for (int gg = lane / WIN; gg < g; gg += kSlots) corner += __ldcg(src + (size_t)gg * WIN);
#pragma unroll
        for (int d = WIN; d < 32; d <<= 1) corner += __shfl_xor_sync(0xffffffffu, corner, d);
    }

    // ii(x, y0 - 1) = corner + prefix over the group's columns of V(x, y0 - 1);
    // column 4 * j + k of acc is column k of chunk j
    int acc[WIN][4 * NCH];
#pragma unroll
    for (int j = 0; j < NCH; ++j) {
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            uint32_t u[WIN / 2];
#pragma unroll
            for (int i = 0; i < WIN / 2; ++i) u[i] = 0;
            if (k < ch.ncol[j]) {
                const uint16_t* src = ws.carry + ((size_t)band * W + ch.x[j] + k) * WIN;
                if (WIN == 4) {
                    const uint2 a = __ldg(reinterpret_cast<const uint2*>(src));
                    u[0] = a.x;
                    u[1 % (WIN / 2)] = a.y;
                } else {
#pragma unroll
                    for (int q = 0; q < WIN / 8; ++q) {
                        const uint4 a = __ldg(reinterpret_cast<const uint4*>(src) + q);
                        u[4 * q] = a.x;
                        u[(4 * q + 1) % (WIN / 2)] = a.y;
                        u[(4 * q + 2) % (WIN / 2)] = a.z;
                        u[(4 * q + 3) % (WIN / 2)] = a.w;
                    }
                }
            }
#pragma unroll
            for (int b = 0; b < WIN; ++b) {
                const int v = (int)((u[b >> 1] >> (16 * (b & 1))) & 0xFFFFu);
                acc[b][4 * j + k] = k == 0 ? v : acc[b][4 * j + k - 1] + v;
            }
        }
    }
#pragma unroll
    for (int b = 0; b < WIN; ++b) {
        int off = (int)__shfl_sync(0xffffffffu, corner, b);
#pragma unroll
        for (int j = 0; j < NCH; ++j) {
            const int tot = acc[b][4 * j + 3];
            const int incl = (int)warp_incl_scan((uint32_t)tot, lane);
            const int o = off + incl - tot;
#pragma unroll
            for (int k = 0; k < 4; ++k) acc[b][4 * j + k] += o;
            off += __shfl_sync(0xffffffffu, incl, 31);  // all of this slice precedes the next
        }
    }
    __syncwarp();

    // rows of the band: ii(x, y) = ii(x, y-1) + RL(y) + (count in the row's
    // group columns up to x) = acc + base + in-chunk prefix
    const size_t plane = (size_t)H * W;
    OutT* out_row = ii + (size_t)lo * plane + (size_t)y0 * W + ch.x[0];
    for (int r = 0; r < nrows; ++r, out_row += W) {
        // P[j][k][m] byte e = count of bin lo+4m+e in columns 0..k of chunk j
        uint32_t P[NCH][4][NM];
#pragma unroll
        for (int j = 0; j < NCH; ++j) {
            const uint32_t w = st[r][lane][j];
            uint32_t run[NM];
#pragma unroll
            for (int m = 0; m < NM; ++m) run[m] = 0;
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                const int b = (int)byte_at(w, k);
#pragma unroll
                for (int m = 0; m < NM; ++m) {
                    run[m] += bit_or_zero((uint32_t)(8 * (b - lo - 4 * m)));
                    P[j][k][m] = run[m];
                }
            }
        }
        // E[j][m]: count in the group columns before chunk j of this lane, 8-bit
        // fields: slice 0's total is at most 128, and an exclusive prefix over
        // the lanes of a slice at most 124
        uint32_t E[NCH][NM];
#pragma unroll
        for (int m = 0; m < NM; ++m) {
            uint32_t before = 0;
#pragma unroll
            for (int j = 0; j < NCH; ++j) {
                const uint32_t incl = warp_incl_scan(P[j][3][m], lane);
                E[j][m] = before + incl - P[j][3][m];
                if (j + 1 < NCH) before += __shfl_sync(0xffffffffu, incl, 31);
            }
        }
        uint4 rl4[WIN / 4];
#pragma unroll
        for (int k = 0; k < WIN / 4; ++k) rl4[k] = reinterpret_cast<const uint4*>(rl_s[r])[k];
#pragma unroll
        for (int b = 0; b < WIN; ++b) {
            const int m = b >> 2, e = b & 3;
            const uint32_t rlv = e == 0 ? rl4[m].x : (e == 1 ? rl4[m].y : (e == 2 ? rl4[m].z : rl4[m].w));
#pragma unroll
            for (int j = 0; j < NCH; ++j) {
                const int base = (int)(rlv + byte_at(E[j][m], e));
#pragma unroll
                for (int k = 0; k < 4; ++k) acc[b][4 * j + k] += base + (int)byte_at(P[j][k][m], e);
            }
        }
        OutT* p = out_row;
#pragma unroll
        for (int b = 0; b < WIN; ++b, p += plane)
            if (b < wins)
#pragma unroll
                for (int j = 0; j < NCH; ++j)
                    if (ch.ncol[j] > 0) store_chunk<OutT>(p + kSlice * j, &acc[b][4 * j], ch.ncol[j], vec);
    }
}

// ---------------------------------------------------------------- single pass
constexpr int kOpRowsPerWarp = 2;

// Shared-memory slot of column x (0..127) of a group: lane x / 4 owns
// columns 4L..4L+3, so slot (x % 4) * 32 + x / 4 makes a warp's accesses to
// "column 4L + k" consecutive (no bank conflicts).
__device__ __forceinline__ int cslot(int x) { return (x & 3) * 32 + (x >> 2); }

struct OpWs {
    void* header;      // tag of the last launch (onepass.cuh)
    uint32_t* flags;   // [tile]            tag of the launch that published the tile's aggregates
    uint32_t* colagg;  // [band][NM][W]     column counts over the tile's rows, 8-bit fields
    uint16_t* rowagg;  // [y][group][WIN]   row counts over the tile's columns
    uint32_t* totagg;  // [band][group][WIN] tile totals
};

template <int WIN, int NW, typename OutT>
__global__ void __launch_bounds__(32 * NW)
    ii_onepass_kernel(const uint8_t* __restrict__ bins, int W, int H, int n_groups, int lo, int n_bins, bool vec,
                      OpWs ws, OutT* __restrict__ ii, unsigned int* status) {
    constexpr int NM = (WIN + 3) / 4, HW = kOpRowsPerWarp, R = HW * NW, NT = 32 * NW;
    static_assert(R <= 32, "a tile's column counts must fit 8-bit fields");
    static_assert(NT % WIN == 0, "every thread sums one bin of the corner");
    __shared__ uint32_t st[R][32];             // the tile's bins, 4 per lane and row
    __shared__ uint32_t colw[NW][NM][kSlice];  // per-warp column counts, 8-bit fields, by cslot
    __shared__ uint32_t vtop[2 * NM][kSlice];  // V at the tile top, 16-bit fields, by cslot:
                                               // word 2m bins 4m, 4m+2; word 2m+1 bins 4m+1, 4m+3
    __shared__ int rl_s[R][WIN];               // the tile rows' counts over the group
    __shared__ uint32_t rl16_s[R][WIN / 2];    // RL of the tile's rows, 16-bit fields (bins 2i, 2i + 1)
    __shared__ int rlpre_s[R][WIN];            // RL summed over the tile's rows above each row
    __shared__ int corner_s[WIN];
    __shared__ uint32_t tag_s;

    const int t = blockIdx.x;
    const int I = t / n_groups, g = t - I * n_groups;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int y_tile = I * R;
    const int y0 = y_tile + warp * HW;
    const int nrows = max(0, min(HW, H - y0));
    const int x0 = g * kSlice + 4 * lane;
    const int ncol = max(0, min(4, W - x0));
    const int wins = min(WIN, n_bins - lo);

    pdl_wait();
    if (tid == 0) tag_s = onepass::launch_tag(ws.header);
    if (tid < WIN) corner_s[tid] = 0;
    for (int e = tid; e < 2 * NM * kSlice; e += NT) (&vtop[0][0])[e] = 0;
    for (int e = tid; e < R * (WIN / 2); e += NT) (&rl16_s[0][0])[e] = 0;

    // ---- this warp's rows: stage the bins, count per column and per row
    {
        uint32_t v[HW];
#pragma unroll
        for (int k = 0; k < HW; ++k)
            v[k] = k < nrows ? load_chunk(bins + (size_t)(y0 + k) * W + x0, ncol, vec) : 0xFFFFFFFFu;
        uint32_t col[4][NM];
#pragma unroll
        for (int c = 0; c < 4; ++c)
#pragma unroll
            for (int m = 0; m < NM; ++m) col[c][m] = 0;
#pragma unroll
        for (int k = 0; k < HW; ++k) {
            uint32_t rowt[NM];
#pragma unroll
            for (int m = 0; m < NM; ++m) rowt[m] = 0;
#pragma unroll
            for (int c = 0; c < 4; ++c) {
                const int sh = 8 * ((int)byte_at(v[k], c) - lo);
#pragma unroll
                for (int m = 0; m < NM; ++m) {
                    const uint32_t oh = bit_or_zero((uint32_t)(sh - 32 * m));
                    col[c][m] += oh;
                    rowt[m] += oh;
                }
            }
#pragma unroll
            for (int m = 0; m < NM; ++m) {
                const uint32_t sum = __reduce_add_sync(0xffffffffu, rowt[m]);  // at most 128 per bin
                if (lane < 4 && 4 * m + lane < WIN) rl_s[warp * HW + k][4 * m + lane] = (int)byte_at(sum, lane);
            }
            st[warp * HW + k][lane] = v[k];
        }
#pragma unroll
        for (int m = 0; m < NM; ++m)
#pragma unroll
            for (int c = 0; c < 4; ++c) colw[warp][m][c * 32 + lane] = col[c][m];
    }
    __syncthreads();

    // ---- publish the tile's aggregates, then its flag
    const uint32_t tag = tag_s;
    for (int p = tid; p < NM * kSlice; p += NT) {
        const int m = p / kSlice, x = p - m * kSlice;
        uint32_t a = 0;
#pragma unroll
        for (int w2 = 0; w2 < NW; ++w2) a += colw[w2][m][cslot(x)];  // at most R <= 32 per field
        if (g * kSlice + x < W) ws.colagg[((size_t)I * NM + m) * W + g * kSlice + x] = a;
    }
    for (int e = tid; e < R * WIN; e += NT) {
        const int r = e / WIN, b = e - r * WIN;
        if (y_tile + r < H) ws.rowagg[((size_t)(y_tile + r) * n_groups + g) * WIN + b] = (uint16_t)rl_s[r][b];
    }
    if (tid < WIN) {
        int tot = 0;
#pragma unroll 8
        for (int r = 0; r < R; ++r) tot += rl_s[r][tid];
        ws.totagg[((size_t)I * n_groups + g) * WIN + tid] = (uint32_t)tot;
    }
    __syncthreads();  // every thread's aggregates are stored
    if (tid == 0) {
        __threadfence();  // ... and visible to the GPU before the flag
        onepass::st_release(ws.flags + t, tag);
    }

    // ---- wait for the tiles above and to the left (all of lower number): the first warp
    // checks their flags (a lane per flag, independent loads), then acquires
    if (warp == 0) {
        const int nd = (I + 1) * (g + 1) - 1;
        bool ok = true;
        for (int e0 = 0; e0 < nd; e0 += 8 * 32) {
            const uint64_t t0 = ptx::globaltimer_ns();
            while (true) {
                bool all = true;
#pragma unroll
                for (int k = 0; k < 8; ++k) {
                    const int e = e0 + k * 32 + lane;
                    if (e < nd) {
                        const int Ip = e / (g + 1), gp = e - Ip * (g + 1);
                        all &= onepass::ld_relaxed(ws.flags + (size_t)Ip * n_groups + gp) == tag;
                    }
                }
                if (__all_sync(0xffffffffu, all)) break;
                if (ptx::globaltimer_ns() - t0 > kWaitLimitNs) {
                    ok = false;
                    break;
                }
            }
        }
        asm volatile("fence.acq_rel.gpu;" ::: "memory");
        if (!ok) atomicOr(status, kStatusTimeout);
    }
    __syncthreads();
    // the last tile has seen every tile's flag, so every tile has read the old tag
    if (tid == 0 && t == (int)gridDim.x - 1) onepass::end_launch(ws.header, tag);
    pdl_trigger();

    // ---- carries from the aggregates (loads from L2, many in flight per thread)
    // The first RL and corner loads of this thread go out first, so that their latency
    // overlaps that of the V loads.
    constexpr int RL_NSL = NT / R;
    const int rl_r = tid % R, rl_sl0 = tid / R, rl_y = y_tile + rl_r;
    uint32_t rl_pf[WIN / 2];
#pragma unroll
    for (int i = 0; i < WIN / 2; ++i) rl_pf[i] = 0;
    if (rl_y < H && rl_sl0 < g) {
        const uint32_t* src =
            reinterpret_cast<const uint32_t*>(ws.rowagg + ((size_t)rl_y * n_groups + rl_sl0) * WIN);
        if (WIN == 4) {
            const uint2 v2 = __ldcg(reinterpret_cast<const uint2*>(src));
            rl_pf[0] = v2.x;
            rl_pf[1 % (WIN / 2)] = v2.y;
        } else {
#pragma unroll
            for (int q = 0; q < WIN / 8; ++q) {
                const uint4 v4 = __ldcg(reinterpret_cast<const uint4*>(src) + q);
                rl_pf[4 * q] = v4.x;
                rl_pf[(4 * q + 1) % (WIN / 2)] = v4.y;
                rl_pf[(4 * q + 2) % (WIN / 2)] = v4.z;
                rl_pf[(4 * q + 3) % (WIN / 2)] = v4.w;
            }
        }
    }
    const int n_corner = I * g;
    uint4 c_pf[2][WIN / 4];
#pragma unroll
    for (int u = 0; u < 2; ++u) {
        const int task = tid + u * NT;
#pragma unroll
        for (int qd = 0; qd < WIN / 4; ++qd) c_pf[u][qd] = make_uint4(0, 0, 0, 0);
        if (task < n_corner) {
            const int Ip = task / g, gp = task - Ip * g;
            const uint4* src = reinterpret_cast<const uint4*>(ws.totagg + ((size_t)Ip * n_groups + gp) * WIN);
#pragma unroll
            for (int qd = 0; qd < WIN / 4; ++qd) c_pf[u][qd] = __ldcg(src + qd);
        }
    }
    // V at the tile top: task (m, column quad q), the bands above split over NT / (32 NM)
    // slices; 8-bit fields widened to 16 (V <= H < 65536), slices added in shared memory
    {
        constexpr int NTASK = 32 * NM, NSL = NT / NTASK;
        static_assert(NT % NTASK == 0, "every thread takes one task and one slice of the bands");
        {
            const int task = tid % NTASK, s0 = tid / NTASK;
            const int m = task >> 5, q = task & 31;
            const int xg = g * kSlice + 4 * q;
            uint32_t even[4] = {0, 0, 0, 0}, odd[4] = {0, 0, 0, 0};
            for (int sl = s0; xg < W && sl < I; sl += NSL * 8) {
                uint32_t a[8][4];  // eight bands' loads in flight
#pragma unroll
                for (int u = 0; u < 8; ++u) {
                    const int Ip = sl + u * NSL;
                    const uint32_t* src = ws.colagg + ((size_t)Ip * NM + m) * W + xg;
                    if (Ip >= I) {
                        a[u][0] = a[u][1] = a[u][2] = a[u][3] = 0;
                    } else if (vec) {
                        const uint4 v4 = __ldcg(reinterpret_cast<const uint4*>(src));
                        a[u][0] = v4.x;
                        a[u][1] = v4.y;
                        a[u][2] = v4.z;
                        a[u][3] = v4.w;
                    } else {
#pragma unroll
                        for (int k = 0; k < 4; ++k) a[u][k] = xg + k < W ? __ldcg(src + k) : 0u;
                    }
                }
#pragma unroll
                for (int u = 0; u < 8; ++u)
#pragma unroll
                    for (int k = 0; k < 4; ++k) {
                        even[k] += a[u][k] & 0x00FF00FFu;
                        odd[k] += (a[u][k] >> 8) & 0x00FF00FFu;
                    }
            }
#pragma unroll
            for (int k = 0; k < 4; ++k) {  // packed 16-bit adds: no field passes H < 65536
                if (even[k]) atomicAdd(&vtop[2 * m][cslot(4 * q + k)], even[k]);
                if (odd[k]) atomicAdd(&vtop[2 * m + 1][cslot(4 * q + k)], odd[k]);
            }
        }
    }
    // RL of the tile's rows: task (row r, group slice), the groups to the left split over
    // NT / R slices; WIN 16-bit counts per (row, group) load as one vector
    {
        constexpr int NSL = RL_NSL;
        const int r = rl_r, sl0 = rl_sl0;
        const int y = rl_y;
        uint32_t acc[WIN / 2];
#pragma unroll
        for (int i = 0; i < WIN / 2; ++i) acc[i] = rl_pf[i];  // group sl0, loaded above
        if (y < H) {
            const uint16_t* row = ws.rowagg + (size_t)y * n_groups * WIN;
#pragma unroll 2
            for (int gp = sl0 + NSL; gp < g; gp += NSL) {
                const uint32_t* src = reinterpret_cast<const uint32_t*>(row + (size_t)gp * WIN);
                if (WIN == 4) {
                    const uint2 v2 = __ldcg(reinterpret_cast<const uint2*>(src));
                    acc[0] += v2.x;
                    acc[1 % (WIN / 2)] += v2.y;
                } else {
#pragma unroll
                    for (int q = 0; q < WIN / 8; ++q) {
                        const uint4 v4 = __ldcg(reinterpret_cast<const uint4*>(src) + q);
                        acc[4 * q] += v4.x;
                        acc[(4 * q + 1) % (WIN / 2)] += v4.y;
                        acc[(4 * q + 2) % (WIN / 2)] += v4.z;
                        acc[(4 * q + 3) % (WIN / 2)] += v4.w;
                    }
                }
            }
        }
#pragma unroll
        for (int i = 0; i < WIN / 2; ++i)  // a row holds at most W < 65536 of a bin
            if (acc[i]) atomicAdd(&rl16_s[r][i], acc[i]);
    }
    // corner: the totals of the tiles above-left, task (band, group), warp sums per bin
    {
        int acc[WIN];
#pragma unroll
        for (int b = 0; b < WIN; ++b) acc[b] = 0;
#pragma unroll
        for (int u = 0; u < 2; ++u)  // the two tasks loaded above
#pragma unroll
            for (int qd = 0; qd < WIN / 4; ++qd) {
                acc[4 * qd] += (int)c_pf[u][qd].x;
                acc[4 * qd + 1] += (int)c_pf[u][qd].y;
                acc[4 * qd + 2] += (int)c_pf[u][qd].z;
                acc[4 * qd + 3] += (int)c_pf[u][qd].w;
            }
        const int n = n_corner;
        for (int task = tid + 2 * NT; task < n; task += NT) {
            const int Ip = task / g, gp = task - Ip * g;
            const uint4* src = reinterpret_cast<const uint4*>(ws.totagg + ((size_t)Ip * n_groups + gp) * WIN);
#pragma unroll
            for (int q = 0; q < WIN / 4; ++q) {
                const uint4 v4 = __ldcg(src + q);
                acc[4 * q] += (int)v4.x;
                acc[4 * q + 1] += (int)v4.y;
                acc[4 * q + 2] += (int)v4.z;
                acc[4 * q + 3] += (int)v4.w;
            }
        }
#pragma unroll
        for (int b = 0; b < WIN; ++b) {
            int v = acc[b];
#pragma unroll
            for (int d = 16; d > 0; d >>= 1) v += __shfl_xor_sync(0xffffffffu, v, d);
            if (lane == 0 && v != 0) atomicAdd(&corner_s[b], v);
        }
    }
    __syncthreads();
    // RL summed over the rows above each row of the tile (independent loads, one task per (row, bin))
    for (int e = tid; e < R * WIN; e += NT) {
        const int r = e / WIN, b = e - r * WIN;
        int sum = 0;
#pragma unroll
        for (int r2 = 0; r2 < R - 1; ++r2)
            if (r2 < r) sum += (int)((rl16_s[r2][b >> 1] >> (16 * (b & 1))) & 0xFFFFu);
        rlpre_s[r][b] = sum;
    }
    // the column counts of the warps above each warp, in place (8-bit fields: at most 2 (NW - 1)
    // rows): one task per (word, column), a running sum down the warps
    for (int e = tid; e < NM * kSlice; e += NT) {
        const int m = e / kSlice, sl = e - m * kSlice;
        uint32_t run = 0;
#pragma unroll
        for (int w2 = 0; w2 < NW; ++w2) {
            const uint32_t a = colw[w2][m][sl];
            colw[w2][m][sl] = run;
            run += a;
        }
    }
    __syncthreads();

    // ---- this warp's rows: ii(x, y0 - 1) = corner of the rows above + prefix of V over the columns
    int acc[WIN][4];
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        const int sl = k * 32 + lane;  // cslot(4 * lane + k)
#pragma unroll
        for (int m = 0; m < NM; ++m) {
            uint32_t even = vtop[2 * m][sl], odd = vtop[2 * m + 1][sl];
            const uint32_t a = colw[warp][m][sl];  // the counts of the warps above this one
            even += a & 0x00FF00FFu;
            odd += (a >> 8) & 0x00FF00FFu;
            const int vb[4] = {(int)(even & 0xFFFFu), (int)(odd & 0xFFFFu), (int)(even >> 16), (int)(odd >> 16)};
#pragma unroll
            for (int e = 0; e < 4; ++e) {
                const int b = 4 * m + e;
                if (b < WIN) acc[b][k] = k == 0 ? vb[e] : acc[b][k - 1] + vb[e];
            }
        }
    }
#pragma unroll
    for (int b = 0; b < WIN; ++b) {
        const int corner = corner_s[b] + rlpre_s[warp * HW][b];
        const int tot = acc[b][3];
        const int incl = (int)warp_incl_scan((uint32_t)tot, lane);
        const int o = corner + incl - tot;
#pragma unroll
        for (int k = 0; k < 4; ++k) acc[b][k] += o;
    }

    const size_t plane = (size_t)H * W;
    OutT* out_row = ii + (size_t)lo * plane + (size_t)y0 * W + x0;
    for (int r = 0; r < nrows; ++r, out_row += W) {
        // P[k][m] byte e = count of bin lo+4m+e in columns 0..k of this lane's chunk
        const uint32_t w = st[warp * HW + r][lane];
        uint32_t P[4][NM], run[NM];
#pragma unroll
        for (int m = 0; m < NM; ++m) run[m] = 0;
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            const int b = (int)byte_at(w, k);
#pragma unroll
            for (int m = 0; m < NM; ++m) {
                run[m] += bit_or_zero((uint32_t)(8 * (b - lo - 4 * m)));
                P[k][m] = run[m];
            }
        }
        // E[m]: count in the group's columns left of this lane (8-bit fields: at most 124)
        uint32_t E[NM];
#pragma unroll
        for (int m = 0; m < NM; ++m) E[m] = warp_incl_scan(P[3][m], lane) - P[3][m];
#pragma unroll
        for (int b = 0; b < WIN; ++b) {
            const int m = b >> 2, e = b & 3;
            const int base = (int)((rl16_s[warp * HW + r][b >> 1] >> (16 * (b & 1))) & 0xFFFFu) +
                             (int)byte_at(E[m], e);
#pragma unroll
            for (int k = 0; k < 4; ++k) acc[b][k] += base + (int)byte_at(P[k][m], e);
        }
        if (ncol > 0) {
            OutT* p = out_row;
#pragma unroll
            for (int b = 0; b < WIN; ++b, p += plane)
                if (b < wins) store_chunk<OutT>(p, acc[b], ncol, vec);
        }
    }
}

// ---------------------------------------------------------------- cluster pass
// One thread-block cluster per 128-column group, its CTAs stacked down the
// image (rank k owns rows k R .. k R + R - 1, R = HW rows per warp x NW
// warps, at most 16 CTAs per cluster, so images up to 16 R rows).  Nothing
// is published to global memory and no CTA waits on a flag:
//   V(x, tile top - 1)  the column counts of the CTAs above in the cluster,
//                       read from their shared memory (distributed shared
//                       memory) after one cluster barrier;
//   RL(y)               counted by the CTA itself from the bins left of the
//                       group in its own rows (the bin map is one byte per
//                       pixel, so this is a short read);
//   corner              the sums of RL over the rows of the CTAs above,
//                       read the same way as V.
// A second cluster barrier, arrived at after the reads and waited on at the
// very end, keeps every CTA's shared memory alive until its peers are done
// reading it.  Inside a CTA, warp w owns HW rows and the scan of each row is
// that of the single pass.

__device__ __forceinline__ uint32_t cl_rank() {
    uint32_t r;
    asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
    return r;
}
__device__ __forceinline__ uint32_t cl_ld(const void* local, uint32_t rank) {
    uint32_t a, v;
    asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(a) : "r"(ptx::smem_addr(local)), "r"(rank));
    asm volatile("ld.shared::cluster.u32 %0, [%1];" : "=r"(v) : "r"(a) : "memory");
    return v;
}
__device__ __forceinline__ void cl_arrive() { asm volatile("barrier.cluster.arrive.release.aligned;" ::: "memory"); }
__device__ __forceinline__ void cl_wait() { asm volatile("barrier.cluster.wait.acquire.aligned;" ::: "memory"); }

constexpr int kClMaxCtas = 16;   // CTAs per cluster at most (non-portable size)
constexpr int kClMaxGroups = 63; // groups left of a tile: 4 per lane and row in 8-bit fields
// Warps per CTA at most: 20 of 2 rows (one CTA per SM), else 10 (two CTAs per SM,
// so that a cluster packs into fewer SMs).
__host__ __device__ constexpr int cl_max_warps(int HW) { return HW == 2 ? 20 : 10; }

// One-hot counts of the 4 bins in w in 4-bit fields (bin lo + k in bits 4k .. 4k + 3;
// bins outside lo .. lo + 7, and 0xFF, shift out of the word).
__device__ __forceinline__ uint32_t onehot4(uint32_t w, int lo) {
    uint32_t n = 0;
#pragma unroll
    for (int c = 0; c < 4; ++c) n += bit_or_zero(4u * (byte_at(w, c) - (uint32_t)lo));
    return n;
}

// 4 nibbles (bits 16h .. 16h + 15 of x) spread to the 4 bytes of a word.
__device__ __forceinline__ uint32_t nibbles_to_bytes(uint32_t x, int h) {
    uint32_t a = (x >> (16 * h)) & 0xFFFFu;
    a = (a | (a << 8)) & 0x00FF00FFu;
    return (a | (a << 4)) & 0x0F0F0F0Fu;
}

// Shared-memory layout of the cluster kernel (32-bit words), for NW warps of HW rows.
struct ClSmem {
    int st, colw, colcnt, vtop, rl, rlpre, rltile, corner, words;
    __host__ __device__ ClSmem(int HW, int NW, int WIN) {
        const int NM = (WIN + 3) / 4, R = HW * NW;
        st = 0;                         // [R][32]        the tile's bins, 4 per lane and row
        colw = st + R * 32;             // [NW][NM][128]  per-warp column counts, then their prefix over warps
        colcnt = colw + NW * NM * 128;  // [NM][128]      the CTA's column counts (read by the CTAs below)
        vtop = colcnt + NM * 128;       // [2 NM][128]    V at the tile top, 16-bit fields
        rl = vtop + 2 * NM * 128;       // [R][WIN]       RL of each row
        rlpre = rl + R * WIN;           // [R][WIN]       RL summed over the tile's rows above
        rltile = rlpre + R * WIN;       // [WIN]          RL summed over the tile (read by the CTAs below)
        corner = rltile + WIN;          // [WIN]
        words = corner + WIN;
    }
};

template <int WIN, int HW, typename OutT>
__global__ void __launch_bounds__(32 * cl_max_warps(HW), HW == 2 ? 1 : 2)
    ii_cluster_kernel(const uint8_t* __restrict__ bins, int W, int H, int lo, int n_bins, bool vec,
                      OutT* __restrict__ ii) {
    static_assert(WIN <= 8, "the 4-bit one-hot counts hold 8 bins");
    constexpr int NM = (WIN + 3) / 4, MAXW = cl_max_warps(HW);
    extern __shared__ __align__(16) uint32_t sm[];
    const int NW = (int)blockDim.x >> 5, NT = (int)blockDim.x, R = HW * NW;
    const ClSmem L(HW, NW, WIN);
    uint32_t* st = sm + L.st;
    uint32_t* colw = sm + L.colw;
    uint32_t* colcnt = sm + L.colcnt;
    uint32_t* vtop = sm + L.vtop;
    int* rl = reinterpret_cast<int*>(sm + L.rl);
    int* rlpre = reinterpret_cast<int*>(sm + L.rlpre);
    int* rltile = reinterpret_cast<int*>(sm + L.rltile);
    int* corner = reinterpret_cast<int*>(sm + L.corner);

    const int g = blockIdx.x;
    const int k = (int)cl_rank();
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int y_tile = k * R;
    const int y0 = y_tile + warp * HW;
    const int nrows = max(0, min(HW, H - y0));
    const int x0 = g * kSlice + 4 * lane;
    const int ncol = max(0, min(4, W - x0));
    const int wins = min(WIN, n_bins - lo);

    pdl_wait();
    // ---- this warp's rows: the bins of the group, then RL from the bins left of it
    uint32_t v[HW];
#pragma unroll
    for (int r = 0; r < HW; ++r)
        v[r] = r < nrows ? load_chunk(bins + (size_t)(y0 + r) * W + x0, ncol, vec) : 0xFFFFFFFFu;
    {
        // per row, 8-bit fields: ae byte i = bin lo + 2i, ao byte i = bin lo + 2i + 1 (at most
        // 4 g <= 252 per lane); 4-bit sums of 3 words (at most 12) are folded in
        uint32_t ae[HW], ao[HW];
#pragma unroll
        for (int r = 0; r < HW; ++r) ae[r] = ao[r] = 0;
        for (int j0 = 0; j0 < g; j0 += 3) {  // 3 x HW loads in flight; every column left of the group exists
            uint32_t wv[HW][3];
#pragma unroll
            for (int r = 0; r < HW; ++r)
#pragma unroll
                for (int u = 0; u < 3; ++u)
                    wv[r][u] = r < nrows && j0 + u < g
                                   ? load_chunk(bins + (size_t)(y0 + r) * W + kSlice * (j0 + u) + 4 * lane, 4, vec)
                                   : 0xFFFFFFFFu;
#pragma unroll
            for (int r = 0; r < HW; ++r) {
                const uint32_t n4 = onehot4(wv[r][0], lo) + onehot4(wv[r][1], lo) + onehot4(wv[r][2], lo);
                ae[r] += n4 & 0x0F0F0F0Fu;
                ao[r] += (n4 >> 4) & 0x0F0F0F0Fu;
            }
        }
#pragma unroll
        for (int r = 0; r < HW; ++r) {  // 16-bit fields for the warp sums: a row holds at most W < 65536
            // bins lo + {0, 4}, {2, 6}, {1, 5}, {3, 7}
            const uint32_t s0 = __reduce_add_sync(0xffffffffu, ae[r] & 0x00FF00FFu);
            const uint32_t s2 = __reduce_add_sync(0xffffffffu, (ae[r] >> 8) & 0x00FF00FFu);
            const uint32_t s1 = __reduce_add_sync(0xffffffffu, ao[r] & 0x00FF00FFu);
            const uint32_t s3 = __reduce_add_sync(0xffffffffu, (ao[r] >> 8) & 0x00FF00FFu);
            if (lane < WIN) {
                const int q = lane & 3;
                const uint32_t f = q == 0 ? s0 : (q == 1 ? s1 : (q == 2 ? s2 : s3));
                rl[(warp * HW + r) * WIN + lane] = (int)((f >> (16 * (lane >> 2))) & 0xFFFFu);
            }
        }
    }
    {
        uint32_t col4[4] = {0, 0, 0, 0};  // 4-bit fields: at most HW <= 8 per column
#pragma unroll
        for (int r = 0; r < HW; ++r) {
#pragma unroll
            for (int c = 0; c < 4; ++c) col4[c] += bit_or_zero(4u * (byte_at(v[r], c) - (uint32_t)lo));
            st[(warp * HW + r) * 32 + lane] = v[r];
        }
#pragma unroll
        for (int m = 0; m < NM; ++m)
#pragma unroll
            for (int c = 0; c < 4; ++c) colw[(warp * NM + m) * kSlice + c * 32 + lane] = nibbles_to_bytes(col4[c], m);
    }
    __syncthreads();

    // ---- the CTA's aggregates: column counts (and each warp's prefix over the warps above),
    // RL summed over the rows above each row and over the tile
    for (int e = tid; e < NM * kSlice; e += NT) {
        uint32_t a[MAXW];
#pragma unroll
        for (int w2 = 0; w2 < MAXW; ++w2) a[w2] = w2 < NW ? colw[w2 * NM * kSlice + e] : 0u;
        uint32_t run = 0;  // at most R <= 80 per 8-bit field
#pragma unroll
        for (int w2 = 0; w2 < MAXW; ++w2)
            if (w2 < NW) {
                colw[w2 * NM * kSlice + e] = run;
                run += a[w2];
            }
        colcnt[e] = run;
    }
    for (int b = warp; b < WIN; b += NW) {  // lane L: rows 4L .. 4L + 3 (R <= 80)
        int rv[4], tot = 0;
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const int r = 4 * lane + q;
            rv[q] = r < R ? rl[r * WIN + b] : 0;
            tot += rv[q];
        }
        const int incl = (int)warp_incl_scan((uint32_t)tot, lane);
        int ex = incl - tot;
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const int r = 4 * lane + q;
            if (r < R) rlpre[r * WIN + b] = ex;
            ex += rv[q];
        }
        if (lane == 31) rltile[b] = incl;
    }
    cl_arrive();  // this CTA's aggregates are ready (release) ...
    cl_wait();    // ... and so are those of every CTA of the cluster (acquire)

    // ---- carries from the CTAs above: V (per column, widened to 16-bit fields) and the corner
    for (int e = tid; e < NM * kSlice; e += NT) {
        uint32_t a[kClMaxCtas - 1];
#pragma unroll
        for (int q = 0; q < kClMaxCtas - 1; ++q) a[q] = q < k ? cl_ld(colcnt + e, (uint32_t)q) : 0u;
        uint32_t even = 0, odd = 0;  // packed 16-bit adds: no field passes H < 65536
#pragma unroll
        for (int q = 0; q < kClMaxCtas - 1; ++q) {
            even += a[q] & 0x00FF00FFu;
            odd += (a[q] >> 8) & 0x00FF00FFu;
        }
        const int m = e / kSlice, sl = e - m * kSlice;
        vtop[(2 * m) * kSlice + sl] = even;
        vtop[(2 * m + 1) * kSlice + sl] = odd;
    }
    if (tid >= NT - WIN) {
        const int b = tid - (NT - WIN);
        int c = 0;
        for (int q = 0; q < k; ++q) c += (int)cl_ld(rltile + b, (uint32_t)q);
        corner[b] = c;
    }
    cl_arrive();  // done reading the other CTAs' shared memory (waited on before exit)
    __syncthreads();
    pdl_trigger();

    // ---- this warp's rows: ii(x, y0 - 1) = corner + RL above + prefix of V over the columns
    int acc[WIN][4];
#pragma unroll
    for (int c = 0; c < 4; ++c) {
        const int sl = c * 32 + lane;  // cslot(4 * lane + c)
#pragma unroll
        for (int m = 0; m < NM; ++m) {
            uint32_t even = vtop[(2 * m) * kSlice + sl], odd = vtop[(2 * m + 1) * kSlice + sl];
            const uint32_t a = colw[(warp * NM + m) * kSlice + sl];  // the counts of the warps above this one
            even += a & 0x00FF00FFu;
            odd += (a >> 8) & 0x00FF00FFu;
            const int vb[4] = {(int)(even & 0xFFFFu), (int)(odd & 0xFFFFu), (int)(even >> 16), (int)(odd >> 16)};
#pragma unroll
            for (int e = 0; e < 4; ++e) {
                const int b = 4 * m + e;
                if (b < WIN) acc[b][c] = c == 0 ? vb[e] : acc[b][c - 1] + vb[e];
            }
        }
    }
#pragma unroll
    for (int b = 0; b < WIN; ++b) {
        const int cb = corner[b] + rlpre[(warp * HW) * WIN + b];
        const int tot = acc[b][3];
        const int incl = (int)warp_incl_scan((uint32_t)tot, lane);
        const int o = cb + incl - tot;
#pragma unroll
        for (int c = 0; c < 4; ++c) acc[b][c] += o;
    }

    const size_t plane = (size_t)H * W;
    OutT* out_row = ii + (size_t)lo * plane + (size_t)y0 * W + x0;
#pragma unroll
    for (int r = 0; r < HW; ++r, out_row += W) {
        if (r >= nrows) break;
        const uint32_t w = st[(warp * HW + r) * 32 + lane];
        uint32_t P[4][NM], run[NM];
#pragma unroll
        for (int m = 0; m < NM; ++m) run[m] = 0;
#pragma unroll
        for (int c = 0; c < 4; ++c) {
            const uint32_t sh = 8u * (byte_at(w, c) - (uint32_t)lo);
#pragma unroll
            for (int m = 0; m < NM; ++m) {
                run[m] += bit_or_zero(sh - 32u * m);
                P[c][m] = run[m];
            }
        }
        uint32_t E[NM];  // count in the group's columns left of this lane (8-bit fields: at most 124)
#pragma unroll
        for (int m = 0; m < NM; ++m) E[m] = warp_incl_scan(P[3][m], lane) - P[3][m];
#pragma unroll
        for (int b = 0; b < WIN; ++b) {
            const int m = b >> 2, e = b & 3;
            const int base = rl[(warp * HW + r) * WIN + b] + (int)byte_at(E[m], e);
#pragma unroll
            for (int c = 0; c < 4; ++c) acc[b][c] += base + (int)byte_at(P[c][m], e);
        }
        if (ncol > 0) {
            OutT* p = out_row;
#pragma unroll
            for (int b = 0; b < WIN; ++b, p += plane)
                if (b < wins) store_chunk<OutT>(p, acc[b], ncol, vec);
        }
    }
    cl_wait();  // every CTA of the cluster has read what it needed from this one
}

template <int WIN, typename OutT>
hog_status run_window(const Plan& p, const uint8_t* bins, int n_bins, int lo, OutT* ii, const Ws& ws, bool vec,
                      cudaStream_t st) {
    const int tiles = p.n_bands * p.n_groups;
    hog_status s = launch_pdl(ii_tile_reduce_kernel<WIN>, dim3(tiles), dim3(32), 0, st, bins, p.W, p.H, p.h,
                              p.n_bands, p.n_groups, lo, vec, ws);
    if (s != HOG_OK) return s;
    const int na = ceil_div(p.W, 32);
    const int nbb = ceil_div((long)p.n_groups * WIN, 32);
    const int nc = ceil_div(p.H, kCarryThreads / 32);
    s = launch_pdl(ii_carry_kernel<WIN>, dim3(na + nbb + nc), dim3(kCarryThreads), 0, st, p.W, p.H, p.n_bands,
                   p.n_groups, na, nbb, ws);
    if (s != HOG_OK) return s;
    return launch_pdl(ii_tile_scan_kernel<WIN, OutT>, dim3(tiles), dim3(32), 0, st, bins, p.W, p.H, p.h,
                      p.n_groups, lo, n_bins, vec, ws, ii);
}

template <typename OutT>
hog_status run_all(const Plan& p, const uint8_t* bins, int n_bins, OutT* ii, const Ws& ws, bool vec,
                   cudaStream_t st) {
    for (int wi = 0; wi < p.n_windows; ++wi) {
        const int lo = wi * p.win;
        hog_status s = p.win == 4   ? run_window<4, OutT>(p, bins, n_bins, lo, ii, ws, vec, st)
                       : p.win == 8 ? run_window<8, OutT>(p, bins, n_bins, lo, ii, ws, vec, st)
                                    : run_window<16, OutT>(p, bins, n_bins, lo, ii, ws, vec, st);
        if (s != HOG_OK) return s;
    }
    return HOG_OK;
}

// ---- workspace: [sync region: tag word, one flag per single-pass tile]
//                 [either the three-phase arrays or the single-pass aggregates]
// The sync region is the only part that must start zero-filled; nothing else
// writes into it, so the two paths can share one workspace.
constexpr int kOpMinRows = 16;  // the shorter single-pass tile (8 warps of 2 rows)

struct OpPlan {
    int R, n_bands, n_groups, n_tiles, win, n_windows;
};

OpPlan op_plan(int W, int H, int n_bins, int R) {
    OpPlan o{};
    o.R = R;
    o.n_bands = ceil_div(H, R);
    o.n_groups = ceil_div(W, kSlice);
    o.n_tiles = o.n_bands * o.n_groups;
    o.win = n_bins <= 4 ? 4 : (n_bins <= 8 ? 8 : 16);
    o.n_windows = ceil_div(n_bins, o.win);
    return o;
}

size_t sync_bytes(int W, int H) {
    const OpPlan o = op_plan(W, H, 1, kOpMinRows);  // the most tiles
    return align256((size_t)onepass::kHeaderBytes + (size_t)o.n_tiles * 4);
}

size_t op_agg_bytes(int W, int H, int n_bins) {
    const OpPlan o = op_plan(W, H, n_bins, kOpMinRows);
    const int nm = (o.win + 3) / 4;
    return align256((size_t)o.n_bands * nm * W * 4) + align256((size_t)H * o.n_groups * o.win * 2) +
           align256((size_t)o.n_bands * o.n_groups * o.win * 4);
}

OpWs op_carve(const OpPlan& o, int W, int H, void* base) {
    uint8_t* b = static_cast<uint8_t*>(base);
    OpWs w;
    w.header = b;
    w.flags = reinterpret_cast<uint32_t*>(b + onepass::kHeaderBytes);
    b += sync_bytes(W, H);
    const int nm = (o.win + 3) / 4;
    w.colagg = reinterpret_cast<uint32_t*>(b);
    b += align256((size_t)o.n_bands * nm * W * 4);
    w.rowagg = reinterpret_cast<uint16_t*>(b);
    b += align256((size_t)H * o.n_groups * o.win * 2);
    w.totagg = reinterpret_cast<uint32_t*>(b);
    return w;
}

template <int WIN, typename OutT>
hog_status op_window(const OpPlan& o, const uint8_t* bins, int W, int H, int n_bins, int lo, OutT* ii,
                     const OpWs& ws, bool vec, unsigned int* status, cudaStream_t st) {
    if (o.R == 32)
        return launch_pdl(ii_onepass_kernel<WIN, 16, OutT>, dim3(o.n_tiles), dim3(512), 0, st, bins, W, H,
                          o.n_groups, lo, n_bins, vec, ws, ii, status);
    return launch_pdl(ii_onepass_kernel<WIN, 8, OutT>, dim3(o.n_tiles), dim3(256), 0, st, bins, W, H, o.n_groups,
                      lo, n_bins, vec, ws, ii, status);
}

template <typename OutT>
hog_status op_all(const OpPlan& o, const uint8_t* bins, int W, int H, int n_bins, OutT* ii, const OpWs& ws,
                  bool vec, unsigned int* status, cudaStream_t st) {
    for (int wi = 0; wi < o.n_windows; ++wi) {
        const int lo = wi * o.win;
        hog_status s = o.win == 4   ? op_window<4, OutT>(o, bins, W, H, n_bins, lo, ii, ws, vec, status, st)
                       : o.win == 8 ? op_window<8, OutT>(o, bins, W, H, n_bins, lo, ii, ws, vec, status, st)
                                    : op_window<16, OutT>(o, bins, W, H, n_bins, lo, ii, ws, vec, status, st);
        if (s != HOG_OK) return s;
    }
    return HOG_OK;
}

// ---- cluster pass: geometry, co-scheduling check, launch
// Bins per launch: at most 8 (16 would keep 64 accumulators per thread and spill).
inline int cl_win(int n_bins) { return n_bins <= 4 ? 4 : 8; }

struct ClPlan {
    int HW, NW, CL, n_groups;
    size_t smem;
};

// Rows per warp: `want` (2, 4 or 8) if given, else the fewest that cover H
// with at most 16 CTAs; false if no shape does or the group is too far right.
bool cl_plan(int W, int H, int win, int want, ClPlan* p) {
    const int n_groups = ceil_div(W, kSlice);
    if (n_groups - 1 > kClMaxGroups) return false;
    for (int hw : {2, 4, 8}) {
        if (want != 0 && hw != want) continue;
        int nw = ceil_div(H, hw * kClMaxCtas);
        nw = nw < 1 ? 1 : nw;
        if (nw > cl_max_warps(hw)) continue;
        p->HW = hw;
        p->NW = nw;
        p->CL = ceil_div(H, hw * nw);
        p->n_groups = n_groups;
        p->smem = (size_t)ClSmem(hw, nw, win).words * 4;
        return true;
    }
    return false;
}

template <int WIN, int HW, typename OutT>
cudaLaunchConfig_t cl_config(const ClPlan& c, cudaStream_t st, cudaLaunchAttribute* attr) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(c.n_groups, c.CL);
    cfg.blockDim = dim3(32 * c.NW);
    cfg.dynamicSmemBytes = c.smem;
    cfg.stream = st;
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    attr[1].id = cudaLaunchAttributeClusterDimension;
    attr[1].val.clusterDim.x = 1;
    attr[1].val.clusterDim.y = c.CL;
    attr[1].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 2;
    return cfg;
}

template <int WIN, int HW, typename OutT>
cudaError_t cl_attributes(const ClPlan& c) {
    // clusters of up to 16 CTAs: allowed once per kernel and device, before its first launch
    static std::atomic<int> nonportable[64];
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= 64 || nonportable[dev].load(std::memory_order_acquire) == 0) {
        e = cudaFuncSetAttribute(ii_cluster_kernel<WIN, HW, OutT>, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
        if (e != cudaSuccess) return e;
        if (dev >= 0 && dev < 64) nonportable[dev].store(1, std::memory_order_release);
    }
    return smem_at_least<ii_cluster_kernel<WIN, HW, OutT>>(c.smem);
}

// How many clusters of this shape can be resident on the current device at
// once (a cluster's CTAs must all fit the SMs of one GPC); 0 if none can.
// Remembered per device and shape.
template <int WIN, int HW, typename OutT>
int cl_active_t(const ClPlan& c) {
    static std::mutex mu;
    static std::map<std::tuple<int, int, int>, int> seen;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return 0;
    const auto key = std::make_tuple(dev, c.NW, c.CL);
    std::lock_guard<std::mutex> lock(mu);
    auto it = seen.find(key);
    if (it != seen.end()) return it->second;
    int n = 0;
    if (cl_attributes<WIN, HW, OutT>(c) == cudaSuccess) {
        cudaLaunchAttribute attr[2];
        cudaLaunchConfig_t cfg = cl_config<WIN, HW, OutT>(c, nullptr, attr);
        if (cudaOccupancyMaxActiveClusters(&n, ii_cluster_kernel<WIN, HW, OutT>, &cfg) != cudaSuccess) n = 0;
    }
    cudaGetLastError();  // a refused query leaves no error behind
    seen[key] = n;
    return n;
}

template <int WIN, typename OutT>
int cl_active_w(const ClPlan& c) {
    return c.HW == 2 ? cl_active_t<WIN, 2, OutT>(c)
                     : (c.HW == 4 ? cl_active_t<WIN, 4, OutT>(c) : cl_active_t<WIN, 8, OutT>(c));
}

template <typename OutT>
int cl_active(const ClPlan& c, int win) {
    return win == 4 ? cl_active_w<4, OutT>(c) : cl_active_w<8, OutT>(c);
}

template <int WIN, int HW, typename OutT>
hog_status cl_launch_t(const ClPlan& c, const uint8_t* bins, int W, int H, int lo, int n_bins, bool vec, OutT* ii,
                       cudaStream_t st) {
    cudaError_t e = cl_attributes<WIN, HW, OutT>(c);
    if (e != cudaSuccess) return cuda_fail(e);
    cudaLaunchAttribute attr[2];
    cudaLaunchConfig_t cfg = cl_config<WIN, HW, OutT>(c, st, attr);
    e = cudaLaunchKernelEx(&cfg, ii_cluster_kernel<WIN, HW, OutT>, bins, W, H, lo, n_bins, vec, ii);
    return e == cudaSuccess ? HOG_OK : cuda_fail(e);
}

template <typename OutT>
hog_status cl_all(const ClPlan& c, const uint8_t* bins, int W, int H, int n_bins, int win, bool vec, OutT* ii,
                  cudaStream_t st) {
    for (int lo = 0; lo < n_bins; lo += win) {
        hog_status s;
        if (c.HW == 2)
            s = win == 4 ? cl_launch_t<4, 2, OutT>(c, bins, W, H, lo, n_bins, vec, ii, st)
                         : cl_launch_t<8, 2, OutT>(c, bins, W, H, lo, n_bins, vec, ii, st);
        else if (c.HW == 4)
            s = win == 4 ? cl_launch_t<4, 4, OutT>(c, bins, W, H, lo, n_bins, vec, ii, st)
                         : cl_launch_t<8, 4, OutT>(c, bins, W, H, lo, n_bins, vec, ii, st);
        else
            s = win == 4 ? cl_launch_t<4, 8, OutT>(c, bins, W, H, lo, n_bins, vec, ii, st)
                         : cl_launch_t<8, 8, OutT>(c, bins, W, H, lo, n_bins, vec, ii, st);
        if (s != HOG_OK) return s;
    }
    return HOG_OK;
}

constexpr int kClDefaultRows = 640;  // the library takes the cluster pass up to this image height

// The cluster pass for this call, if it applies and a cluster of its shape
// fits the device.  Forced by the tuning knob, it takes any image it can
// cover.  The library's own choice (measured): images up to 640 rows and 8
// bins, with 2 rows per warp when every cluster can be resident at once,
// else 4 (two CTAs per SM); past that, three launches are as fast or faster.
bool use_cluster(int W, int H, int n_bins, int ii_dtype, ClPlan* c) {
    const int path = tune_get(HOG_TUNE_INTEGRAL_PATH);
    if (path != 3 && path != 0) return false;
    const int win = cl_win(n_bins);
    const int want = tune_get(HOG_TUNE_INTEGRAL_WARP_ROWS);
    auto active = [&](const ClPlan& p) {
        return ii_dtype == HOG_U16 ? cl_active<uint16_t>(p, win) : cl_active<int32_t>(p, win);
    };
    if (path == 3) return cl_plan(W, H, win, want, c) && active(*c) >= 1;
    if (H > kClDefaultRows || n_bins > 8) return false;
    for (int hw : {2, 4}) {
        if (want != 0 && hw != want) continue;
        if (cl_plan(W, H, win, hw, c) && active(*c) >= c->n_groups) return true;
    }
    return false;
}

// Whether the single pass is the library's choice where the cluster pass is
// not: never.  Alone on the GPU it beats three launches only on small images
// (about 1.4 us up to 640 x 360), which the cluster pass takes; with many
// streams sharing the GPU its tiles wait on tiles that other kernels keep off
// the SMs (a request server's throughput fell to a third in some runs), so
// it runs only when the tuning knob asks for it.
bool onepass_default(int W, int H) {
    (void)W;
    (void)H;
    return false;
}

}  // namespace

size_t integral_sync_bytes(int W, int H) { return sync_bytes(W, H); }

bool integral_uses_sync(int W, int H, int n_bins, int ii_dtype) {
    ClPlan c{};
    if (use_cluster(W, H, n_bins, ii_dtype, &c)) return false;
    const int path = tune_get(HOG_TUNE_INTEGRAL_PATH);
    return path == 2 || (path == 0 && onepass_default(W, H));
}

int integral_launches(int W, int H, int n_bins) {
    const int path = tune_get(HOG_TUNE_INTEGRAL_PATH);
    ClPlan c{};
    if (use_cluster(W, H, n_bins, HOG_I32, &c)) return ceil_div(n_bins, cl_win(n_bins));
    const bool one = path == 2 || (path == 0 && onepass_default(W, H));
    const int win = n_bins <= 4 ? 4 : (n_bins <= 8 ? 8 : 16);
    return (one ? 1 : 3) * ceil_div(n_bins, win);
}

size_t integral_workspace_bytes(int W, int H, int n_bins) {
    // enough for every band height and both paths, so a workspace stays valid whatever the tuning
    size_t most = op_agg_bytes(W, H, n_bins);
    for (int h : {4, 8, 16, 32}) {
        const Plan p = make_plan(W, H, n_bins, h);
        const size_t b = p.colcnt_bytes + p.rowcnt_bytes + p.bt_bytes + p.carry_bytes;
        most = b > most ? b : most;
    }
    return sync_bytes(W, H) + most;
}

hog_status launch_integral(const uint8_t* bins, int W, int H, int n_bins, int ii_dtype, void* ii, void* ws,
                           cudaStream_t st) {
    // vector path: a chunk's 4 bins load as one word, its 4 outputs store as
    // one 16-byte (int32) or 8-byte (uint16) vector, and every row starts aligned
    const bool vec = (reinterpret_cast<uintptr_t>(bins) % 4 == 0) && (reinterpret_cast<uintptr_t>(ii) % 16 == 0) &&
                     (W % 4 == 0);
    ClPlan c{};
    if (use_cluster(W, H, n_bins, ii_dtype, &c)) {
        const int win = cl_win(n_bins);
        if (ii_dtype == HOG_U16)
            return cl_all<uint16_t>(c, bins, W, H, n_bins, win, vec, static_cast<uint16_t*>(ii), st);
        return cl_all<int32_t>(c, bins, W, H, n_bins, win, vec, static_cast<int32_t*>(ii), st);
    }
    const int path = tune_get(HOG_TUNE_INTEGRAL_PATH);
    if (path == 2 || (path == 0 && onepass_default(W, H))) {
        unsigned int* status = nullptr;
        hog_status s = device_status_word(&status);
        if (s != HOG_OK) return s;
        const int rows = tune_get(HOG_TUNE_INTEGRAL_BAND_ROWS);
        const OpPlan o = op_plan(W, H, n_bins, rows == 32 ? 32 : 16);
        const OpWs w = op_carve(o, W, H, ws);
        if (ii_dtype == HOG_U16)
            return op_all<uint16_t>(o, bins, W, H, n_bins, static_cast<uint16_t*>(ii), w, vec, status, st);
        return op_all<int32_t>(o, bins, W, H, n_bins, static_cast<int32_t*>(ii), w, vec, status, st);
    }
    const Plan p = make_plan(W, H, n_bins);
    const Ws w = carve(p, static_cast<uint8_t*>(ws) + sync_bytes(W, H));
    if (ii_dtype == HOG_U16) return run_all<uint16_t>(p, bins, n_bins, static_cast<uint16_t*>(ii), w, vec, st);
    return run_all<int32_t>(p, bins, n_bins, static_cast<int32_t*>(ii), w, vec, st);
}

}  // namespace fasthog
