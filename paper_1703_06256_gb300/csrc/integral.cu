// integral.cu -- one integral image per bin (paper Section 3.2, Eq. 4-5).
//
//   ii_n(x, y) = #{ (x', y') : x' <= x, y' <= y, bin(x', y') = n }
//
// The one-hot images of Eq. 4 are never stored: every phase tests the bin
// map on the fly.  The planes are written exactly once, which is the bulk of
// the work (4 * N_b bytes per pixel for int32, 2 * N_b for uint16).
//
// Tiling.  The image is cut into tiles of h rows (a band) by G = 512 columns
// (a group).  A tile's values need three carries from outside it:
//   V(x, top-1)      column sums above the band, per column and bin;
//   RL(y)            per row, the count of each bin left of the group;
//   corner           ii(group_left - 1, top - 1).
// With those, ii(x, y) = ii(x, y-1) + RL(y) + (row prefix inside the group),
// starting from ii(x, top-1) = corner + (prefix of V over the group's
// columns up to x).  Because V is a whole row vector per band, a chained
// look-back scan would move tens of KiB per link; the carries come instead
// from a reduce-then-scan in which no CTA ever waits for another:
//
//   A  tile reduce   per tile: per-column counts over the band's rows
//                    (8-bit fields), per-row counts over the group's columns
//                    (16-bit), and the tile's total per bin.
//   B  carries       (a) per column, the exclusive prefix of the column counts
//                    over bands = V at every band top, two-level over bands;
//                    (b) per group and bin, the exclusive prefix of the tile
//                    totals over bands, a warp shuffle scan in chunks of 32.
//   C  tile scan     per tile: corner = sum of (b) over the groups to the
//                    left; RL(y) = sum of the row counts of those groups; one
//                    block scan of V over the group's columns; then the rows,
//                    each with a packed 16-bit row prefix (two bins per word:
//                    thread-local running sums, a warp shuffle scan and one
//                    cross-warp step, one barrier per row).
//
// Bins are handled in windows of at most 16; larger N_b runs the phases once
// per window.  Limits: W, H < 65536 (16-bit fields and carries).
#include "internal.cuh"

namespace fasthog {

namespace {

constexpr int kQ = 4;             // columns per thread
constexpr int kThreads = 128;     // threads per tile CTA
constexpr int kGroup = kQ * kThreads;  // 512 columns per group
constexpr int kWarps = kThreads / 32;
constexpr int kSegments = 32;     // phase B(a): band segments per column
constexpr int kMaxBand = 32;

struct Plan {
    int W, H, h, n_bands, n_groups, win, n_windows;
    size_t colcnt_bytes, rowcnt_bytes, bt_bytes, carry_bytes, gv_bytes;
};

inline size_t align256(size_t b) { return (b + 255) & ~size_t(255); }

// Band height h (rows per tile): the tuned value if one is set (force > 0
// overrides both), else the tallest band that still gives every SM four
// tiles (16 warps).
Plan make_plan(int W, int H, int n_bins, int force = 0) {
    Plan p{};
    p.W = W;
    p.H = H;
    p.n_groups = ceil_div(W, kGroup);
    const int tuned = force > 0 ? force : tune_get(HOG_TUNE_INTEGRAL_BAND_ROWS);
    if (tuned > 0) {
        p.h = tuned;
    } else {
        const int target = 4 * sm_count();
        p.h = 4;
        for (int h : {32, 16, 8})
            if ((long)ceil_div(H, h) * p.n_groups >= target) {
                p.h = h;
                break;
            }
    }
    p.n_bands = ceil_div(H, p.h);
    p.win = n_bins <= 4 ? 4 : (n_bins <= 8 ? 8 : 16);
    p.n_windows = ceil_div(n_bins, p.win);
    p.colcnt_bytes = align256((size_t)p.n_bands * (p.win / 4) * W * 4);
    p.rowcnt_bytes = align256((size_t)H * p.n_groups * p.win * 2);
    p.bt_bytes = align256((size_t)p.n_groups * p.win * p.n_bands * 4);
    p.carry_bytes = align256((size_t)p.n_bands * p.win * W * 2);
    p.gv_bytes = align256((size_t)p.n_bands * p.n_groups * p.win * 4);
    return p;
}

struct Ws {
    uint32_t* colcnt;  // [band][win/4][W]       packed 8-bit column counts
    uint16_t* rowcnt;  // [y][group][win]        row counts inside the group
    uint32_t* bt;      // [group][win][band]     tile totals
    uint16_t* carry;   // [band][win][W]         V(x, band top - 1)
    uint32_t* gv;      // [band][group][win]     sum over bands above of tile totals
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
    b += p.carry_bytes;
    w.gv = reinterpret_cast<uint32_t*>(b);
    return w;
}

// Load the bins of this thread's kQ columns of row y (0xFF past the right edge).
__device__ __forceinline__ void load_bins4(const uint8_t* __restrict__ bins, int W, int y, int x0, int ncol,
                                           bool vec, uint32_t v[kQ]) {
    const uint8_t* p = bins + (size_t)y * W + x0;
    if (vec && ncol == kQ) {
        const uint32_t w = __ldg(reinterpret_cast<const uint32_t*>(p));
#pragma unroll
        for (int c = 0; c < kQ; ++c) v[c] = (w >> (8 * c)) & 0xFFu;
    } else {
#pragma unroll
        for (int c = 0; c < kQ; ++c) v[c] = c < ncol ? (uint32_t)__ldg(p + c) : 0xFFu;
    }
}

// Issue the loads of this thread's kQ bins for every row of the band up
// front, so their latency is paid once per tile rather than once per row,
// and park them in shared memory (each thread reads back only its own slot).
__device__ __forceinline__ void stage_band(const uint8_t* __restrict__ bins, int W, int y0, int y1, int x0, int ncol,
                                           bool vec, uint32_t (*slot)[kThreads]) {
    for (int y = y0; y < y1; y += 8) {
        uint32_t w[8];
#pragma unroll
        for (int k = 0; k < 8; ++k) {
            w[k] = 0xFFFFFFFFu;
            if (y + k < y1) {
                uint32_t v[kQ];
                load_bins4(bins, W, y + k, x0, ncol, vec, v);
                w[k] = v[0] | (v[1] << 8) | (v[2] << 16) | (v[3] << 24);
            }
        }
#pragma unroll
        for (int k = 0; k < 8; ++k)
            if (y + k < y1) slot[y + k - y0][threadIdx.x] = w[k];
    }
}

// SIMD-within-a-register helpers built from single integer instructions
// (shifts, logic, add, multiply).  A thread's 4 bins sit in one 32-bit word,
// one byte per column.
//
// 1 << n, or 0 when n >= 32 (PTX clamps the shift amount).
__device__ __forceinline__ uint32_t bit_or_zero(uint32_t n) {
    uint32_t r;
    asm("shl.b32 %0, %1, %2;" : "=r"(r) : "r"(1u), "r"(n));
    return r;
}
// Per-column one-hot masks of the bins [lo, lo + 8): byte c of the result has
// bit k set iff column c holds bin lo + k (0xFF and bins outside the range
// set nothing).
__device__ __forceinline__ uint32_t onehot_cols8(uint32_t w, uint32_t lo) {
    uint32_t p = 0;
#pragma unroll
    for (int c = 0; c < 4; ++c) p |= (bit_or_zero(((w >> (8 * c)) & 0xFFu) - lo) & 0xFFu) << (8 * c);
    return p;
}
// Byte c = 1 iff column c holds bin lo + k.
__device__ __forceinline__ uint32_t col_flags(uint32_t p, int k) { return (p >> k) & 0x01010101u; }
// The 4 bits of a nibble to the 4 bytes (bit k -> byte k): the products
// n_k * 2^(7j) land on a multiple of 8 only for j = k, without carries.
__device__ __forceinline__ uint32_t spread4(uint32_t nib) { return (nib * 0x00204081u) & 0x01010101u; }
// Counts of 4 bins in 8-bit fields (word m: bins 4m..4m+3) widen to 16-bit
// fields two bins per word, paired as E[2m] = (4m, 4m+2), E[2m+1] = (4m+1, 4m+3).
__device__ __forceinline__ uint32_t even16(uint32_t t) { return t & 0x00FF00FFu; }
__device__ __forceinline__ uint32_t odd16(uint32_t t) { return (t >> 8) & 0x00FF00FFu; }
__host__ __device__ constexpr int e_word(int b) { return 2 * (b >> 2) + (b & 1); }
__host__ __device__ constexpr int e_half(int b) { return (b >> 1) & 1; }

// ---------------------------------------------------------------- phase A
template <int WIN>
__global__ void __launch_bounds__(kThreads)
    ii_tile_reduce_kernel(const uint8_t* __restrict__ bins, int W, int H, int h, int n_bands, int n_groups,
                          int bin_base, bool vec, Ws ws) {
    constexpr int NM = WIN / 4;  // 8-bit-field words (4 bins each)
    constexpr int NE = WIN / 2;  // 16-bit-field words (2 bins each)
    __shared__ uint32_t row_acc[kMaxBand][NE];
    __shared__ uint32_t band_bins[kMaxBand][kThreads];
    const int band = blockIdx.x, g = blockIdx.y;
    const int tid = threadIdx.x, lane = tid & 31;
    const int x0 = g * kGroup + tid * kQ;
    const int ncol = max(0, min(kQ, W - x0));
    const int y0 = band * h, y1 = min(H, y0 + h);

    pdl_trigger();
    pdl_wait();
    stage_band(bins, W, y0, y1, x0, ncol, vec, band_bins);
    for (int i = tid; i < kMaxBand * NE; i += kThreads) (&row_acc[0][0])[i] = 0;
    __syncthreads();

    // col[c][m]: counts over the band's rows of bins 4m..4m+3 in column c (8-bit fields)
    uint32_t col[kQ][NM];
#pragma unroll
    for (int c = 0; c < kQ; ++c)
#pragma unroll
        for (int m = 0; m < NM; ++m) col[c][m] = 0;

    for (int y = y0; y < y1; ++y) {
        const uint32_t w = band_bins[y - y0][tid];
        uint32_t rowt[NM];
#pragma unroll
        for (int g8 = 0; g8 < (WIN + 7) / 8; ++g8) {
            const uint32_t p = onehot_cols8(w, (uint32_t)(bin_base + 8 * g8));
#pragma unroll
            for (int hh = 0; hh < 2; ++hh) {
                const int m = 2 * g8 + hh;  // bins 4m..4m+3 = nibble hh of each byte of p
                if (m < NM) {
                    uint32_t tsum = 0;
#pragma unroll
                    for (int c = 0; c < kQ; ++c) {
                        const uint32_t t = spread4((p >> (8 * c + 4 * hh)) & 0xFu);
                        col[c][m] += t;
                        tsum += t;
                    }
                    rowt[m] = tsum;
                }
            }
        }
#pragma unroll
        for (int m = 0; m < NM; ++m) {
            uint32_t s = rowt[m];  // 8-bit fields: a warp's row count is at most 128
#pragma unroll
            for (int d = 16; d > 0; d >>= 1) s += __shfl_xor_sync(0xffffffffu, s, d);
            if (lane == 0 && s) {
                atomicAdd(&row_acc[y - y0][2 * m], even16(s));
                atomicAdd(&row_acc[y - y0][2 * m + 1], odd16(s));
            }
        }
    }
    // per-column counts of the band
    if (ncol > 0) {
#pragma unroll
        for (int c = 0; c < kQ; ++c)
            if (c < ncol)
#pragma unroll
                for (int m = 0; m < NM; ++m) ws.colcnt[((size_t)band * NM + m) * W + x0 + c] = col[c][m];
    }
    __syncthreads();
    // per-row counts of the group, and the tile total
    for (int i = tid; i < (y1 - y0) * WIN; i += kThreads) {
        const int r = i / WIN, b = i - r * WIN;
        const uint32_t v = (row_acc[r][e_word(b)] >> (16 * e_half(b))) & 0xFFFFu;
        ws.rowcnt[((size_t)(y0 + r) * n_groups + g) * WIN + b] = (uint16_t)v;
    }
    if (tid < WIN) {
        uint32_t t = 0;
        for (int r = 0; r < y1 - y0; ++r) t += (row_acc[r][e_word(tid)] >> (16 * e_half(tid))) & 0xFFFFu;
        ws.bt[((size_t)g * WIN + tid) * n_bands + band] = t;
    }
}

// ---------------------------------------------------------------- phase B
// Blocks [0, nb_a): (a) column carries; block b covers 32 columns x one
//   8-bit word (4 bins); threads (lane, seg).
// Blocks [nb_a, nb_a + ceil(n_groups*WIN/kSegments)): (b) one warp per
//   (group, bin), scanning the tile totals over bands in chunks of 32.
template <int WIN>
__global__ void __launch_bounds__(32 * kSegments)
    ii_carry_kernel(int W, int n_bands, int n_groups, int nb_a, Ws ws) {
    constexpr int NWD = WIN / 4;
    const int lane = threadIdx.x, seg = threadIdx.y;
    pdl_trigger();
    pdl_wait();
    if ((int)blockIdx.x >= nb_a) {
        const int pair = (blockIdx.x - nb_a) * kSegments + seg;
        if (pair >= n_groups * WIN) return;
        const int g = pair / WIN, b = pair - g * WIN;
        const uint32_t* src = ws.bt + ((size_t)g * WIN + b) * n_bands;
        uint32_t run = 0;
        for (int k0 = 0; k0 < n_bands; k0 += 32) {
            const int k = k0 + lane;
            const uint32_t v = k < n_bands ? __ldg(src + k) : 0u;
            uint32_t s = v;
#pragma unroll
            for (int d = 1; d < 32; d <<= 1) {
                const uint32_t t = __shfl_up_sync(0xffffffffu, s, d);
                if (lane >= d) s += t;
            }
            if (k < n_bands) ws.gv[((size_t)k * n_groups + g) * WIN + b] = run + s - v;
            run += __shfl_sync(0xffffffffu, s, 31);
        }
        return;
    }
    __shared__ uint32_t seg_sum[kSegments][32][4];
    const int words_x = (W + 31) / 32;
    const int kw = blockIdx.x / words_x;
    const int x = (blockIdx.x - kw * words_x) * 32 + lane;
    const int per = (n_bands + kSegments - 1) / kSegments;
    const int b0 = seg * per, b1 = min(n_bands, b0 + per);
    constexpr int kPF = 8;  // loads in flight per thread
    uint32_t s[4] = {0, 0, 0, 0};
    for (int b = b0; b < b1; b += kPF) {
        uint32_t wv[kPF];
#pragma unroll
        for (int k = 0; k < kPF; ++k)
            wv[k] = (x < W && b + k < b1) ? __ldg(ws.colcnt + ((size_t)(b + k) * NWD + kw) * W + x) : 0u;
#pragma unroll
        for (int k = 0; k < kPF; ++k)
#pragma unroll
            for (int e = 0; e < 4; ++e) s[e] += (wv[k] >> (8 * e)) & 0xFFu;
    }
#pragma unroll
    for (int e = 0; e < 4; ++e) seg_sum[seg][lane][e] = s[e];
    __syncthreads();
    uint32_t run[4] = {0, 0, 0, 0};
    for (int t = 0; t < seg; ++t)
#pragma unroll
        for (int e = 0; e < 4; ++e) run[e] += seg_sum[t][lane][e];
    if (x >= W) return;
    for (int b = b0; b < b1; b += kPF) {
        uint32_t wv[kPF];
#pragma unroll
        for (int k = 0; k < kPF; ++k)
            wv[k] = b + k < b1 ? __ldg(ws.colcnt + ((size_t)(b + k) * NWD + kw) * W + x) : 0u;
#pragma unroll
        for (int k = 0; k < kPF; ++k) {
            if (b + k < b1) {
#pragma unroll
                for (int e = 0; e < 4; ++e) {
                    ws.carry[((size_t)(b + k) * WIN + 4 * kw + e) * W + x] = (uint16_t)run[e];
                    run[e] += (wv[k] >> (8 * e)) & 0xFFu;
                }
            }
        }
    }
}

// ---------------------------------------------------------------- phase C
template <typename OutT>
__device__ __forceinline__ void store4(OutT* p, const int* v, int n, bool vec);
template <>
__device__ __forceinline__ void store4<int32_t>(int32_t* p, const int* v, int n, bool vec) {
    if (vec && n == 4) {
        *reinterpret_cast<int4*>(p) = make_int4(v[0], v[1], v[2], v[3]);
    } else {
        for (int c = 0; c < n; ++c) p[c] = v[c];
    }
}
template <>
__device__ __forceinline__ void store4<uint16_t>(uint16_t* p, const int* v, int n, bool vec) {
    if (vec && n == 4) {
        const uint32_t a = (uint32_t)(v[0] & 0xFFFF) | ((uint32_t)v[1] << 16);
        const uint32_t b = (uint32_t)(v[2] & 0xFFFF) | ((uint32_t)v[3] << 16);
        *reinterpret_cast<uint2*>(p) = make_uint2(a, b);
    } else {
        for (int c = 0; c < n; ++c) p[c] = (uint16_t)v[c];
    }
}

template <int WIN, typename OutT>
__global__ void __launch_bounds__(kThreads)
    ii_tile_scan_kernel(const uint8_t* __restrict__ bins, int W, int H, int h, int n_groups, int bin_base,
                        int n_bins, bool vec, Ws ws, OutT* __restrict__ ii) {
    constexpr int NM = WIN / 4;  // 8-bit-field words (4 bins each)
    constexpr int NE = WIN / 2;  // 16-bit-field words (2 bins each, e_word/e_half pairing)
    __shared__ int corner_s[WIN];
    __shared__ uint32_t rl_s[kMaxBand][NE];
    __shared__ int wtot_init[kWarps][WIN];
    __shared__ uint32_t wtot[2][kWarps][NM];

    const int band = blockIdx.x, g = blockIdx.y;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int x0 = g * kGroup + tid * kQ;
    const int ncol = max(0, min(kQ, W - x0));
    const int y0 = band * h, y1 = min(H, y0 + h);
    const int wins = min(WIN, n_bins - bin_base);
    __shared__ uint32_t band_bins[kMaxBand][kThreads];
    pdl_trigger();
    pdl_wait();
    stage_band(bins, W, y0, y1, x0, ncol, vec, band_bins);

    // corner = ii(group_left - 1, y0 - 1); RL(y) for the band's rows
    if (tid < WIN) {
        uint32_t s = 0;
        for (int gg = 0; gg < g; ++gg) s += __ldg(ws.gv + ((size_t)band * n_groups + gg) * WIN + tid);
        corner_s[tid] = (int)s;
    }
    for (int i = tid; i < (y1 - y0) * NE; i += kThreads) {
        const int r = i / NE, k = i - r * NE;
        const int blo = 4 * (k >> 1) + (k & 1), bhi = blo + 2;  // the bins of E[k]
        uint32_t lo = 0, hi = 0;
        const uint16_t* rc = ws.rowcnt + (size_t)(y0 + r) * n_groups * WIN;
        for (int gg = 0; gg < g; ++gg) {
            lo += __ldg(rc + gg * WIN + blo);
            hi += __ldg(rc + gg * WIN + bhi);
        }
        rl_s[r][k] = lo | (hi << 16);
    }

    // ii(x, y0 - 1) = corner + prefix over the group's columns of V(x, y0 - 1)
    int acc[kQ][WIN];
    int tot[WIN];
#pragma unroll
    for (int b = 0; b < WIN; ++b) {
        const uint16_t* cp = ws.carry + ((size_t)band * WIN + b) * W + x0;
        int cv[kQ];
        if (vec && ncol == kQ) {
            const uint2 u = __ldg(reinterpret_cast<const uint2*>(cp));
            cv[0] = (int)(u.x & 0xFFFFu);
            cv[1] = (int)(u.x >> 16);
            cv[2] = (int)(u.y & 0xFFFFu);
            cv[3] = (int)(u.y >> 16);
        } else {
#pragma unroll
            for (int c = 0; c < kQ; ++c) cv[c] = c < ncol ? (int)__ldg(cp + c) : 0;
        }
        int run = 0;
#pragma unroll
        for (int c = 0; c < kQ; ++c) {
            run += cv[c];
            acc[c][b] = run;
        }
        tot[b] = run;
    }
#pragma unroll
    for (int b = 0; b < WIN; ++b) {
        int v = tot[b];
#pragma unroll
        for (int d = 1; d < 32; d <<= 1) {
            const int t = __shfl_up_sync(0xffffffffu, v, d);
            if (lane >= d) v += t;
        }
        if (lane == 31) wtot_init[warp][b] = v;
        tot[b] = v - tot[b];
    }
    __syncthreads();
#pragma unroll
    for (int b = 0; b < WIN; ++b) {
        int off = corner_s[b] + tot[b];
        for (int w = 0; w < warp; ++w) off += wtot_init[w][b];
#pragma unroll
        for (int c = 0; c < kQ; ++c) acc[c][b] += off;
    }

    // rows of the band: ii(x, y) = ii(x, y-1) + R(x, y), R = row prefix of
    // the one-hot row = RL(y) + (count left of this thread in the group)
    //                        + (count in this thread's columns up to x)
    const size_t plane = (size_t)H * W;
    OutT* out_row = ii + (size_t)bin_base * plane + (size_t)y0 * W + x0;
    int buf = 0;
    for (int y = y0; y < y1; ++y, out_row += W) {
        const uint32_t w = band_bins[y - y0][tid];
        // pre4[b] byte c = count of bin b in this thread's columns 0..c
        uint32_t pre4[WIN];
#pragma unroll
        for (int g8 = 0; g8 < (WIN + 7) / 8; ++g8) {
            const uint32_t p = onehot_cols8(w, (uint32_t)(bin_base + 8 * g8));
#pragma unroll
            for (int k = 0; k < 8; ++k)
                if (8 * g8 + k < WIN) pre4[8 * g8 + k] = col_flags(p, k) * 0x01010101u;
        }
        // thread totals (8-bit fields) and their inclusive warp scan
        uint32_t T[NM], S[NM];
#pragma unroll
        for (int m = 0; m < NM; ++m) {
            T[m] = __byte_perm(__byte_perm(pre4[4 * m], pre4[4 * m + 1], 0x0073),
                               __byte_perm(pre4[4 * m + 2], pre4[4 * m + 3], 0x0073), 0x5410);
            S[m] = T[m];
        }
#pragma unroll
        for (int d = 1; d < 32; d <<= 1) {
#pragma unroll
            for (int m = 0; m < NM; ++m) {
                const uint32_t t = __shfl_up_sync(0xffffffffu, S[m], d);
                if (lane >= d) S[m] += t;  // a warp's row count per bin is at most 128
            }
        }
        if (lane == 31) {
#pragma unroll
            for (int m = 0; m < NM; ++m) wtot[buf][warp][m] = S[m];
        }
        __syncthreads();
        // exclusive offset of this thread's first column, 16-bit fields
        uint32_t E[NE];
#pragma unroll
        for (int m = 0; m < NM; ++m) {
            const uint32_t x = S[m] - T[m];
            E[2 * m] = rl_s[y - y0][2 * m] + even16(x);
            E[2 * m + 1] = rl_s[y - y0][2 * m + 1] + odd16(x);
        }
        for (int w2 = 0; w2 < warp; ++w2) {
#pragma unroll
            for (int m = 0; m < NM; ++m) {
                const uint32_t t = wtot[buf][w2][m];
                E[2 * m] += even16(t);
                E[2 * m + 1] += odd16(t);
            }
        }
        buf ^= 1;
#pragma unroll
        for (int b = 0; b < WIN; ++b) {
            const uint32_t base = (E[e_word(b)] >> (16 * e_half(b))) & 0xFFFFu;
#pragma unroll
            for (int c = 0; c < kQ; ++c) acc[c][b] += (int)(base + ((pre4[b] >> (8 * c)) & 0xFFu));
        }
        if (ncol > 0) {
#pragma unroll
            for (int b = 0; b < WIN; ++b) {
                if (b < wins) {
                    int vals[kQ];
#pragma unroll
                    for (int c = 0; c < kQ; ++c) vals[c] = acc[c][b];
                    store4<OutT>(out_row + (size_t)b * plane, vals, ncol, vec);
                }
            }
        }
    }
}

template <int WIN, typename OutT>
hog_status run_window(const Plan& p, const uint8_t* bins, int n_bins, int bin_base, OutT* ii, const Ws& ws,
                      bool vec, cudaStream_t st) {
    dim3 grid_tiles(p.n_bands, p.n_groups);
    hog_status s = launch_pdl(ii_tile_reduce_kernel<WIN>, grid_tiles, dim3(kThreads), 0, st, bins, p.W, p.H, p.h,
                              p.n_bands, p.n_groups, bin_base, vec, ws);
    if (s != HOG_OK) return s;
    const int nb_a = ceil_div(p.W, 32) * (WIN / 4);
    const int nb_b = ceil_div(p.n_groups * WIN, kSegments);
    s = launch_pdl(ii_carry_kernel<WIN>, dim3(nb_a + nb_b), dim3(32, kSegments), 0, st, p.W, p.n_bands, p.n_groups,
                   nb_a, ws);
    if (s != HOG_OK) return s;
    return launch_pdl(ii_tile_scan_kernel<WIN, OutT>, grid_tiles, dim3(kThreads), 0, st, bins, p.W, p.H, p.h,
                      p.n_groups, bin_base, n_bins, vec, ws, ii);
}

template <typename OutT>
hog_status run_all(const Plan& p, const uint8_t* bins, int n_bins, OutT* ii, const Ws& ws, bool vec,
                   cudaStream_t st) {
    for (int wi = 0; wi < p.n_windows; ++wi) {
        const int base = wi * p.win;
        hog_status s = p.win == 4   ? run_window<4, OutT>(p, bins, n_bins, base, ii, ws, vec, st)
                       : p.win == 8 ? run_window<8, OutT>(p, bins, n_bins, base, ii, ws, vec, st)
                                    : run_window<16, OutT>(p, bins, n_bins, base, ii, ws, vec, st);
        if (s != HOG_OK) return s;
    }
    return HOG_OK;
}

}  // namespace

size_t integral_workspace_bytes(int W, int H, int n_bins) {
    // enough for every band height, so a workspace stays valid whatever the tuning
    size_t most = 0;
    for (int h : {4, 8, 16, 32}) {
        const Plan p = make_plan(W, H, n_bins, h);
        const size_t b = p.colcnt_bytes + p.rowcnt_bytes + p.bt_bytes + p.carry_bytes + p.gv_bytes;
        most = b > most ? b : most;
    }
    return most;
}

hog_status launch_integral(const uint8_t* bins, int W, int H, int n_bins, int ii_dtype, void* ii, void* ws,
                           cudaStream_t st) {
    const Plan p = make_plan(W, H, n_bins);
    const Ws w = carve(p, ws);
    const size_t elem = ii_dtype == HOG_U16 ? 2 : 4;
    // vector path: 4-byte bin loads and 4-element stores stay aligned
    const bool vec = (reinterpret_cast<uintptr_t>(bins) % 4 == 0) &&
                     (reinterpret_cast<uintptr_t>(ii) % (4 * elem) == 0) && (W % 4 == 0);
    if (ii_dtype == HOG_U16) return run_all<uint16_t>(p, bins, n_bins, static_cast<uint16_t*>(ii), w, vec, st);
    return run_all<int32_t>(p, bins, n_bins, static_cast<int32_t*>(ii), w, vec, st);
}

}  // namespace fasthog
