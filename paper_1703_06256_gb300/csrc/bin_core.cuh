// bin_core.cuh -- per-pixel gradients and orientation bins of a quad of 4
// pixels (paper Section 2, Eq. 1 and the table lookup), shared by the
// bin-map kernel, the fused image-to-cells kernel and the soft-vote kernel.
// See bin_map.cu for the method.
#pragma once

#include "internal.cuh"
#include "ptx.cuh"

namespace fasthog {

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

// Fetch the whole table (511 rows of kLutPitch bytes) into L2, one slice per
// CTA of the grid, issued by thread 0 at kernel start.  After other work has
// evicted it, the first lookups would otherwise each wait for DRAM once the
// gradients are known; the prefetch overlaps that with the image loads.
// The table is 16-byte aligned and its size a multiple of 16.
__device__ __forceinline__ void prefetch_table_l2(const uint8_t* __restrict__ lut) {
    if (threadIdx.x != 0) return;
    constexpr uint32_t kUnits = (uint32_t)kLutSide * kLutPitch / 16;
    const uint32_t per = (kUnits + gridDim.x - 1) / gridDim.x;
    const uint32_t u0 = blockIdx.x * per;
    if (u0 >= kUnits) return;
    const uint32_t n = min(per, kUnits - u0);
    ptx::bulk_prefetch_l2(lut + (size_t)u0 * 16, n * 16);
}

// Byte i of a little-endian word array, i a compile-time constant (one byte
// permute: byte i & 3 of the word, zero-extended).
template <int N>
__device__ __forceinline__ int byte_of(const uint32_t (&w)[N], int i) {
    return (int)__byte_perm(w[i >> 2], 0u, 0x4440u | (uint32_t)(i & 3));
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

// Eq. 1 for pixel p (a compile-time constant after unrolling) of the quad in
// q: central differences, and for RGB the channel with the largest
// dx^2 + dy^2 (ties keep the lower channel).  Channel c of pixel x + p:
// right neighbour at byte 4 + (p+1)*CH + c of wc, left at 4 + (p-1)*CH + c,
// below / above at byte p*CH + c of wd / wu.
template <int CH>
__device__ __forceinline__ void quad_gradient(const QuadWords<CH>& q, int p, int& dx, int& dy) {
    dx = byte_of(q.wc, 4 + (p + 1) * CH) - byte_of(q.wc, 4 + (p - 1) * CH);
    dy = byte_of(q.wd, p * CH) - byte_of(q.wu, p * CH);
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
}

// The bin of one gradient (dx, dy), not (0, 0), from the quadrant table
// (QUAD) or the whole table.  Branch-free: neighbouring pixels fall in
// different quadrants, so the quadrant turn is a pair of selects.
template <bool QUAD>
__device__ __forceinline__ uint32_t bin_of(int dx, int dy, const uint8_t* __restrict__ lutq,
                                           const uint8_t* __restrict__ lut, int nb, int nb4) {
    if (QUAD) {
        // Half-turn the lower half-plane (dy < 0, or dy = 0 and dx < 0) to the
        // upper one, then quarter-turn its left part (ex <= 0) to the first
        // quadrant: (u, v) has u in 1..255 and v in 0..255, and the turns add
        // 2 and 1 quarter(s), each worth N_b/4 bins.
        const bool upper = dy > 0 || (dy == 0 && dx > 0);
        const int ex = upper ? dx : -dx, ey = upper ? dy : -dy;
        const bool right = ex > 0;
        const int u = right ? ex : ey, v = right ? ey : -ex;
        const int turns = (upper ? 0 : 2) + (right ? 0 : 1);
        const int idx = max(v * 256 + u - 1, 0);  // (0, 0) has no entry; the caller discards it
        const int t = (int)lutq[idx] + turns * nb4;
        return (uint32_t)(t >= nb ? t - nb : t);
    }
    return __ldg(lut + (size_t)(dy + kDMax) * kLutPitch + (dx + kDMax));  // (0, 0) holds no bin
}

// Eq. 1 and the table lookup for the 4 pixels of quad x (row loaded in q).
// A quad whose pixels all have both horizontal neighbours skips the
// per-pixel border test.
template <int CH, bool QUAD>
__device__ __forceinline__ uint32_t bins_of_quad(const QuadWords<CH>& q, int x, int W, const uint8_t* __restrict__ lutq,
                                                 const uint8_t* __restrict__ lut, int nb, int nb4) {
    uint32_t packed = 0;
    if (x >= 1 && x + 4 <= W - 1) {
#pragma unroll
        for (int p = 0; p < 4; ++p) {
            int dx, dy;
            quad_gradient<CH>(q, p, dx, dy);
            uint32_t bin = bin_of<QUAD>(dx, dy, lutq, lut, nb, nb4);
            if (QUAD) bin = (dx != 0 || dy != 0) ? bin : (uint32_t)kNoBin;
            packed |= bin << (8 * p);
        }
    } else {
#pragma unroll
        for (int p = 0; p < 4; ++p) {
            int dx, dy;
            quad_gradient<CH>(q, p, dx, dy);
            const int xp = x + p;
            const bool binned = xp > 0 && xp < W - 1 && (dx != 0 || dy != 0);
            const uint32_t bin = bin_of<QUAD>(dx, dy, lutq, lut, nb, nb4);
            packed |= (binned ? bin : (uint32_t)kNoBin) << (8 * p);
        }
    }
    return packed;
}

}  // namespace fasthog
