// lut.cu -- the 511 x 511 gradient lookup table (paper Section 2).
//
// One thread per (dx, dy).  The bin of a gradient is the number of sector
// boundaries theta_k = 2*pi*k/N_b (k = 1..N_b-1) at or below its angle phi in
// [0, 2*pi).  The decision is exact and uses integers only:
//
//  1. The quadrant q of (dx, dy) is found by sign tests; quadrant q holds the
//     angles [q*pi/2, (q+1)*pi/2).
//  2. Boundaries below the quadrant start all count (4k < q*N_b); boundaries
//     past the quadrant end never do.
//  3. A boundary theta_k inside the quadrant counts iff the cross product
//     cos(theta_k)*dy - sin(theta_k)*dx >= 0, because phi - theta_k then lies
//     in (-pi/2, pi/2).  cos and sin are fixed-point integers scaled by 2^40,
//     and the product is formed in 64-bit integer arithmetic.
//
// Exactness: boundaries at multiples of pi/2 have exact fixed-point values
// (0, +-2^40).  At odd multiples of pi/4, |cos| and |sin| get the same
// integer, so the cross product of a lattice point on that ray is exactly 0.
// No other boundary ray passes through a lattice point (Niven's theorem), and
// the fixed-point rounding moves the cross product by at most
// (|dx| + |dy|) * 0.5 * 2^-40 < 2.4e-10, far below the smallest true
// |cross product| of any lattice point against such a boundary (about
// 9.2e-6 over all N_b <= 64).
//
// The buffer also carries a contiguous copy of one quadrant of the table
// (dx in 1..255, dy in 0..255, rows of 256 bytes), which the bin-map kernel
// pulls into shared memory with a single bulk copy.
#include <cmath>

#include "internal.cuh"

namespace fasthog {

namespace {

// Bin of the gradient (dx, dy) != (0, 0), decided exactly as described above.
__device__ __forceinline__ int exact_bin(const LutParams& p, int dx, int dy) {
    int q;
    if (dx > 0 && dy >= 0) q = 0;
    else if (dx <= 0 && dy > 0) q = 1;
    else if (dx < 0 && dy <= 0) q = 2;
    else q = 3;
    const int nb = p.n_bins;
    int bin = 0;
    for (int k = 1; k < nb; ++k) {
        const int k4 = 4 * k;
        if (k4 < q * nb) {
            ++bin;
        } else if (k4 < (q + 1) * nb) {
            const long long cr = p.c[k] * dy - p.s[k] * dx;
            bin += cr >= 0;
        } else {
            break;
        }
    }
    return bin;
}

// Entries [0, 511*512): the table, row dy + 255, column dx + 255, pad column 511.
// Entries [511*512, +65536): the quadrant copy, row dy (0..255), column dx - 1
// (dx = 1..256; dx = 256 is outside the table and holds 0xFF).
__global__ void __launch_bounds__(256) build_lut_kernel(LutParams p, uint8_t* __restrict__ lut) {
    const int idx = blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= kLutTotal) return;
    int dx, dy;
    bool pad;
    if (idx < kLutSide * kLutPitch) {
        dy = idx / kLutPitch - kDMax;
        const int col = idx % kLutPitch;
        dx = col - kDMax;
        pad = col == kLutSide;
    } else {
        const int q = idx - kLutSide * kLutPitch;
        dy = q >> 8;
        dx = (q & 255) + 1;
        pad = dx > kDMax;
    }
    lut[idx] = (pad || (dx == 0 && dy == 0)) ? kNoBin : static_cast<uint8_t>(exact_bin(p, dx, dy));
}

}  // namespace

hog_status launch_build_lut(const LutParams& p, uint8_t* lut, cudaStream_t st) {
    build_lut_kernel<<<ceil_div(kLutTotal, 256), 256, 0, st>>>(p, lut);
    return check_launch();
}

}  // namespace fasthog
