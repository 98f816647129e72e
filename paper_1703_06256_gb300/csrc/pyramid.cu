// pyramid.cu -- image pyramid by 2:1 decimation (hog_pyramid): level l is
// (W >> l) x (H >> l) and its pixel (x, y) is pixel (x << l, y << l) of the
// image.  One thread per pixel of level 1 copies it, and, where its
// coordinates are multiples of 2^(l-1), the same pixel into level l.
#include "batch_plan.cuh"
#include "internal.cuh"

namespace fasthog {

namespace {

constexpr int kMaxLevels = 16;

struct LevelTable {
    int W[kMaxLevels], H[kMaxLevels];
    long long off[kMaxLevels];  // byte offset of level l (l >= 1) in the output
};

template <int CH>
__global__ void __launch_bounds__(256)
    pyramid_kernel(const uint8_t* __restrict__ img, size_t pitch, int levels, LevelTable t, uint8_t* __restrict__ out) {
    pdl_wait();
    pdl_trigger();
    const int x = blockIdx.x * 32 + (threadIdx.x & 31);
    const int y = blockIdx.y * 8 + (threadIdx.x >> 5);
    if (x >= t.W[1] || y >= t.H[1]) return;
    const uint8_t* src = img + (size_t)(2 * y) * pitch + (size_t)(2 * x) * CH;
    uint8_t px[CH];
#pragma unroll
    for (int c = 0; c < CH; ++c) px[c] = __ldg(src + c);
    for (int l = 1; l < levels; ++l) {
        const int m = (1 << (l - 1)) - 1;
        if ((x & m) || (y & m)) break;
        const int xl = x >> (l - 1), yl = y >> (l - 1);
        if (xl >= t.W[l] || yl >= t.H[l]) break;
        uint8_t* dst = out + t.off[l] + ((size_t)yl * t.W[l] + xl) * CH;
#pragma unroll
        for (int c = 0; c < CH; ++c) dst[c] = px[c];
    }
}

void level_table(int W, int H, int channels, int levels, LevelTable* t, size_t* total) {
    long long off = 0;
    for (int l = 0; l < kMaxLevels; ++l) {
        t->W[l] = l < levels ? W >> l : 0;
        t->H[l] = l < levels ? H >> l : 0;
        t->off[l] = l >= 1 ? off : 0;
        if (l >= 1 && l < levels) off += (long long)t->W[l] * t->H[l] * channels;
    }
    if (total) *total = (size_t)off;
}

}  // namespace

size_t pyramid_bytes(int W, int H, int channels, int levels) {
    if (W < 1 || H < 1 || (channels != 1 && channels != 3) || levels < 1 || levels > kMaxLevels) return 0;
    LevelTable t;
    size_t total = 0;
    level_table(W, H, channels, levels, &t, &total);
    return total;
}

hog_status launch_pyramid(const uint8_t* img, int W, int H, int channels, size_t pitch, int levels, uint8_t* out,
                          cudaStream_t st) {
    LevelTable t;
    level_table(W, H, channels, levels, &t, nullptr);
    if (levels < 2 || t.W[1] == 0 || t.H[1] == 0) return HOG_OK;
    const dim3 grid((t.W[1] + 31) / 32, (t.H[1] + 7) / 8);
    if (channels == 1) return launch_pdl(pyramid_kernel<1>, grid, dim3(256), 0, st, img, pitch, levels, t, out);
    return launch_pdl(pyramid_kernel<3>, grid, dim3(256), 0, st, img, pitch, levels, t, out);
}

}  // namespace fasthog
