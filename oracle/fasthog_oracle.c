/*
 * fasthog_oracle.c -- plain, slow CPU oracle for the fast-HOG detection path.
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product path may call, link or
 * load this file: only the test-suite, the smoke check and the CPU-baseline
 * leg of the benchmark use it.  It shares no code, header, table or constant
 * generator with the CUDA library; it is written from the paper
 * ("A Fast HOG Descriptor Using Lookup Table and Integral Image") directly.
 *
 * Everything here is the plain definition of what the paper computes, in
 * the paper's order, without blocking, fusion or reordering:
 *
 *   Section 2, Eq. 1   central differences dx, dy per pixel and channel
 *   Section 2, Fig. 2  unit magnitude, angle in [0, 2*pi) split into N_b bins
 *   Section 2          the 511 x 511 lookup table over all (dx, dy)
 *   Section 3.1, Eq. 2 integral image (inclusive prefix sum in x and y)
 *   Section 3.1, Eq. 3 four-corner box sum
 *   Section 3.2, Eq. 4 one-hot decomposition of the bin map, one image per bin
 *   Section 3.2, Eq. 5 one integral image per bin
 *   Section 3.3, Eq. 6 per-bin area histogram from four corners
 *   Section 1 / 4      linear objectness score per window, threshold, list
 *
 * Readings where the paper is silent or garbled (each one is also listed in
 * the design notes of the repository):
 *   - dx, dy range over [-255, 255] (the paper's "-225" is a typo: 511 = 2*255+1).
 *   - phi = angle of the vector (dx, dy) measured from +x towards +y with the
 *     image y axis pointing down, in [0, 2*pi) (signed orientation).
 *   - bins are half-open sectors [k*2*pi/N_b, (k+1)*2*pi/N_b).
 *   - (dx, dy) = (0, 0) and border pixels (where Eq. 1 would read outside the
 *     image) get no bin (value 0xFF) and enter no integral image.
 *   - colour: per pixel the channel with the largest dx^2 + dy^2 wins, ties go
 *     to the lowest channel index.
 *   - box corners of Eq. 3 / Eq. 6: 1 = (x0-1, y0-1), 2 = (x1, y0-1),
 *     3 = (x0-1, y1), 4 = (x1, y1); an index of -1 reads as 0.
 *   - window feature index (cy * cells_x + cx) * N_b + b; score = bias + w . h.
 *   - detections: score >= threshold, listed in row-major window order.
 *
 * Floating point is FP64 throughout.
 */

#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define ORACLE_NO_BIN 0xFF
#define ORACLE_DMAX 255
#define ORACLE_LUT_SIDE 511

/* Smallest |cross product| met so far against an irrational sector boundary;
 * the FP64 evaluation is trusted only while this stays far above its own
 * rounding error.  Read with oracle_min_margin(). */
static double g_min_margin = 1e300;
static int g_margin_violation = 0;

double oracle_min_margin(void) { return g_min_margin; }
int oracle_margin_violation(void) { return g_margin_violation; }
void oracle_reset_margin(void) {
    g_min_margin = 1e300;
    g_margin_violation = 0;
}

/* phi in [0, pi) ?  (Fig. 2 reading: the upper half plane includes the +x ray
 * and excludes the -x ray.) */
static int in_upper_half(int dx, int dy) { return dy > 0 || (dy == 0 && dx > 0); }

/* Sign of cross(u_k, v) = cos(theta_k) * dy - sin(theta_k) * dx, where u_k is the
 * unit vector of boundary theta_k = 2*pi*k/nb.  Returns +1, 0 or -1.
 *
 * Boundaries at multiples of pi/4 have integer direction vectors, so the
 * sign is exact.  Any other boundary has an irrational slope (Niven's
 * theorem: tan of a rational multiple of pi is rational only for 0 and +-1),
 * so no lattice point lies on it; there the cross product is evaluated in
 * FP64 and the margin is recorded. */
static int cross_sign(int k, int nb, int dx, int dy) {
    if ((8 * k) % nb == 0) {
        static const int dir[8][2] = {{1, 0}, {1, 1}, {0, 1}, {-1, 1},
                                      {-1, 0}, {-1, -1}, {0, -1}, {1, -1}};
        int m = (8 * k) / nb; /* theta_k = m * pi / 4 */
        long c = dir[m][0], s = dir[m][1];
        long cr = c * dy - s * dx;
        return (cr > 0) - (cr < 0);
    }
    double theta = 2.0 * M_PI * (double)k / (double)nb;
    double cr = cos(theta) * (double)dy - sin(theta) * (double)dx;
    double a = fabs(cr);
    if (a < g_min_margin) g_min_margin = a;
    if (a < 1e-9) g_margin_violation = 1;
    return (cr > 0) - (cr < 0);
}

/* Is theta_k <= phi(dx, dy)?  Both angles in [0, 2*pi). */
static int boundary_at_or_below(int k, int nb, int dx, int dy) {
    int upper = in_upper_half(dx, dy);
    if (2 * k == nb) return !upper;          /* theta_k = pi */
    if (2 * k < nb) {                        /* theta_k in (0, pi) */
        if (!upper) return 1;                /* phi >= pi > theta_k */
        return cross_sign(k, nb, dx, dy) >= 0;
    }
    /* theta_k in (pi, 2*pi) */
    if (upper) return 0;                     /* phi < pi < theta_k */
    return cross_sign(k, nb, dx, dy) >= 0;
}

/* Section 2: orientation bin of one gradient, unit magnitude.  The bin is the
 * number of sector boundaries theta_1..theta_{nb-1} at or below phi. */
int oracle_sector_bin(int dx, int dy, int nb) {
    if (dx == 0 && dy == 0) return ORACLE_NO_BIN;
    int bin = 0;
    for (int k = 1; k < nb; ++k) bin += boundary_at_or_below(k, nb, dx, dy);
    return bin;
}

/* Section 2: the 511 x 511 table over every (dx, dy) in [-255, 255]^2,
 * entry index (dy + 255) * 511 + (dx + 255). */
int oracle_lut(int nb, uint8_t* lut) {
    if (nb < 1 || nb > 64) return -1;
    for (int dy = -ORACLE_DMAX; dy <= ORACLE_DMAX; ++dy)
        for (int dx = -ORACLE_DMAX; dx <= ORACLE_DMAX; ++dx)
            lut[(dy + ORACLE_DMAX) * ORACLE_LUT_SIDE + (dx + ORACLE_DMAX)] =
                (uint8_t)oracle_sector_bin(dx, dy, nb);
    return 0;
}

/* Section 2, Eq. 1: oriented-gradient map.  img holds H rows of `pitch` bytes;
 * a gray pixel is img[y*pitch + x], an RGB pixel img[y*pitch + 3*x + c]. */
int oracle_bin_map(const uint8_t* img, int W, int H, int channels, long pitch, int nb,
                   uint8_t* bins) {
    if (channels != 1 && channels != 3) return -1;
    if (nb < 1 || nb > 64) return -1;
    for (int y = 0; y < H; ++y) {
        for (int x = 0; x < W; ++x) {
            uint8_t out = ORACLE_NO_BIN;
            if (x > 0 && x < W - 1 && y > 0 && y < H - 1) {
                int best_dx = 0, best_dy = 0;
                long best_mag = -1;
                for (int c = 0; c < channels; ++c) {
                    int right = img[y * pitch + (long)channels * (x + 1) + c];
                    int left = img[y * pitch + (long)channels * (x - 1) + c];
                    int down = img[(y + 1) * pitch + (long)channels * x + c];
                    int up = img[(y - 1) * pitch + (long)channels * x + c];
                    int dx = right - left;
                    int dy = down - up;
                    long mag = (long)dx * dx + (long)dy * dy;
                    if (mag > best_mag) { /* strict: ties keep the lower channel */
                        best_mag = mag;
                        best_dx = dx;
                        best_dy = dy;
                    }
                }
                out = (uint8_t)oracle_sector_bin(best_dx, best_dy, nb);
            }
            bins[(long)y * W + x] = out;
        }
    }
    return 0;
}

/* Section 3.2, Eq. 4 and Eq. 5 written out literally: for every bin n and
 * point (x, y), count the points (x', y') with x' <= x, y' <= y whose bin is n.
 * O(W^2 H^2 N_b): tiny images only.  Output ii[n][y][x]. */
int oracle_integral_brute(const uint8_t* bins, int W, int H, int nb, int32_t* ii) {
    for (int n = 0; n < nb; ++n)
        for (int y = 0; y < H; ++y)
            for (int x = 0; x < W; ++x) {
                int32_t s = 0;
                for (int yy = 0; yy <= y; ++yy)
                    for (int xx = 0; xx <= x; ++xx)
                        s += bins[(long)yy * W + xx] == n;
                ii[((long)n * H + y) * W + x] = s;
            }
    return 0;
}

/* Section 3.2, Eq. 5 by running sums: a running sum along each row of the
 * one-hot image i_n, added to the integral row above. */
int oracle_integral(const uint8_t* bins, int W, int H, int nb, int32_t* ii) {
    if ((long)W * H > 2147483647L) return -1;
    for (int n = 0; n < nb; ++n) {
        int32_t* plane = ii + (long)n * H * W;
        for (int y = 0; y < H; ++y) {
            int32_t row = 0;
            for (int x = 0; x < W; ++x) {
                row += bins[(long)y * W + x] == n;
                plane[(long)y * W + x] = row + (y > 0 ? plane[(long)(y - 1) * W + x] : 0);
            }
        }
    }
    return 0;
}

/* Number of cell origins along one axis: origins at 0, s, 2s, ... with the
 * whole cell inside the image. */
static int n_positions(int extent, int box, int stride) {
    return extent < box ? 0 : (extent - box) / stride + 1;
}

/* Section 3 / 3.3: histogram of every cell (an area R of the oriented-gradient
 * map) by counting its pixels directly.  Cells of cell x cell pixels at
 * origins (s*i, s*j).  Output cells[j][i][b] (int32). */
int oracle_cell_hist_direct(const uint8_t* bins, int W, int H, int nb, int cell, int stride,
                            int32_t* cells) {
    int ncx = n_positions(W, cell, stride), ncy = n_positions(H, cell, stride);
    for (int j = 0; j < ncy; ++j)
        for (int i = 0; i < ncx; ++i) {
            int32_t* h = cells + ((long)j * ncx + i) * nb;
            for (int b = 0; b < nb; ++b) h[b] = 0;
            for (int y = j * stride; y < j * stride + cell; ++y)
                for (int x = i * stride; x < i * stride + cell; ++x) {
                    int v = bins[(long)y * W + x];
                    if (v < nb) h[v] += 1;
                }
        }
    return 0;
}

/* Read ii_n(x, y) with the convention that an index of -1 reads 0. */
static long ii_at(const int32_t* ii, int W, int H, int n, int x, int y) {
    if (x < 0 || y < 0) return 0;
    return ii[((long)n * H + y) * W + x];
}

/* Section 3.3, Eq. 6 (Eq. 3 per bin): V_R^B = ii_B(4) + ii_B(1) - ii_B(2) - ii_B(3). */
int oracle_cell_hist_ii(const int32_t* ii, int W, int H, int nb, int cell, int stride,
                        int32_t* cells) {
    int ncx = n_positions(W, cell, stride), ncy = n_positions(H, cell, stride);
    for (int j = 0; j < ncy; ++j)
        for (int i = 0; i < ncx; ++i) {
            int x0 = i * stride, y0 = j * stride;
            int x1 = x0 + cell - 1, y1 = y0 + cell - 1;
            for (int b = 0; b < nb; ++b) {
                long v4 = ii_at(ii, W, H, b, x1, y1);
                long v1 = ii_at(ii, W, H, b, x0 - 1, y0 - 1);
                long v2 = ii_at(ii, W, H, b, x1, y0 - 1);
                long v3 = ii_at(ii, W, H, b, x0 - 1, y1);
                cells[((long)j * ncx + i) * nb + b] = (int32_t)(v4 + v1 - v2 - v3);
            }
        }
    return 0;
}

/* Sections 1 and 4: objectness score of every window position.  A window of
 * cells_x x cells_y cells (each `cell` pixels) at (px*s, py*s) concatenates
 * the histograms of its cells; with r = cell / s, its cell (i, j) is the
 * cell-map entry (px + i*r, py + j*r).  score = bias + sum_k w_k h_k in FP64.
 * Output S[py][px] with nx = ncx - (cells_x-1)*r, ny = ncy - (cells_y-1)*r. */
int oracle_window_score(const int32_t* cells, int ncx, int ncy, int nb, int cells_x,
                        int cells_y, int cell, int stride, const double* w, double bias,
                        double* S) {
    if (stride <= 0 || cell % stride != 0) return -1;
    int r = cell / stride;
    int nx = ncx - (cells_x - 1) * r, ny = ncy - (cells_y - 1) * r;
    if (nx <= 0 || ny <= 0) return 0;
    for (int py = 0; py < ny; ++py)
        for (int px = 0; px < nx; ++px) {
            double acc = bias;
            for (int j = 0; j < cells_y; ++j)
                for (int i = 0; i < cells_x; ++i)
                    for (int b = 0; b < nb; ++b)
                        acc += w[((long)j * cells_x + i) * nb + b] *
                               (double)cells[((long)(py + j * r) * ncx + (px + i * r)) * nb + b];
            S[(long)py * nx + px] = acc;
        }
    return 0;
}

/* The same score straight from the bin map: every window's feature vector is
 * built by visiting each of its pixels (no cell map, no integral image). */
int oracle_window_score_from_bins(const uint8_t* bins, int W, int H, int nb, int cells_x,
                                  int cells_y, int cell, int stride, const double* w,
                                  double bias, double* S) {
    if (stride <= 0) return -1;
    int nx = n_positions(W, cells_x * cell, stride), ny = n_positions(H, cells_y * cell, stride);
    int K = cells_x * cells_y * nb;
    long* feat = (long*)malloc(sizeof(long) * (size_t)K);
    if (!feat) return -2;
    for (int py = 0; py < ny; ++py)
        for (int px = 0; px < nx; ++px) {
            memset(feat, 0, sizeof(long) * (size_t)K);
            for (int j = 0; j < cells_y; ++j)
                for (int i = 0; i < cells_x; ++i)
                    for (int y = py * stride + j * cell; y < py * stride + (j + 1) * cell; ++y)
                        for (int x = px * stride + i * cell; x < px * stride + (i + 1) * cell; ++x) {
                            int v = bins[(long)y * W + x];
                            if (v < nb) feat[((long)j * cells_x + i) * nb + v] += 1;
                        }
            double acc = bias;
            for (int k = 0; k < K; ++k) acc += w[k] * (double)feat[k];
            S[(long)py * nx + px] = acc;
        }
    free(feat);
    return 0;
}

/* Threshold and list: every window with score >= thr, in row-major order,
 * as (x, y, score) with x = px*s, y = py*s.  Returns the number of
 * detections; entries beyond max_out are counted but not written. */
long oracle_detect(const double* S, int nx, int ny, int stride, double thr, int32_t* xs,
                   int32_t* ys, double* scores, long max_out) {
    long n = 0;
    for (int py = 0; py < ny; ++py)
        for (int px = 0; px < nx; ++px) {
            double v = S[(long)py * nx + px];
            if (v >= thr) {
                if (n < max_out) {
                    xs[n] = px * stride;
                    ys[n] = py * stride;
                    scores[n] = v;
                }
                ++n;
            }
        }
    return n;
}

/* Soft votes: the two-bin vote of Section 2 (OpenCV's way, which the paper
 * sets aside for single-bin unit votes).  The gradient angle phi in [0, 2 pi)
 * is placed among the bin centres c_k = (k + 1/2) 2 pi / nb:
 *   t = phi nb / (2 pi) - 1/2,  k0 = floor(t) mod nb,  alpha = t - floor(t),
 * and the pixel (unit magnitude) votes q - a to bin k0 and a to bin k0 + 1
 * (mod nb), a = round(q alpha) to nearest.  a = q is written as (k0 + 1, 0),
 * so that an angle on a bin centre has one encoding.  The distance of
 * q alpha from the nearest half-integer is recorded (oracle_soft_lut returns
 * its minimum): a rounding tie would make the vote depend on the last bit
 * of atan2, and the tables' lattice points keep far from one.
 * Operation order is fixed (FP contraction off): ((phi * nb) / 2pi) - 1/2. */
static const double ORACLE_TWO_PI = 6.283185307179586; /* 2 pi rounded to double */

static int soft_vote(int dx, int dy, int nb, int q, int* k0_out, double* margin) {
    double phi = atan2((double)dy, (double)dx);
    if (phi < 0.0) phi += ORACLE_TWO_PI;
    double t = phi * (double)nb / ORACLE_TWO_PI - 0.5;
    double fl = floor(t);
    double x = (double)q * (t - fl);
    double m = fabs(x - floor(x) - 0.5);
    if (margin && m < *margin) *margin = m;
    int a = (int)floor(x + 0.5);
    int k0 = (int)fl % nb;
    if (k0 < 0) k0 += nb;
    if (a >= q) {
        a = 0;
        k0 = (k0 + 1) % nb;
    }
    *k0_out = k0;
    return a;
}

/* The soft table: entry (dy + 255) * 511 + (dx + 255) = k0 | a << 8, or
 * 0xFFFF for (0, 0).  *margin receives the smallest distance of q alpha from
 * a half-integer over the table. */
int oracle_soft_lut(int nb, int q, uint16_t* lut, double* margin) {
    if (nb < 1 || nb > 64 || q < 2 || q > 255) return -1;
    double m = 1.0;
    for (int dy = -ORACLE_DMAX; dy <= ORACLE_DMAX; ++dy)
        for (int dx = -ORACLE_DMAX; dx <= ORACLE_DMAX; ++dx) {
            long idx = (long)(dy + ORACLE_DMAX) * (2 * ORACLE_DMAX + 1) + (dx + ORACLE_DMAX);
            if (dx == 0 && dy == 0) {
                lut[idx] = 0xFFFF;
                continue;
            }
            int k0;
            int a = soft_vote(dx, dy, nb, q, &k0, &m);
            lut[idx] = (uint16_t)(k0 | (a << 8));
        }
    if (margin) *margin = m;
    return 0;
}

/* Per-pixel soft votes [H][W][nb]: Eq. 1 gradients with the strongest
 * channel (as oracle_bin_map), then the two-bin vote; border pixels and
 * (0, 0) gradients vote nothing. */
int oracle_soft_votes(const uint8_t* img, int W, int H, int channels, long pitch, int nb, int q, int32_t* votes) {
    if (channels != 1 && channels != 3) return -1;
    if (nb < 1 || nb > 64 || q < 2 || q > 255) return -1;
    memset(votes, 0, sizeof(int32_t) * (size_t)W * H * nb);
    for (int y = 1; y < H - 1; ++y)
        for (int x = 1; x < W - 1; ++x) {
            int best_dx = 0, best_dy = 0;
            long best_mag = -1;
            for (int c = 0; c < channels; ++c) {
                int dx = img[y * pitch + (long)channels * (x + 1) + c] - img[y * pitch + (long)channels * (x - 1) + c];
                int dy = img[(y + 1) * pitch + (long)channels * x + c] - img[(y - 1) * pitch + (long)channels * x + c];
                long mag = (long)dx * dx + (long)dy * dy;
                if (mag > best_mag) { /* strict: ties keep the lower channel */
                    best_mag = mag;
                    best_dx = dx;
                    best_dy = dy;
                }
            }
            if (best_dx == 0 && best_dy == 0) continue;
            int k0;
            int a = soft_vote(best_dx, best_dy, nb, q, &k0, NULL);
            int32_t* v = votes + ((long)y * W + x) * nb;
            v[k0] += q - a;
            v[(k0 + 1) % nb] += a;
        }
    return 0;
}

/* Overlapping blocks (the "four overlapped sub areas" of a region, Section
 * 3, Fig. 4's caption), read as blocks of 2 x 2 cells with a stride of one
 * cell: block (i, j) of the cell map (positions at the scan stride, r = cell
 * / stride positions per cell) concatenates the histograms of cells (i, j),
 * (i + r, j), (i, j + r), (i + r, j + r) -- quadrant q = 2 cy + cx -- and
 * divides the 4 nb values by sqrt(sum of their squares + eps^2).
 * blocks: [ncy - r][ncx - r][4 nb] doubles. */
int oracle_block_norm(const int32_t* cells, int ncx, int ncy, int nb, int r, double eps, double* blocks) {
    int nbx = ncx - r, nby = ncy - r;
    if (r < 1 || nb < 1) return -1;
    if (nbx <= 0 || nby <= 0) return 0;
    for (int j = 0; j < nby; ++j)
        for (int i = 0; i < nbx; ++i) {
            double* out = blocks + ((long)j * nbx + i) * 4 * nb;
            double ss = 0.0;
            for (int q = 0; q < 4; ++q) {
                int ci = i + (q & 1) * r, cj = j + (q >> 1) * r;
                for (int b = 0; b < nb; ++b) {
                    double v = (double)cells[((long)cj * ncx + ci) * nb + b];
                    out[q * nb + b] = v;
                    ss += v * v;
                }
            }
            double norm = sqrt(ss + eps * eps);
            for (int k = 0; k < 4 * nb; ++k) out[k] = norm > 0.0 ? out[k] / norm : 0.0;
        }
    return 0;
}

/* Image pyramid level by 2:1 decimation: level l+1 keeps the pixels (2x, 2y)
 * of level l; sizes floor(W/2) x floor(H/2).  dst is packed (pitch W/2*ch). */
int oracle_decimate(const uint8_t* src, int W, int H, int channels, long pitch, uint8_t* dst) {
    int w2 = W / 2, h2 = H / 2;
    for (int y = 0; y < h2; ++y)
        for (int x = 0; x < w2; ++x)
            for (int c = 0; c < channels; ++c)
                dst[((long)y * w2 + x) * channels + c] =
                    src[(long)(2 * y) * pitch + (long)(2 * x) * channels + c];
    return 0;
}
