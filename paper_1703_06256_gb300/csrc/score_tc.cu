// score_tc.cu -- window score on the tensor cores (tcgen05), as an implicit
// GEMM (the paper's linear score, Sections 1 and 4: the inner product of the
// window feature with a weight vector at every scan position).
//
//   S[py][px] = bias + sum_{j<16} sum_{i<8} sum_{b<N_b} w[j][i][b] * C[py + j r][px + i r][b]
//
// Output rows split into r residue classes: class phi holds the rows
// py = py_lo + phi + r t (t < Tc), and they read only the cell rows
// rho = py_lo + phi + r rho' of the same class (rho' < Tc + 15), with
// py + j r = rho  <=>  j = rho' - t.  So for one cell row rho',
//
//   S[t][px] += sum_{i, b} C_rho'[px + i r][b] * Wband_rho'[t][(i, b)],
//   Wband_rho'[t][(i, b)] = w[rho' - t][i][b]  (0 unless 0 <= rho' - t < 16)
//
// is a GEMM with M = windows px, N = Tc output rows, K = 8 cells x N_b bins,
// accumulated over the Tc + 15 cell rows of the class into one fixed block
// of TMEM columns.
//
// Neither operand is materialised per row.  A: in shared memory a cell row is
// kept as in HBM, [px][N_b bins] bf16.  With N_b = 8 a cell is 16 bytes, so
// the 8 x 16-byte core matrix (windows px0 + 8g .. +7, cell i) starts at
// byte (8g + i r) * 16: the descriptor of an MMA over cells i, i+1 points at
// cell i r with a K-direction core-matrix stride (LBO) of r * 16 bytes and an
// M-direction stride (SBO) of 128 bytes -- an im2col done by the descriptor.
// With N_b = 16 a cell is two 16-byte halves (bins 0-7, 8-15); the same
// descriptor over 16-byte rows makes A row m half m % 2 of window m / 2, so
// a CTA covers 64 windows, and each half h of the weights gets its own MMA
// into its own Tc columns: only half h of the rows in those columns is kept,
// and the epilogue adds the two halves of a window (neighbouring lanes).
// B: for each cell i and half h the 16 filter rows sit in a zero-padded,
// reversed plane plane_{i,h}[v] = w[Tc + 14 - v][i][8h .. 8h + 7] (16 bytes);
// rows t = 0..Tc-1 of Wband_rho' are the consecutive plane rows
// v = Tc + 14 - rho' + t, so the band of cell row rho' is the same planes
// with the descriptor start moved back 16 bytes per row (LBO = distance
// between the planes of cells i and i + 1, SBO = 128 bytes).
//
// One CTA: 128 accumulator rows (one TMEM lane each) by the Tc output rows of
// one residue class (blockIdx.z = phi), so the r classes of a row band run in
// separate CTAs and read disjoint cell rows; 4 warps.
// Warp 0 lane 0 streams cell rows into a ring of shared-memory stages with
// bulk async copies (mbarrier full/empty pipeline), warp 1 lane 0 issues
// the MMAs (the first of each class overwrites its columns, the rest
// accumulate), then all four warps read their 32 TMEM lanes back
// (tcgen05.ld), add the bias and store.  Every wait is bounded: on a timeout
// the kernel flags the device status, lets its copies and MMAs drain (again
// bounded), frees its TMEM and returns.
//
// Exactness: bin counts (<= 64) are exact in bf16, products of bf16 values
// are exact in fp32.  With int8 weights (exact in bf16) every partial sum is
// an integer of magnitude <= 127 * 8192 (a window has 8192 pixels, each in
// at most one bin) < 2^24, so the fp32 accumulation is exact in any order
// and the int32 scores are bit-exact.
#include <cuda_bf16.h>

#include <cmath>
#include <type_traits>

#include "batch_plan.cuh"
#include "internal.cuh"
#include "ptx.cuh"
#include "tcgen05.cuh"

namespace fasthog {

namespace {

using namespace tc;

constexpr int kCX = 8, kCY = 16;
constexpr int kM = 128;                   // windows per CTA (TMEM lanes)
constexpr int kThreads = 128;
constexpr int kStages = 4;
constexpr int kRowsPerStage = 4;

constexpr int kMaxFilters = 32;  // filters per launch (a group; the API splits larger sets)
// Independent accumulators: the MMAs of K step ks (cells 2ks, 2ks+1) go to
// accumulator ks, so consecutive MMAs never wait on each other's result;
// the epilogue adds the four in a fixed order.
constexpr int kAcc = 4;
constexpr size_t kMaxSmem = 227 * 1024;

// Per-filter biases, passed by value (captured with the launch).
struct FilterBias {
    float b[kMaxFilters];
};

struct TcGeom {
    int r, Tc, rows;      // residue count, output rows per CTA (one class), cell rows per CTA
    int halves;           // N_b / 8: 16-byte halves of a cell (1 or 2)
    int filters;          // filters scored by one CTA
    int parts;            // bf16 parts per weight (3 for f32 weights, else 1)
    int wpc;              // windows per CTA: 128 / halves
    int row_cells;        // cells staged per cell row: wpc + (kCX - 1) r
    int row_bytes;        // row_cells * 16 * halves
    int stage_bytes;      // kRowsPerStage rows
    int plane_rows;       // rows of one band plane: 2 Tc + 16
    int plane_bytes;      // plane_rows * 16
    int band_bytes;       // filters * kCX * halves planes
    int cols;             // TMEM columns allocated (power of two >= 32)
    __host__ __device__ TcGeom(int r_, int Tc_, int halves_, int filters_ = 1, int parts_ = 1)
        : r(r_), Tc(Tc_), halves(halves_), filters(filters_), parts(parts_) {
        rows = Tc + kCY - 1;
        wpc = kM / halves;
        row_cells = wpc + (kCX - 1) * r;
        row_bytes = row_cells * 16 * halves;
        stage_bytes = kRowsPerStage * row_bytes;
        plane_rows = 2 * Tc + 16;
        plane_bytes = plane_rows * 16;
        band_bytes = filters * parts * kCX * halves * plane_bytes;
        cols = 32;
        while (cols < kAcc * filters * halves * Tc) cols *= 2;
    }
    __host__ __device__ size_t smem_bytes() const {
        return 1024 + (size_t)band_bytes + (size_t)kStages * stage_bytes + 256;
    }
};

// Columns c0 .. c0 + 15 of filter f, half h: the sum of the kAcc accumulators
// ((d0 + d1) + (d2 + d3)), as f32 bit patterns.
__device__ __forceinline__ void acc_sum(uint32_t lane_base, int f, int h, int n_filters, int halves, int Tc, int c0,
                                        uint32_t (&v)[16]) {
    uint32_t d[kAcc][16];
#pragma unroll
    for (int a = 0; a < kAcc; ++a)
        tmem_load16_async(lane_base + (uint32_t)(((a * n_filters + f) * halves + h) * Tc + c0), d[a]);
    tmem_wait_ld();
#pragma unroll
    for (int c = 0; c < 16; ++c)
        v[c] = __float_as_uint((__uint_as_float(d[0][c]) + __uint_as_float(d[1][c])) +
                               (__uint_as_float(d[2][c]) + __uint_as_float(d[3][c])));
}

// BATCH = false: one image, CTA (blockIdx.x, .y, .z) = (window column, row
// band, residue class).  BATCH = true: the CTAs of every item of a batch
// plan in one 1-D grid; each CTA finds its item and its (column, band,
// class) from the plan and overrides the image arguments.
template <int NB, typename WT, typename OutT, bool BATCH>
__global__ void __launch_bounds__(kThreads, 1)
    score_tc_kernel(const uint16_t* __restrict__ cells, int ncx, int ncy, int r, int Tc, const WT* __restrict__ w,
                    float bias, int n_filters, const __grid_constant__ FilterBias fbias, int nx, int ny,
                    OutT* __restrict__ scores,
                    const PlanItem* __restrict__ items, int n_items, unsigned int* status) {
    extern __shared__ uint8_t smem_raw[];
    constexpr int HALVES = NB / 8, CB = NB * 2;  // 16-byte halves per cell, bytes per cell
    constexpr int PARTS = weight_parts<WT>();
    const TcGeom G(r, Tc, HALVES, n_filters, PARTS);
    // 1024-byte aligned working area: band planes, A stages, barriers
    uint8_t* base = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
    uint8_t* band = base;
    uint8_t* stages = base + G.band_bytes;
    uint64_t* bars = reinterpret_cast<uint64_t*>(stages + (size_t)kStages * G.stage_bytes);
    uint64_t* full = bars;                                // [kStages]
    uint64_t* empty = bars + kStages;                     // [kStages]
    uint64_t* done = bars + 2 * kStages;
    uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(bars + 2 * kStages + 1);
    __shared__ int aborted;

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    int xt = blockIdx.x, yband = blockIdx.y, phi = blockIdx.z;  // phi: residue class of this CTA
    if constexpr (BATCH) {
        const PlanItem* it = items + find_item<Stage::kScore>(items, n_items, (int)blockIdx.x);
        const int local = (int)blockIdx.x - it->score_c0, tx = it->score_tx, bands = it->score_bands;
        xt = local % tx;
        yband = (local / tx) % bands;
        phi = local / (tx * bands);
        cells = static_cast<const uint16_t*>(it->it.cells);
        scores = static_cast<OutT*>(it->it.scores);
        ncx = it->ncx;
        ncy = it->ncy;
        nx = it->nx;
        ny = it->ny;
    }
    const int px0 = xt * G.wpc;
    const int py_lo = yband * Tc * r + phi;  // first output row; rows step by r

    // band planes, one per (cell i, half h): plane_{i,h}[v][b] = w[Tc + 14 - v][i][8h + b]
    // for filter rows 0..15, zero elsewhere.  Thread t < 128 moves the bins of filter cell
    // (j, i) = (t / 8, t % 8), 8 per load; the rows of the planes that hold no filter row are
    // zeroed by 16-byte stores.
    // With several filters, filter f's planes follow filter f - 1's.
    {
        const int j = tid / kCX, i = tid % kCX;
        for (int f = 0; f < n_filters; ++f) {
#pragma unroll
            for (int part = 0; part < PARTS; ++part) {
#pragma unroll
                for (int h = 0; h < HALVES; ++h) {
                    const uint4 v =
                        load_weight8_part<WT>(w, f * (kCX * kCY * NB) + (j * kCX + i) * NB + 8 * h, part);
                    const int plane = ((f * PARTS + part) * kCX + i) * HALVES + h;
                    *reinterpret_cast<uint4*>(band + (size_t)plane * G.plane_bytes + (size_t)(Tc + 14 - j) * 16) = v;
                }
            }
        }
        const int zero_rows = G.plane_rows - kCY;  // v < Tc - 1 or v > Tc + 14
        for (int e = tid; e < n_filters * PARTS * kCX * HALVES * zero_rows; e += kThreads) {
            const int pi = e / zero_rows, zr = e % zero_rows;
            const int vrow = zr < Tc - 1 ? zr : zr + kCY;
            *reinterpret_cast<uint4*>(band + (size_t)pi * G.plane_bytes + (size_t)vrow * 16) = make_uint4(0, 0, 0, 0);
        }
    }
    if (tid == 0) {
        aborted = 0;
        for (int s = 0; s < kStages; ++s) {
            ptx::mbar_init(&full[s], 1);
            ptx::mbar_init(&empty[s], 1);
        }
        ptx::mbar_init(done, 1);
        ptx::fence_mbar_init();
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                         ptx::smem_addr(tmem_slot)),
                     "r"(G.cols)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    // the band was written by ordinary stores; the MMAs read it through the async proxy
    ptx::fence_proxy_async_smem();
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *tmem_slot;
    pdl_trigger();  // tail of the path: the successor is small, launch it early
    pdl_wait();  // set-up above read only the weights; the cell rows come from the predecessor

    const int n_stage_loads = (G.rows + kRowsPerStage - 1) / kRowsPerStage;
    const int valid_cells = min(G.row_cells, ncx - px0);  // > 0: px0 < nx <= ncx
    if (warp == 0 && lane == 0) {
        // producer: cell rows py_lo + r rho (rho < rows) into the stage ring
        int armed = 0;  // stages whose copies were issued
        for (int k = 0; k < n_stage_loads; ++k) {
            const int s = k % kStages;
            if (!ptx::mbar_wait_bounded(&empty[s], ((k / kStages) & 1) ^ 1, kWaitLimitNs)) {
                atomicOr(status, kStatusTimeout);
                atomicExch(&aborted, 1);
                break;
            }
            uint32_t bytes = 0;
            for (int q = 0; q < kRowsPerStage; ++q) {
                const int row = py_lo + r * (k * kRowsPerStage + q);
                if (k * kRowsPerStage + q < G.rows && row < ncy) bytes += (uint32_t)valid_cells * CB;
            }
            ptx::mbar_arrive_expect_tx(&full[s], bytes);
            for (int q = 0; q < kRowsPerStage; ++q) {
                const int row = py_lo + r * (k * kRowsPerStage + q);
                if (k * kRowsPerStage + q < G.rows && row < ncy)
                    ptx::bulk_g2s(stages + (size_t)s * G.stage_bytes + (size_t)q * G.row_bytes,
                                  cells + ((size_t)row * ncx + px0) * NB, (uint32_t)valid_cells * CB, &full[s]);
            }
            armed = k + 1;
        }
        if (*reinterpret_cast<volatile int*>(&aborted)) {
            // let the copies already issued land before the CTA can exit (bounded)
            for (int k = armed > kStages ? armed - kStages : 0; k < armed; ++k)
                ptx::mbar_wait_bounded(&full[k % kStages], (k / kStages) & 1, kWaitLimitNs);
        }
    } else if (warp == 1 && lane == 0) {
        // MMA issuer
        const uint32_t idesc = instr_desc(kM, Tc);
        const uint32_t band_addr = ptx::smem_addr(band);
        for (int k = 0; k < n_stage_loads; ++k) {
            const int s = k % kStages;
            if (!ptx::mbar_wait_bounded(&full[s], (k / kStages) & 1, kWaitLimitNs) ||
                *reinterpret_cast<volatile int*>(&aborted)) {
                atomicOr(status, kStatusTimeout);
                atomicExch(&aborted, 1);
                break;
            }
            tc_fence_after();
            for (int q = 0; q < kRowsPerStage; ++q) {
                const int rho = k * kRowsPerStage + q;  // cell row within the class
                if (rho >= G.rows) break;
                const uint32_t a_addr = ptx::smem_addr(stages + (size_t)s * G.stage_bytes + (size_t)q * G.row_bytes);
                const uint32_t b_row = band_addr + (uint32_t)((Tc + 14 - rho) * 16);
#pragma unroll
                for (int ks = 0; ks < kCX / 2; ++ks) {
                    // cells 2ks, 2ks+1: A at cell 2ks*r (with two halves, A row m is half m % 2 of
                    // window m / 2), B at the planes of half h of cells 2ks, 2ks+1, D at h * Tc
                    const uint64_t ad = smem_desc(a_addr + (uint32_t)(2 * ks * r * CB), (uint32_t)(r * CB), 128);
                    for (int f = 0; f < n_filters; ++f) {
#pragma unroll
                        for (int part = 0; part < PARTS; ++part) {
#pragma unroll
                            for (int h = 0; h < HALVES; ++h) {
                                const int plane = ((f * PARTS + part) * kCX + 2 * ks) * HALVES + h;
                                const uint64_t bd = smem_desc(b_row + (uint32_t)(plane * G.plane_bytes),
                                                              (uint32_t)(HALVES * G.plane_bytes), 128);
                                const int acc = (ks * n_filters + f) * HALVES + h;  // accumulator ks
                                mma_bf16(tmem + (uint32_t)(acc * Tc), ad, bd, idesc,
                                         (rho == 0 && part == 0) ? 0u : 1u);
                            }
                        }
                    }
                }
            }
            mma_commit(&empty[s]);  // the stage is free once these MMAs have read it
        }
        mma_commit(done);
    }
    __syncwarp();

    // epilogue: all warps, after the last MMA
    const bool ok = ptx::mbar_wait_bounded(done, 0, kWaitLimitNs);
    if (!ok) atomicOr(status, kStatusTimeout);
    tc_fence_after();
    __syncthreads();
    // lane m of the accumulator: window px0 + m (one half) or px0 + m / 2, half m % 2 (two
    // halves, whose valid sums are columns [0, Tc) of even rows and [Tc, 2 Tc) of odd rows)
    const int m = warp * 32 + lane;
    const int px = px0 + m / HALVES;
    const bool writer = HALVES == 1 || (lane & 1) == 0;
    if (ok && !*reinterpret_cast<volatile int*>(&aborted)) {
        for (int f = 0; f < n_filters; ++f) {
            const float bias_f = n_filters == 1 ? bias : fbias.b[f];
            OutT* out = scores + (size_t)f * nx * ny;
            const uint32_t lane_base = tmem + ((uint32_t)(warp * 32) << 16);
            for (int c0 = 0; c0 < Tc; c0 += 16) {
                uint32_t v[16];
                acc_sum(lane_base, f, 0, n_filters, HALVES, Tc, c0, v);
                if constexpr (HALVES == 2) {
                    uint32_t u[16];
                    acc_sum(lane_base, f, 1, n_filters, HALVES, Tc, c0, u);
#pragma unroll
                    for (int c = 0; c < 16; ++c) {
                        const float mine = __uint_as_float((lane & 1) ? u[c] : v[c]);
                        const float other = __shfl_xor_sync(0xffffffffu, mine, 1);
                        v[c] = __float_as_uint((lane & 1) ? other + mine : mine + other);  // half 0 + half 1
                    }
                }
#pragma unroll
                for (int c = 0; c < 16; ++c) {
                    const int py = py_lo + r * (c0 + c);
                    if (writer && px < nx && py < ny) {
                        const float sc = __uint_as_float(v[c]) + bias_f;
                        if constexpr (std::is_same<OutT, int32_t>::value) {
                            out[(size_t)py * nx + px] = __float2int_rn(sc);  // exact integer
                        } else {
                            out[(size_t)py * nx + px] = sc;
                        }
                    }
                }
            }
        }
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 0) {
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(G.cols) : "memory");
    }
}

int choose_tc(int nx, int ny, int r, int wpc) {
    // 32 output rows per CTA when that still gives every SM a CTA, else 16
    const long tiles_x = (nx + wpc - 1) / wpc;
    const int tuned = tune_get(HOG_TUNE_SCORE_TC_ROWS);
    if (tuned == 16 || tuned == 32) return tuned;  // the banded kernel's two heights; other values: its own choice
    const long ctas32 = tiles_x * ((ny + 32 * r - 1) / (32 * r)) * r;
    return ctas32 >= sm_count() ? 32 : 16;
}

template <int NB, typename WT, typename OutT>
hog_status launch_t(const uint16_t* cells, int ncx, int ncy, int r, const void* w, float bias, void* scores,
                    cudaStream_t st) {
    const int nx = ncx - (kCX - 1) * r, ny = ncy - (kCY - 1) * r;
    if (nx <= 0 || ny <= 0) return HOG_OK;
    unsigned int* status = nullptr;
    hog_status s = device_status_word(&status);
    if (s != HOG_OK) return s;
    const int wpc = kM / (NB / 8);
    const int Tc = choose_tc(nx, ny, r, wpc);
    const TcGeom G(r, Tc, NB / 8, 1, weight_parts<WT>());
    if (G.cols > 512) return HOG_ERR_UNSUPPORTED;
    const size_t smem = G.smem_bytes();
    auto kern = score_tc_kernel<NB, WT, OutT, false>;
    cudaError_t e = smem_at_least<score_tc_kernel<NB, WT, OutT, false>>(smem);
    if (e != cudaSuccess) return cuda_fail(e);
    dim3 grid((nx + wpc - 1) / wpc, (ny + Tc * r - 1) / (Tc * r), r);
    return launch_pdl(kern, grid, dim3(kThreads), smem, st, cells, ncx, ncy, r, Tc, static_cast<const WT*>(w), bias,
                      1, FilterBias{}, nx, ny, static_cast<OutT*>(scores), static_cast<const PlanItem*>(nullptr), 0,
                      status);
}

template <int NB, typename WT, typename OutT>
hog_status launch_batch_t(const PlanHeader& h, const void* plan_dev, const void* w, float bias, cudaStream_t st) {
    unsigned int* status = nullptr;
    hog_status s = device_status_word(&status);
    if (s != HOG_OK) return s;
    const TcGeom G(h.r, h.score_tc, NB / 8, 1, weight_parts<WT>());
    if (G.cols > 512) return HOG_ERR_UNSUPPORTED;
    const size_t smem = G.smem_bytes();
    auto kern = score_tc_kernel<NB, WT, OutT, true>;
    cudaError_t e = smem_at_least<score_tc_kernel<NB, WT, OutT, true>>(smem);
    if (e != cudaSuccess) return cuda_fail(e);
    return launch_pdl(kern, dim3(h.score_ctas), dim3(kThreads), smem, st, static_cast<const uint16_t*>(nullptr), 0,
                      0, h.r, h.score_tc, static_cast<const WT*>(w), bias, 1, FilterBias{}, 0, 0,
                      static_cast<OutT*>(nullptr), plan_items(plan_dev), h.n_items, status);
}

// Several filters: groups of filters per launch, as many as the shared
// memory (their weight planes) and the TMEM columns allow.
template <int NB, typename WT, typename OutT>
hog_status launch_multi_t(const uint16_t* cells, int ncx, int ncy, int r, const WT* w, int n_filters,
                          const float* biases, OutT* scores, cudaStream_t st) {
    const int nx = ncx - (kCX - 1) * r, ny = ncy - (kCY - 1) * r;
    if (nx <= 0 || ny <= 0) return HOG_OK;
    unsigned int* status = nullptr;
    hog_status s = device_status_word(&status);
    if (s != HOG_OK) return s;
    const int wpc = kM / (NB / 8);
    int Tc = choose_tc(nx, ny, r, wpc);
    auto fits = [&](int tc, int g) {
        const TcGeom G(r, tc, NB / 8, g, weight_parts<WT>());
        return G.cols <= 512 && G.smem_bytes() <= kMaxSmem;
    };
    int group = kMaxFilters < n_filters ? kMaxFilters : n_filters;
    while (group > 1 && !fits(Tc, group)) --group;
    if (!fits(Tc, group) && Tc == 32) {
        Tc = 16;
        group = kMaxFilters < n_filters ? kMaxFilters : n_filters;
        while (group > 1 && !fits(Tc, group)) --group;
    }
    if (!fits(Tc, group)) return HOG_ERR_UNSUPPORTED;
    auto kern = score_tc_kernel<NB, WT, OutT, false>;
    const size_t smem_max = TcGeom(r, Tc, NB / 8, group, weight_parts<WT>()).smem_bytes();
    cudaError_t e = smem_at_least<score_tc_kernel<NB, WT, OutT, false>>(smem_max);
    if (e != cudaSuccess) return cuda_fail(e);
    const dim3 grid((nx + wpc - 1) / wpc, (ny + Tc * r - 1) / (Tc * r), r);
    const size_t per_filter = (size_t)kCX * kCY * NB;
    for (int f0 = 0; f0 < n_filters; f0 += group) {
        const int g = n_filters - f0 < group ? n_filters - f0 : group;
        FilterBias fb{};
        for (int k = 0; k < g; ++k) {
            const float b = biases[f0 + k];
            fb.b[k] = std::is_same<OutT, int32_t>::value ? (float)std::llround((double)b) : b;
        }
        s = launch_pdl(kern, grid, dim3(kThreads), TcGeom(r, Tc, NB / 8, g, weight_parts<WT>()).smem_bytes(), st,
                       cells, ncx, ncy, r, Tc,
                       w + f0 * per_filter, fb.b[0], g, fb, nx, ny, scores + (size_t)f0 * nx * ny,
                       static_cast<const PlanItem*>(nullptr), 0, status);
        if (s != HOG_OK) return s;
    }
    return HOG_OK;
}

template <int NB>
hog_status multi_by_w(const uint16_t* cells, int ncx, int ncy, int r, const void* w, int w_dtype, int n_filters,
                      const float* biases, void* scores, cudaStream_t st) {
    if (w_dtype == HOG_F32)
        return launch_multi_t<NB, float, float>(cells, ncx, ncy, r, static_cast<const float*>(w), n_filters, biases,
                                                static_cast<float*>(scores), st);
    if (w_dtype == HOG_BF16)
        return launch_multi_t<NB, uint16_t, float>(cells, ncx, ncy, r, static_cast<const uint16_t*>(w), n_filters,
                                                   biases, static_cast<float*>(scores), st);
    if (w_dtype == HOG_I8)
        return launch_multi_t<NB, int8_t, int32_t>(cells, ncx, ncy, r, static_cast<const int8_t*>(w), n_filters,
                                                   biases, static_cast<int32_t*>(scores), st);
    return HOG_ERR_UNSUPPORTED;
}

template <int NB>
hog_status batch_by_w(const PlanHeader& h, const void* plan_dev, const void* w, int w_dtype, float bias,
                      cudaStream_t st) {
    if (w_dtype == HOG_F32) return launch_batch_t<NB, float, float>(h, plan_dev, w, bias, st);
    if (w_dtype == HOG_BF16) return launch_batch_t<NB, uint16_t, float>(h, plan_dev, w, bias, st);
    if (w_dtype == HOG_I8) return launch_batch_t<NB, int8_t, int32_t>(h, plan_dev, w, bias, st);
    return HOG_ERR_UNSUPPORTED;
}

template <int NB>
hog_status by_w(const uint16_t* cells, int ncx, int ncy, int r, const void* w, int w_dtype, float bias, void* scores,
                cudaStream_t st) {
    if (w_dtype == HOG_F32) return launch_t<NB, float, float>(cells, ncx, ncy, r, w, bias, scores, st);
    if (w_dtype == HOG_BF16) return launch_t<NB, uint16_t, float>(cells, ncx, ncy, r, w, bias, scores, st);
    if (w_dtype == HOG_I8) return launch_t<NB, int8_t, int32_t>(cells, ncx, ncy, r, w, bias, scores, st);
    return HOG_ERR_UNSUPPORTED;
}

}  // namespace

hog_status launch_score_tc_batch(const PlanHeader& h, const void* plan_dev, const void* w, int w_dtype, float bias,
                                 cudaStream_t st) {
    if (h.score_ctas == 0) return HOG_OK;
    return h.n_bins == 16 ? batch_by_w<16>(h, plan_dev, w, w_dtype, bias, st)
                          : batch_by_w<8>(h, plan_dev, w, w_dtype, bias, st);
}

int score_tc_rows_for(long ctas32) {
    const int tuned = tune_get(HOG_TUNE_SCORE_TC_ROWS);
    return (tuned == 16 || tuned == 32) ? tuned : (ctas32 >= kNumSMs ? 32 : 16);
}

int score_tc_windows(int n_bins) { return kM / (n_bins == 16 ? 2 : 1); }

bool score_tc_fills_gpu(int ncx, int ncy, int n_bins, int r) {
    const long nx = (long)ncx - (kCX - 1) * r, ny = (long)ncy - (kCY - 1) * r;
    if (nx <= 0 || ny <= 0) return false;
    const long wpc = score_tc_windows(n_bins);
    const long ctas = ((nx + wpc - 1) / wpc) * ((ny + 16 * r - 1) / (16 * r)) * r;  // at 16 rows per CTA
    return ctas >= sm_count();
}

bool score_tc_supported(int cell_dtype, int n_bins, int cells_x, int cells_y, int r, int ncx) {
    (void)ncx;
    return cell_dtype == HOG_BF16 && (n_bins == 8 || n_bins == 16) && cells_x == kCX && cells_y == kCY &&
           (r == 1 || r == 2 || r == 4);
}

hog_status launch_score_tc_multi(const uint16_t* cells_bf16, int ncx, int ncy, int n_bins, int r, const void* w,
                                 int w_dtype, int n_filters, const float* biases, void* scores, cudaStream_t st) {
    if (reinterpret_cast<uintptr_t>(cells_bf16) % 16 != 0) return HOG_ERR_UNSUPPORTED;
    return n_bins == 16 ? multi_by_w<16>(cells_bf16, ncx, ncy, r, w, w_dtype, n_filters, biases, scores, st)
                        : multi_by_w<8>(cells_bf16, ncx, ncy, r, w, w_dtype, n_filters, biases, scores, st);
}

hog_status launch_score_tc(const uint16_t* cells_bf16, int ncx, int ncy, int n_bins, int cells_x, int cells_y, int r,
                           const void* w, int w_dtype, float bias, void* scores, cudaStream_t st) {
    (void)cells_x;
    (void)cells_y;
    if (reinterpret_cast<uintptr_t>(cells_bf16) % 16 != 0) return HOG_ERR_UNSUPPORTED;
    return n_bins == 16 ? by_w<16>(cells_bf16, ncx, ncy, r, w, w_dtype, bias, scores, st)
                        : by_w<8>(cells_bf16, ncx, ncy, r, w, w_dtype, bias, scores, st);
}

}  // namespace fasthog
