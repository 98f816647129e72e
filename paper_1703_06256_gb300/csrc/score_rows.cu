// score_rows.cu -- window score on the tensor cores, one GEMM per cell row
// (the paper's linear score, Sections 1 and 4: the inner product of the
// window feature with a weight vector at every scan position), for windows
// of 8 x 16 cells of 8 bins.
//
//   P[c][px][j] = sum_{i<8, b<8} w[j][i][b] * C[c][px + i r][b]
//   S[py][px]   = bias + sum_{j<16} P[py + j r][px][j]
//
// P of one cell row c is a dense GEMM: M = 128 windows px, N = the 16 filter
// rows j, K = 8 cells x 8 bins.  A is the cell row in shared memory as it
// lies in HBM ([px][8 bins] bf16, 16 bytes per cell): the 8 x 16-byte core
// matrix (windows px0 + 8g .. +7, cell i) starts at byte (8g + i r) * 16, so
// an MMA over cells i, i + 1 takes a descriptor at cell i r with a K-direction
// stride (LBO) of r * 16 bytes and an M-direction stride (SBO) of 128 bytes:
// the descriptor does the im2col.  B holds, per cell i, the N rows of its
// weights (one row per filter row j and weight part; 8 bins each).  f32
// weights become three exact bf16 parts (each the bf16 rounding of what the
// parts before it leave), which sit side by side as N = 48 accumulator
// columns; bf16 and int8 weights (exact in bf16) are one part, N = 16.
// Counts are exact in bf16 and a count times a bf16 part is exact in f32, so
// every product is exact; only the f32 sums round.
//
// Several filters (hog_window_score_multi) widen the GEMM: filter f's rows
// follow filter f - 1's in B, N = 16 x parts x filters (up to 256), each
// filter keeps its own ring of running sums, and one pass over the cell rows
// scores all of them; a filter's sums are formed in the same order as when it
// is scored alone, so its scores are the same bit for bit.
//
// Every MMA row is useful: a CTA streams the cell rows py0 .. py1 - 1 + 15 r
// of one strip of 128 windows through a ring of shared-memory stages of up to
// four rows each (one bulk copy per row, one mbarrier per stage), one thread
// issues 4 MMAs per row (K = 64) into the stage's TMEM accumulator (row t of
// the stage at column t N; two to four accumulators in turn), and eight
// epilogue warps (two groups of four, one warp per 32 TMEM lanes in each:
// lane m is window px0 + m) read P back row by row, add the parts ((lo +
// mid) + hi), and add P_j into a running sum per window py = c - j r kept
// in shared memory (a ring of 16 r rows per window column).  With r > 1 one
// group takes the cell rows of even index and the other those of odd index:
// their ring rows never meet.  After row c the window py = c - 15 r has all
// 16 of its rows: it is written (with the bias) and its ring slot cleared.
// Rows of windows above py0 fall in the ring too and are cleared unwritten.
// Synchronising once per stage and per accumulator rather than once per row
// keeps the handoffs between the copy, MMA and epilogue threads off the
// critical path.
//
// Every wait is bounded: on a timeout the kernel sets the device status bit,
// lets its copies and MMAs drain (again bounded), frees TMEM and returns.
#include <cmath>
#include <type_traits>

#include "batch_plan.cuh"
#include "internal.cuh"
#include "ptx.cuh"
#include "tcgen05.cuh"

namespace fasthog {

namespace {

using namespace tc;

constexpr int kM = 128;        // windows per CTA (TMEM lanes)
constexpr int kEpiWarps = 8;   // two groups of four, one warp per 32 TMEM lanes in each
constexpr int kThreads = 32 * (kEpiWarps + 2);
constexpr int kStages = 4;     // stages (of STEP cell rows each) in flight
constexpr int kMaxBufs = 4;    // TMEM accumulators at most

constexpr int kMaxFilters = 16;  // filters per launch at most (N <= 256 with one part)

// Per-filter biases, passed by value (captured with the launch).
struct RowsBias {
    float b[kMaxFilters];
};

// Shared-memory and TMEM layout for nf filters of `parts` weight parts at r.
constexpr int kSplit = 4;       // CTAs of a cluster that share a window block by filter rows (4 each)
constexpr int kSplitRows = 16;  // output rows per CTA at most when split (their partial sums meet in shared memory)

struct RowsGeom {
    int N, STEP, BUF, NBUF, COLS, RS, ROW_BYTES, PLANE_BYTES;
    size_t planes, stages, ring, bars;
    // split: one filter, 4 of its 16 rows per CTA (N = 16 with the parts of the 4 rows, zero-padded)
    __host__ __device__ RowsGeom(int r, int parts, int nf, bool split = false) {
        N = split ? 16 : 16 * parts * nf;                     // accumulator columns of one row
        STEP = N <= 64 ? 4 : (N <= 128 ? 2 : 1);              // cell rows per stage and per accumulator
        BUF = 16;
        while (BUF < STEP * N) BUF *= 2;                      // column stride of the accumulators
        NBUF = BUF <= 128 ? kMaxBufs : 2;                     // at most 512 TMEM columns
        COLS = NBUF * BUF < 32 ? 32 : NBUF * BUF;             // TMEM columns allocated
        RS = 16 * r;                                          // ring rows per window column and filter
        ROW_BYTES = (kM + 7 * r) * 16;
        PLANE_BYTES = N * 16;                                 // one cell's weights: N rows of 8 bf16
        planes = (size_t)8 * PLANE_BYTES;
        stages = (size_t)kStages * STEP * ROW_BYTES;
        ring = split ? (size_t)kSplit * kSplitRows * kM * 4     // the partial sums of the cluster's CTAs
                     : (size_t)nf * RS * kM * 4;
        bars = (2 * kStages + 2 * kMaxBufs + 2) * 8;
    }
    __host__ __device__ size_t smem_bytes() const { return 1024 + planes + stages + ring + bars; }
};

// The epilogue of one filter: the running sums of the windows in flight stay
// in registers.  A group's cell rows arrive two (r > 1) or four (r = 1) per
// stage of four; counting the group's rows with u, row u adds P_j to the
// window u - j H (H = r / 2, or 1 for r = 1) and completes the window
// u - 15 H.  The windows in flight fit a ring of 16 H registers, indexed at
// compile time: the loop over stages is unrolled by one turn of the ring.
template <int R, int PARTS, typename OutT>
__device__ __forceinline__ void epilogue_one_filter(uint32_t lane_base, int nsteps, int nrows, int py0, int nbuf,
                                                    int buf_cols, int grp, int px, int nx, float bias,
                                                    OutT* __restrict__ scores, uint64_t* dfull, uint64_t* dempty,
                                                    int* aborted, unsigned int* status) {
    constexpr int N = 16 * PARTS;
    constexpr int G2 = R > 1 ? 2 : 1;   // epilogue groups that share the rows
    constexpr int H = R > 1 ? R / 2 : 1;
    constexpr int RG = 16 * H;          // ring registers
    constexpr int RPS = 4 / G2;         // the group's rows per stage of four
    constexpr int PERIOD = RG / RPS;    // stages per turn of the ring
    const int lane = threadIdx.x & 31;
    const int t0 = R > 1 ? ((grp - py0) & 1) : 0;  // the group's first row within a stage
    float ring[RG];
#pragma unroll
    for (int i = 0; i < RG; ++i) ring[i] = 0.f;
    for (int k0 = 0; k0 < nsteps; k0 += PERIOD) {
#pragma unroll
        for (int kk = 0; kk < PERIOD; ++kk) {
            const int k = k0 + kk;
            if (k >= nsteps) break;
            const int b = k % nbuf, rows = min(4, nrows - 4 * k);
            if (!ptx::mbar_wait_bounded(&dfull[b], (k / nbuf) & 1, kWaitLimitNs) ||
                *reinterpret_cast<volatile int*>(aborted)) {
                atomicOr(status, kStatusTimeout);
                atomicExch(aborted, 1);
                return;
            }
            tc_fence_after();
#pragma unroll
            for (int tp = 0; tp < RPS; ++tp) {
                const int t = t0 + G2 * tp;
                if (t >= rows) break;
                uint32_t v[PARTS][16];
#pragma unroll
                for (int p = 0; p < PARTS; ++p)
                    tmem_load16_async(lane_base + (uint32_t)(b * buf_cols + t * N + 16 * p), v[p]);
                tmem_wait_ld();
                const int u = kk * RPS + tp;  // the group's row, modulo one turn of the ring
#pragma unroll
                for (int j = 0; j < 16; ++j) {
                    float pj;
                    if constexpr (PARTS == 3) {
                        pj = (__uint_as_float(v[2][j]) + __uint_as_float(v[1][j])) + __uint_as_float(v[0][j]);
                    } else {
                        pj = __uint_as_float(v[0][j]);
                    }
                    ring[(u - j * H + 16 * RG) % RG] += pj;
                }
                const int fin = (u - 15 * H + 16 * RG) % RG;  // the window this row completes
                const float sum = ring[fin];
                ring[fin] = 0.f;
                const int py = py0 + 4 * k + t - 15 * R;
                if (py >= py0 && px < nx) {
                    if constexpr (std::is_same<OutT, int32_t>::value) {
                        scores[(size_t)py * nx + px] = __float2int_rn(sum + bias);  // exact integer
                    } else {
                        scores[(size_t)py * nx + px] = sum + bias;
                    }
                }
            }
            // this warp's reads of the accumulator are done: the MMAs of stage k + nbuf may overwrite it
            tc_fence_before();
            __syncwarp();
            if (lane == 0) ptx::mbar_arrive(&dempty[b]);
        }
    }
}

__device__ __forceinline__ uint32_t mapa_shared(uint32_t addr, uint32_t rank) {
    uint32_t r;
    asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(r) : "r"(addr), "r"(rank));
    return r;
}
__device__ __forceinline__ void st_cluster_f32(uint32_t addr, float v) {
    asm volatile("st.shared::cluster.f32 [%0], %1;" ::"r"(addr), "f"(v) : "memory");
}
__device__ __forceinline__ void cluster_sync_all() {
    asm volatile("barrier.cluster.arrive.release.aligned;\n\tbarrier.cluster.wait.acquire.aligned;" ::: "memory");
}

// The epilogue of CTA q of a split cluster (filter rows 4q .. 4q + 3 of one
// filter): as epilogue_one_filter with 4 filter rows, a ring of 4 H
// registers; a window's partial sum over the CTA's rows goes into shared
// memory of the cluster's first CTA, slot [q][py - py0][m].
template <int R, int PARTS>
__device__ __forceinline__ void epilogue_split(uint32_t lane_base, int nsteps, int nrows, int c0, int py0, int py1,
                                               int q, int nbuf, int buf_cols, int grp, int m, uint32_t partial0,
                                               uint64_t* dfull, uint64_t* dempty, int* aborted,
                                               unsigned int* status) {
    constexpr int G2 = R > 1 ? 2 : 1;
    constexpr int H = R > 1 ? R / 2 : 1;
    constexpr int RG = 4 * H;          // ring registers
    constexpr int RPS = 4 / G2;        // the group's rows per stage of four
    constexpr int PERIOD = RG / RPS > 0 ? RG / RPS : 1;
    const int lane = threadIdx.x & 31;
    const int t0 = R > 1 ? ((grp - c0) & 1) : 0;
    const uint32_t leader = mapa_shared(partial0, 0);
    float ring[RG];
#pragma unroll
    for (int i = 0; i < RG; ++i) ring[i] = 0.f;
    for (int k0 = 0; k0 < nsteps; k0 += PERIOD) {
#pragma unroll
        for (int kk = 0; kk < PERIOD; ++kk) {
            const int k = k0 + kk;
            if (k >= nsteps) break;
            const int b = k % nbuf, rows = min(4, nrows - 4 * k);
            if (!ptx::mbar_wait_bounded(&dfull[b], (k / nbuf) & 1, kWaitLimitNs) ||
                *reinterpret_cast<volatile int*>(aborted)) {
                atomicOr(status, kStatusTimeout);
                atomicExch(aborted, 1);
                return;
            }
            tc_fence_after();
#pragma unroll
            for (int tp = 0; tp < RPS; ++tp) {
                const int t = t0 + G2 * tp;
                if (t >= rows) break;
                uint32_t v[16];  // column part * 4 + jj: part `part` of filter row 4q + jj
                tmem_load16_async(lane_base + (uint32_t)(b * buf_cols + t * 16), v);
                tmem_wait_ld();
                const int u = kk * RPS + tp;
#pragma unroll
                for (int jj = 0; jj < 4; ++jj) {
                    float pj;
                    if constexpr (PARTS == 3) {
                        pj = (__uint_as_float(v[8 + jj]) + __uint_as_float(v[4 + jj])) + __uint_as_float(v[jj]);
                    } else {
                        pj = __uint_as_float(v[jj]);
                    }
                    ring[(u - jj * H + 4 * RG) % RG] += pj;
                }
                const int fin = (u - 3 * H + 4 * RG) % RG;  // the window whose 4 rows this row completes
                const float sum = ring[fin];
                ring[fin] = 0.f;
                const int py = c0 + 4 * k + t - (4 * q + 3) * R;  // the window whose last row of 4q..4q+3 this is
                if (py >= py0 && py < py1)
                    st_cluster_f32(leader + (uint32_t)(((q * kSplitRows + (py - py0)) * kM + m) * 4), sum);
            }
            tc_fence_before();
            __syncwarp();
            if (lane == 0) ptx::mbar_arrive(&dempty[b]);
        }
    }
}

// BATCH = false: one image, CTA (blockIdx.x, .y) = (strip of 128 windows,
// range of rows_per_cta output rows).  BATCH = true: the CTAs of every item
// of a batch plan in one 1-D grid; each CTA finds its item and its (strip,
// range) from the plan and overrides the image arguments.
template <int R, typename WT, typename OutT, bool BATCH, bool SPLIT>
__global__ void __launch_bounds__(kThreads, 1)
    score_rows_kernel(const uint16_t* __restrict__ cells, int ncx, int ncy, const WT* __restrict__ w, int nf,
                      const __grid_constant__ RowsBias fbias, int nx, int ny, int rows_per_cta,
                      OutT* __restrict__ scores, const PlanItem* __restrict__ items, int n_items,
                      unsigned int* status) {
    constexpr int PARTS = weight_parts<WT>();
    const RowsGeom G(R, PARTS, nf, SPLIT);
    extern __shared__ uint8_t smem_raw[];
    uint8_t* base = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
    uint8_t* planes = base;
    uint8_t* stages = planes + G.planes;
    float* ring = reinterpret_cast<float*>(stages + G.stages);
    uint64_t* bars = reinterpret_cast<uint64_t*>(reinterpret_cast<uint8_t*>(ring) + G.ring);
    uint64_t* full = bars;                 // [kStages] a stage's cell rows have landed
    uint64_t* empty = bars + kStages;      // [kStages] their MMAs have read them
    uint64_t* dfull = bars + 2 * kStages;  // [NBUF]    an accumulator holds P of a step's rows
    uint64_t* dempty = dfull + kMaxBufs;   // [NBUF]    the epilogue has read it
    uint64_t* done = dempty + kMaxBufs;    // every MMA issued has completed
    const int nbuf = G.NBUF;
    uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(done + 1);
    __shared__ int aborted;

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    int xt = blockIdx.x, yr = blockIdx.y;
    if constexpr (BATCH) {
        const PlanItem* it = items + find_item<Stage::kScore>(items, n_items, (int)blockIdx.x);
        const int local = (int)blockIdx.x - it->score_c0;
        xt = local % it->score_tx;
        yr = local / it->score_tx;
        cells = static_cast<const uint16_t*>(it->it.cells);
        scores = static_cast<OutT*>(it->it.scores);
        ncx = it->ncx;
        ncy = it->ncy;
        nx = it->nx;
        ny = it->ny;
    }
    const int px0 = xt * kM;
    const int py0 = yr * rows_per_cta;
    const int py1 = min(ny, py0 + rows_per_cta);
    // split: CTA q of the cluster takes filter rows 4q .. 4q + 3, i.e. cell rows py0 + 4 q r ..
    // py1 - 1 + (4 q + 3) r; otherwise cell rows py0 .. py1 - 1 + 15 r (all < ncy)
    const int q = SPLIT ? (int)blockIdx.z : 0;
    const int c0 = py0 + 4 * q * R;
    const int nrows = (py1 - py0) + (SPLIT ? 3 : 15) * R;
    const int step = G.STEP, nsteps = (nrows + step - 1) / step;

    // weights: first the raw values into shared memory (the ring's space, which is cleared
    // afterwards) with all loads in flight at once, then plane i, row n = (f * PARTS + part) *
    // 16 + j holds bins 0..7 of filter f's w[j][i][.], part `part`
    {
        const int raw_bytes = nf * 1024 * (int)sizeof(WT);  // <= the ring's (or partial sums') space
        uint8_t* raw = reinterpret_cast<uint8_t*>(ring);
        if ((reinterpret_cast<uintptr_t>(w) & 15) == 0) {
            for (int e = tid; e < raw_bytes / 16; e += kThreads)
                reinterpret_cast<uint4*>(raw)[e] = __ldg(reinterpret_cast<const uint4*>(w) + e);
        } else {
            for (int e = tid; e < raw_bytes; e += kThreads) raw[e] = __ldg(reinterpret_cast<const uint8_t*>(w) + e);
        }
        __syncthreads();
        // task (f, j, i): the 8 bins of filter f's w[j][i][.] (consecutive in the raw copy: neighbouring
        // tasks read neighbouring 8-value groups), split once into its parts, one plane row per part
        const WT* ws = reinterpret_cast<const WT*>(raw);
        const int nrow = SPLIT ? 4 : 16;  // filter rows this CTA keeps
        for (int e = tid; e < nf * nrow * 8; e += kThreads) {
            const int f = e / (nrow * 8), ji = e - f * nrow * 8, jl = ji >> 3, i = ji & 7;
            const int j = SPLIT ? 4 * q + jl : jl;
            uint4 parts[PARTS];
            weight8_parts<WT, PARTS>(ws + f * 1024 + (j * 8 + i) * 8, parts);
#pragma unroll
            for (int part = 0; part < PARTS; ++part) {
                // row n: split, part * 4 + jj (rows past 4 parts stay zero); else (f * PARTS + part) * 16 + j
                const int n = SPLIT ? part * 4 + jl : (f * PARTS + part) * 16 + j;
                *reinterpret_cast<uint4*>(planes + (size_t)i * G.PLANE_BYTES + (size_t)n * 16) = parts[part];
            }
        }
        if (SPLIT)  // the zero rows past the parts (N = 16)
            for (int e = tid; e < 8 * (16 - 4 * PARTS); e += kThreads) {
                const int i = e / (16 - 4 * PARTS), n = 4 * PARTS + e % (16 - 4 * PARTS);
                *reinterpret_cast<uint4*>(planes + (size_t)i * G.PLANE_BYTES + (size_t)n * 16) = make_uint4(0, 0, 0, 0);
            }
        __syncthreads();
    }
    if (!SPLIT)
        for (int e = tid; e < nf * G.RS * kM; e += kThreads) ring[e] = 0.f;
    if (tid == 0) {
        aborted = 0;
        for (int s = 0; s < kStages; ++s) {
            ptx::mbar_init(&full[s], 1);
            ptx::mbar_init(&empty[s], 1);
        }
        for (int b = 0; b < nbuf; ++b) {
            ptx::mbar_init(&dfull[b], 1);
            ptx::mbar_init(&dempty[b], R > 1 ? kEpiWarps : 4);  // every working epilogue warp, once per step
        }
        ptx::mbar_init(done, 1);
        ptx::fence_mbar_init();
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                         ptx::smem_addr(tmem_slot)),
                     "r"(G.COLS)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    // the planes were written by ordinary stores; the MMAs read them through the async proxy
    ptx::fence_proxy_async_smem();
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *tmem_slot;
    if constexpr (SPLIT) cluster_sync_all();  // every CTA of the cluster runs before any writes to another
    pdl_trigger();  // tail of the path: the successor is small, launch it early
    pdl_wait();     // set-up above read only the weights; the cell rows come from the predecessor

    if (warp == kEpiWarps) {
        if (lane == 0) {
            // producer: cell rows py0 + q into the stage ring
            const int valid = min(kM + 7 * R, ncx - px0);  // > 0: px0 < nx <= ncx
            const uint32_t bytes = (uint32_t)valid * 16;
            int armed = 0;
            for (int k = 0; k < nsteps; ++k) {
                const int s = k % kStages, rows = min(step, nrows - k * step);
                if (!ptx::mbar_wait_bounded(&empty[s], ((k / kStages) & 1) ^ 1, kWaitLimitNs) ||
                    *reinterpret_cast<volatile int*>(&aborted)) {
                    atomicOr(status, kStatusTimeout);
                    atomicExch(&aborted, 1);
                    break;
                }
                ptx::mbar_arrive_expect_tx(&full[s], bytes * rows);
                for (int t = 0; t < rows; ++t)
                    ptx::bulk_g2s(stages + ((size_t)s * step + t) * G.ROW_BYTES,
                                  cells + ((size_t)(c0 + k * step + t) * ncx + px0) * 8, bytes, &full[s]);
                armed = k + 1;
            }
            if (*reinterpret_cast<volatile int*>(&aborted)) {
                // let the copies already issued land before the CTA can exit (bounded)
                for (int k = armed > kStages ? armed - kStages : 0; k < armed; ++k)
                    ptx::mbar_wait_bounded(&full[k % kStages], (k / kStages) & 1, kWaitLimitNs);
            }
        }
    } else if (warp == kEpiWarps + 1) {
        if (lane == 0) {
            // MMA issuer: P of the rows of step k into accumulator k % nbuf (row t at column t N)
            const uint32_t idesc = instr_desc(kM, G.N);
            // descriptors: B of K step ks fixed; A of a row is the stage row's descriptor plus
            // 2 ks r cells (the start-address field counts 16-byte units and never carries: shared
            // addresses are below 2^18)
            uint64_t bdesc[4];
#pragma unroll
            for (int ks = 0; ks < 4; ++ks)
                bdesc[ks] = smem_desc(ptx::smem_addr(planes) + (uint32_t)(2 * ks * G.PLANE_BYTES),
                                      (uint32_t)G.PLANE_BYTES, 128);
            const uint64_t adesc0 = smem_desc(ptx::smem_addr(stages), (uint32_t)(R * 16), 128);
            for (int k = 0; k < nsteps; ++k) {
                const int s = k % kStages, b = k % nbuf, rows = min(step, nrows - k * step);
                if (!ptx::mbar_wait_bounded(&full[s], (k / kStages) & 1, kWaitLimitNs) ||
                    !ptx::mbar_wait_bounded(&dempty[b], ((k / nbuf) & 1) ^ 1, kWaitLimitNs) ||
                    *reinterpret_cast<volatile int*>(&aborted)) {
                    atomicOr(status, kStatusTimeout);
                    atomicExch(&aborted, 1);
                    break;
                }
                tc_fence_after();
                for (int t = 0; t < rows; ++t) {
                    const uint64_t arow = adesc0 + (uint64_t)((((uint32_t)s * step + t) * G.ROW_BYTES) >> 4);
                    const uint32_t d = tmem + (uint32_t)(b * G.BUF + t * G.N);
#pragma unroll
                    for (int ks = 0; ks < 4; ++ks)  // cells 2ks, 2ks + 1
                        mma_bf16(d, arow + (uint64_t)(2 * ks * R), bdesc[ks], idesc, ks > 0 ? 1u : 0u);
                }
                mma_commit(&empty[s]);  // the stage is free once these MMAs have read it
                mma_commit(&dfull[b]);  // the accumulator holds P of the step's rows
            }
            mma_commit(done);
            if (!ptx::mbar_wait_bounded(done, 0, kWaitLimitNs)) atomicOr(status, kStatusTimeout);
        }
    } else {
        // epilogue: lane m = tid % 128 of TMEM, window column px0 + m.  With r > 1 the two groups
        // of four warps take the cell rows of even and of odd index: a row c only touches the ring
        // rows (c - j r) mod 16 r, which keep the parity of c, so the groups share nothing.
        const int m = tid & (kM - 1), grp = R > 1 ? tid / kM : 0;
        const uint32_t lane_base = tmem + ((uint32_t)((warp & 3) * 32) << 16);
        const int px = px0 + m;
        const size_t plane = (size_t)nx * ny;
        const bool works = R > 1 || tid < kM;  // with r = 1 the second group has no rows
        if (SPLIT) {
            if (works)
                epilogue_split<R, PARTS>(lane_base, nsteps, nrows, c0, py0, py1, q, nbuf, G.BUF, grp, m,
                                         ptx::smem_addr(ring), dfull, dempty, &aborted, status);
        } else if (works && nf == 1 && step == 4)
            epilogue_one_filter<R, PARTS, OutT>(lane_base, nsteps, nrows, py0, nbuf, G.BUF, grp, px, nx,
                                                fbias.b[0], scores, dfull, dempty, &aborted, status);
        else if (works)
        for (int k = 0; k < nsteps; ++k) {
            const int b = k % nbuf, rows = min(step, nrows - k * step);
            if (!ptx::mbar_wait_bounded(&dfull[b], (k / nbuf) & 1, kWaitLimitNs) ||
                *reinterpret_cast<volatile int*>(&aborted)) {
                atomicOr(status, kStatusTimeout);
                atomicExch(&aborted, 1);
                break;
            }
            tc_fence_after();
            for (int t = 0; t < rows; ++t) {
                const int c = py0 + k * step + t;  // cell row
                const int py = c - 15 * R;         // the window that has all of its rows after this one
                if (R > 1 && (c & 1) != grp) continue;  // the other group's row
                for (int f = 0; f < nf; ++f) {
                    uint32_t v[PARTS][16];
#pragma unroll
                    for (int p = 0; p < PARTS; ++p)
                        tmem_load16_async(lane_base + (uint32_t)(b * G.BUF + t * G.N + (f * PARTS + p) * 16),
                                          v[p]);
                    tmem_wait_ld();
                    float* col = ring + (size_t)f * G.RS * kM + m;
                    // the 16 running sums this row adds to: distinct slots (16 r <= RS), so every load
                    // goes out before any store
                    float run[16];
#pragma unroll
                    for (int j = 0; j < 16; ++j) run[j] = col[((c - j * R) & (G.RS - 1)) * kM];
#pragma unroll
                    for (int j = 0; j < 16; ++j) {
                        float pj;
                        if constexpr (PARTS == 3) {
                            pj = (__uint_as_float(v[2][j]) + __uint_as_float(v[1][j])) + __uint_as_float(v[0][j]);
                        } else {
                            pj = __uint_as_float(v[0][j]);
                        }
                        col[((c - j * R) & (G.RS - 1)) * kM] = run[j] + pj;
                    }
                    float* slot = col + (py & (G.RS - 1)) * kM;
                    const float sum = *slot;
                    *slot = 0.f;
                    if (py >= py0 && px < nx) {
                        const float sc = sum + fbias.b[f];
                        if constexpr (std::is_same<OutT, int32_t>::value) {
                            scores[f * plane + (size_t)py * nx + px] = __float2int_rn(sc);  // exact integer
                        } else {
                            scores[f * plane + (size_t)py * nx + px] = sc;
                        }
                    }
                }
            }
            // this warp's reads of the accumulator are done: the MMAs of step k + nbuf may overwrite it
            tc_fence_before();
            __syncwarp();
            if (lane == 0) ptx::mbar_arrive(&dempty[b]);
        }
    }
    __syncwarp();
    tc_fence_before();
    __syncthreads();
    if (warp == 0) {
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(G.COLS) : "memory");
    }
    if constexpr (SPLIT) {
        // every CTA's partial sums are in the first CTA's shared memory; it adds the four in order
        cluster_sync_all();
        if (q == 0 && !*reinterpret_cast<volatile int*>(&aborted)) {
            const float* part = ring;
            for (int e = tid; e < (py1 - py0) * kM; e += kThreads) {
                const int row = e / kM, mm = e - row * kM;
                const int px = px0 + mm;
                if (px >= nx) continue;
                float sum = part[(0 * kSplitRows + row) * kM + mm];
#pragma unroll
                for (int qq = 1; qq < kSplit; ++qq) sum += part[(qq * kSplitRows + row) * kM + mm];
                const float sc = sum + fbias.b[0];
                if constexpr (std::is_same<OutT, int32_t>::value) {
                    scores[(size_t)(py0 + row) * nx + px] = __float2int_rn(sc);  // exact integer
                } else {
                    scores[(size_t)(py0 + row) * nx + px] = sc;
                }
            }
        }
    }
}

// Output rows per CTA: the tuned value, else the fewest that keep the grid to
// one CTA per SM (a CTA streams 15 r rows beyond its own, so fewer, longer
// CTAs do less redundant work once every SM has one).
int rows_per_cta(int nx, int ny) {
    const int tuned = tune_get(HOG_TUNE_SCORE_TC_ROWS);
    if (tuned > 0) return tuned;
    const long strips = (nx + kM - 1) / kM;
    const long per = (ny * strips + sm_count() - 1) / sm_count();
    return (int)(per < 1 ? 1 : per);
}

constexpr size_t kMaxSmem = 226 * 1024;  // dynamic shared memory per CTA, below the 227 KiB opt-in limit

// Filters per launch: as many as N <= 256 and the shared memory allow.
int filters_per_launch(int r, int parts, int n_filters) {
    int g = n_filters < kMaxFilters ? n_filters : kMaxFilters;
    while (g > 1 && (16 * parts * g > 256 || RowsGeom(r, parts, g).smem_bytes() > kMaxSmem)) --g;
    return g;
}

// nf filters (w: nf consecutive filters of 1024 weights; scores: nf planes of nx * ny).
template <int R, typename WT, typename OutT>
hog_status launch_t(const uint16_t* cells, int ncx, int ncy, const WT* w, int nf, const RowsBias& bias,
                    OutT* scores, cudaStream_t st) {
    const int nx = ncx - 7 * R, ny = ncy - 15 * R;
    if (nx <= 0 || ny <= 0) return HOG_OK;
    unsigned int* status = nullptr;
    hog_status s = device_status_word(&status);
    if (s != HOG_OK) return s;
    const size_t smem = RowsGeom(R, weight_parts<WT>(), nf).smem_bytes();
    if (smem > kMaxSmem) return HOG_ERR_UNSUPPORTED;
    auto kern = score_rows_kernel<R, WT, OutT, false, false>;
    const cudaError_t e = smem_at_least<score_rows_kernel<R, WT, OutT, false, false>>(smem);
    if (e != cudaSuccess) return cuda_fail(e);
    const int rpc = rows_per_cta(nx, ny);
    const dim3 grid((nx + kM - 1) / kM, (ny + rpc - 1) / rpc);
    return launch_pdl(kern, grid, dim3(kThreads), smem, st, cells, ncx, ncy, w, nf, bias, nx, ny, rpc, scores,
                      static_cast<const PlanItem*>(nullptr), 0, status);
}

// One filter split over clusters of kSplit CTAs (4 filter rows each).
template <int R, typename WT, typename OutT>
hog_status launch_split_t(const uint16_t* cells, int ncx, int ncy, const WT* w, float bias, OutT* scores, int rpc,
                          cudaStream_t st) {
    const int nx = ncx - 7 * R, ny = ncy - 15 * R;
    unsigned int* status = nullptr;
    hog_status s = device_status_word(&status);
    if (s != HOG_OK) return s;
    // at least 80 KiB of shared memory, so that at most two of these CTAs share an SM: their TMEM
    // (256 columns each) then always fits, and no CTA waits in tcgen05.alloc while a CTA of its
    // cluster waits for it at the cluster barrier
    const size_t need = RowsGeom(R, weight_parts<WT>(), 1, true).smem_bytes();
    const size_t smem = need > 80 * 1024 ? need : 80 * 1024;
    static_assert(kSplit * kSplitRows * kM * 4 + 8 * 16 * 16 + kStages * 4 * (kM + 28) * 16 + 2048 < 113 * 1024,
                  "two split CTAs fit one SM");
    auto kern = score_rows_kernel<R, WT, OutT, false, true>;
    cudaError_t e = smem_at_least<score_rows_kernel<R, WT, OutT, false, true>>(smem);
    if (e != cudaSuccess) return cuda_fail(e);
    RowsBias rb{};
    rb.b[0] = bias;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((nx + kM - 1) / kM, (ny + rpc - 1) / rpc, kSplit);
    cfg.blockDim = dim3(kThreads);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    cudaLaunchAttribute attr[2];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    attr[1].id = cudaLaunchAttributeClusterDimension;
    attr[1].val.clusterDim.x = 1;
    attr[1].val.clusterDim.y = 1;
    attr[1].val.clusterDim.z = kSplit;
    cfg.attrs = attr;
    cfg.numAttrs = 2;
    e = cudaLaunchKernelEx(&cfg, kern, cells, ncx, ncy, w, 1, rb, nx, ny, rpc, scores,
                           static_cast<const PlanItem*>(nullptr), 0, status);
    return e == cudaSuccess ? HOG_OK : cuda_fail(e);
}

// Any number of filters: groups of filters_per_launch() per launch.
template <int R, typename WT, typename OutT>
hog_status launch_multi_t(const uint16_t* cells, int ncx, int ncy, const void* w, int n_filters,
                          const float* biases, void* scores, cudaStream_t st) {
    const int nx = ncx - 7 * R, ny = ncy - 15 * R;
    if (nx <= 0 || ny <= 0) return HOG_OK;
    const int path = tune_get(HOG_TUNE_SCORE_PATH);
    const long strips = (nx + kM - 1) / kM;
    if (path == 3 || (path != 2 && (long)ny * strips <= 8L * sm_count())) {
        // small maps: split each filter's 16 rows over clusters of 4 CTAs, so a CTA streams its output
        // rows plus 3 r rows instead of 15 r; one filter per launch, so that a filter's scores are the
        // same whether it is scored alone or with others
        const int tuned = tune_get(HOG_TUNE_SCORE_TC_ROWS);
        int rpc = tuned > 0 ? tuned : (int)(((long)ny * strips * kSplit + sm_count() - 1) / sm_count());
        rpc = rpc < 1 ? 1 : (rpc > kSplitRows ? kSplitRows : rpc);
        for (int f = 0; f < n_filters; ++f) {
            const float b = std::is_same<OutT, int32_t>::value ? (float)std::llround((double)biases[f]) : biases[f];
            const hog_status s = launch_split_t<R, WT, OutT>(
                cells, ncx, ncy, static_cast<const WT*>(w) + (size_t)f * 1024, b,
                static_cast<OutT*>(scores) + (size_t)f * nx * ny, rpc, st);
            if (s != HOG_OK) return s;
        }
        return HOG_OK;
    }
    const int group = filters_per_launch(R, weight_parts<WT>(), n_filters);
    for (int f0 = 0; f0 < n_filters; f0 += group) {
        const int g = n_filters - f0 < group ? n_filters - f0 : group;
        RowsBias rb{};
        for (int k = 0; k < g; ++k) {
            const float b = biases[f0 + k];
            rb.b[k] = std::is_same<OutT, int32_t>::value ? (float)std::llround((double)b) : b;
        }
        const hog_status s = launch_t<R, WT, OutT>(cells, ncx, ncy, static_cast<const WT*>(w) + (size_t)f0 * 1024,
                                                   g, rb, static_cast<OutT*>(scores) + (size_t)f0 * nx * ny, st);
        if (s != HOG_OK) return s;
    }
    return HOG_OK;
}

template <int R, typename WT, typename OutT>
hog_status launch_batch_t(const PlanHeader& h, const void* plan_dev, const void* w, float bias, cudaStream_t st) {
    unsigned int* status = nullptr;
    hog_status s = device_status_word(&status);
    if (s != HOG_OK) return s;
    const size_t smem = RowsGeom(R, weight_parts<WT>(), 1).smem_bytes();
    auto kern = score_rows_kernel<R, WT, OutT, true, false>;
    const cudaError_t e = smem_at_least<score_rows_kernel<R, WT, OutT, true, false>>(smem);
    if (e != cudaSuccess) return cuda_fail(e);
    RowsBias rb{};
    rb.b[0] = bias;
    return launch_pdl(kern, dim3(h.score_ctas), dim3(kThreads), smem, st, static_cast<const uint16_t*>(nullptr), 0,
                      0, static_cast<const WT*>(w), 1, rb, 0, 0, h.score_tc, static_cast<OutT*>(nullptr),
                      plan_items(plan_dev), h.n_items, status);
}

template <int R>
hog_status by_w(const uint16_t* cells, int ncx, int ncy, const void* w, int w_dtype, int n_filters,
                const float* biases, void* scores, cudaStream_t st) {
    if (w_dtype == HOG_F32)
        return launch_multi_t<R, float, float>(cells, ncx, ncy, w, n_filters, biases, scores, st);
    if (w_dtype == HOG_BF16)
        return launch_multi_t<R, uint16_t, float>(cells, ncx, ncy, w, n_filters, biases, scores, st);
    if (w_dtype == HOG_I8)
        return launch_multi_t<R, int8_t, int32_t>(cells, ncx, ncy, w, n_filters, biases, scores, st);
    return HOG_ERR_UNSUPPORTED;
}

template <int R>
hog_status batch_by_w(const PlanHeader& h, const void* plan_dev, const void* w, int w_dtype, float bias,
                      cudaStream_t st) {
    if (w_dtype == HOG_F32) return launch_batch_t<R, float, float>(h, plan_dev, w, bias, st);
    if (w_dtype == HOG_BF16) return launch_batch_t<R, uint16_t, float>(h, plan_dev, w, bias, st);
    if (w_dtype == HOG_I8) return launch_batch_t<R, int8_t, int32_t>(h, plan_dev, w, bias, st);
    return HOG_ERR_UNSUPPORTED;
}

}  // namespace

bool score_rows_supported(const void* cells, int cell_dtype, int n_bins, int cells_x, int cells_y, int r) {
    return cell_dtype == HOG_BF16 && n_bins == 8 && cells_x == 8 && cells_y == 16 &&
           reinterpret_cast<uintptr_t>(cells) % 16 == 0 && (r == 1 || r == 2 || r == 4);
}

int score_rows_batch_rows(long strip_rows) {
    const int tuned = tune_get(HOG_TUNE_SCORE_TC_ROWS);
    if (tuned > 0) return tuned;
    const long per = (strip_rows + 2L * sm_count() - 1) / (2L * sm_count());  // about two CTAs per SM
    return (int)(per < 16 ? 16 : per);
}

hog_status launch_score_rows_batch(const PlanHeader& h, const void* plan_dev, const void* w, int w_dtype, float bias,
                                   cudaStream_t st) {
    if (h.score_ctas == 0) return HOG_OK;
    switch (h.r) {
        case 1: return batch_by_w<1>(h, plan_dev, w, w_dtype, bias, st);
        case 2: return batch_by_w<2>(h, plan_dev, w, w_dtype, bias, st);
        case 4: return batch_by_w<4>(h, plan_dev, w, w_dtype, bias, st);
        default: return HOG_ERR_UNSUPPORTED;
    }
}

hog_status launch_score_rows(const uint16_t* cells_bf16, int ncx, int ncy, int r, const void* w, int w_dtype,
                             int n_filters, const float* biases, void* scores, cudaStream_t st) {
    switch (r) {
        case 1: return by_w<1>(cells_bf16, ncx, ncy, w, w_dtype, n_filters, biases, scores, st);
        case 2: return by_w<2>(cells_bf16, ncx, ncy, w, w_dtype, n_filters, biases, scores, st);
        case 4: return by_w<4>(cells_bf16, ncx, ncy, w, w_dtype, n_filters, biases, scores, st);
        default: return HOG_ERR_UNSUPPORTED;
    }
}

}  // namespace fasthog
