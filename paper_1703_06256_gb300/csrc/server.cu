// server.cu -- hog_server (include/fasthog_server.h): continuous batching of
// detection requests over the per-image calls of fasthog.h.  Host code only;
// every step of a request runs in the library's kernels through the public
// entry points.
//
// A request's life: submit takes a free slot (stream, event, host detection
// buffer) and a first-fit block of the device arena, then enqueues on the
// slot's stream the host-to-device copy of the image, the cell-map call(s),
// the window score and the detection list, which hog_detect writes straight
// into the slot's page-locked host buffer (mapped into the device's address
// space), and records the slot's event.  poll queries the events of the
// requests on the GPU; a finished request gives its arena block back at once
// and hands its host buffer to the caller until release.
#include <atomic>
#include <chrono>
#include <cmath>
#include <deque>
#include <iterator>
#include <map>
#include <mutex>
#include <new>
#include <thread>
#include <vector>

#include "../../include/fasthog_server.h"
#include "internal.cuh"

namespace {

using fasthog::cuda_fail;

constexpr size_t kAlign = 256;
constexpr int kMaxSlots = 64;
constexpr int kCountStride = 16;  // int32 counters 64 bytes apart, one per slot

size_t align_up(size_t x) { return (x + kAlign - 1) / kAlign * kAlign; }
int n_pos(int extent, int box, int stride) { return extent < box ? 0 : (extent - box) / stride + 1; }
bool size_ok(int W, int H) { return W >= 1 && H >= 1 && W <= 65535 && H <= 65535 && (long)W * H < (1L << 31); }

// First-fit sub-allocator over one device allocation.  Free extents are kept
// by offset and merged with their neighbours when a block comes back.
class Arena {
  public:
    void reset(size_t size) {
        free_.clear();
        if (size) free_[0] = size;
        used_ = 0;
    }
    bool take(size_t n, size_t* off) {
        for (auto it = free_.begin(); it != free_.end(); ++it) {
            if (it->second < n) continue;
            *off = it->first;
            const size_t rest = it->second - n, start = it->first + n;
            free_.erase(it);
            if (rest) free_[start] = rest;
            used_ += n;
            return true;
        }
        return false;
    }
    void give(size_t off, size_t n) {
        used_ -= n;
        auto next = free_.lower_bound(off);
        if (next != free_.end() && off + n == next->first) {
            n += next->second;
            next = free_.erase(next);
        }
        if (next != free_.begin()) {
            auto prev = std::prev(next);
            if (prev->first + prev->second == off) {
                prev->second += n;
                return;
            }
        }
        free_[off] = n;
    }
    size_t used() const { return used_; }

  private:
    std::map<size_t, size_t> free_;
    size_t used_ = 0;
};

// Switches to the server's device for the duration of a call.
class DeviceGuard {
  public:
    explicit DeviceGuard(int dev) : dev_(dev) {
        err_ = cudaGetDevice(&prev_);
        if (err_ == cudaSuccess && prev_ != dev_) err_ = cudaSetDevice(dev_);
    }
    ~DeviceGuard() {
        if (err_ == cudaSuccess && prev_ != dev_) cudaSetDevice(prev_);
    }
    cudaError_t error() const { return err_; }

  private:
    int dev_, prev_ = -1;
    cudaError_t err_;
};

// Byte offsets of one request's buffers inside its arena block.
struct Layout {
    int ncx, ncy, nx, ny;
    size_t img, cells, scores, bins, ii, ws_ii, ws_ii_bytes, total;
};

enum class SlotState { kFree, kBusy, kHeld };

constexpr int64_t kPauseNs = 1000000;  // a dispatcher turn longer than 1 ms is recorded as a pause
constexpr size_t kMaxPauses = 4096;     // pauses kept (the most recent)

int64_t clock_ns() {
    return std::chrono::duration_cast<std::chrono::nanoseconds>(std::chrono::steady_clock::now().time_since_epoch())
        .count();
}

// A request waiting for the dispatcher thread.
struct Pending {
    int32_t rid;
    const uint8_t* img;
    int W, H, channels;
    int64_t t_enqueue;
};

struct Slot {
    int64_t t_enqueue = 0, t_admit = 0;  // the dispatcher's stamps of the request on the slot
    cudaStream_t stream = nullptr;
    cudaEvent_t done = nullptr;
    hog_det* dets_host = nullptr;  // page-locked, mapped
    hog_det* dets_dev = nullptr;   // the same memory, as the device addresses it
    void* ws_det = nullptr;        // the slot's detection workspace (largest request), zero-filled once
    SlotState state = SlotState::kFree;
    size_t off = 0, bytes = 0;
    int32_t rid = 0;
    int W = 0, H = 0;
};

}  // namespace

struct hog_server {
    hog_server_config cfg;
    int device = 0;
    int cell_dtype = HOG_F32, score_dtype = HOG_F32;
    bool fused = false;
    size_t max_windows = 0;
    size_t ws_det_bytes = 0;  // each slot's detection workspace
    uint8_t* arena_base = nullptr;
    uint8_t* lut = nullptr;
    void* w = nullptr;
    int32_t* counts_host = nullptr;  // page-locked, mapped; slot i at [i * kCountStride]
    int32_t* counts_dev = nullptr;
    Arena arena;
    std::vector<Slot> slots;
    std::vector<int> free_slots;  // stack of free slot indices
    std::vector<int> busy;        // slots on the GPU, in submission order

    // dispatcher thread (hog_server_start): the queue, finished results and
    // slots to free are shared with the callers' threads under `mu`; every
    // other member belongs to the dispatcher while it runs
    std::thread worker;
    std::atomic<bool> running{false}, stopping{false};
    std::mutex mu;
    std::deque<Pending> queue;
    std::deque<hog_server_timed_result> finished;
    std::vector<int> to_release;
    // stretches of more than kPauseNs between two turns of the dispatcher's loop
    // (since hog_server_start), oldest first, the most recent kMaxPauses kept
    std::deque<std::pair<int64_t, int64_t>> pauses;
    long n_pauses = 0;

    Layout plan(int W, int H, int channels) const {
        Layout L{};
        const hog_server_config& c = cfg;
        L.ncx = n_pos(W, c.cell, c.stride);
        L.ncy = n_pos(H, c.cell, c.stride);
        const int r = c.cell / c.stride;
        L.nx = L.ncx - (c.cells_x - 1) * r > 0 ? L.ncx - (c.cells_x - 1) * r : 0;
        L.ny = L.ncy - (c.cells_y - 1) * r > 0 ? L.ncy - (c.cells_y - 1) * r : 0;
        const size_t cell_bytes = cell_dtype == HOG_BF16 ? 2 : 4;
        const size_t windows = (size_t)L.nx * L.ny;
        size_t o = 0;
        L.img = o;
        o += align_up((size_t)W * H * channels);
        L.cells = o;
        o += align_up((size_t)L.ncx * L.ncy * c.n_bins * cell_bytes + 1);
        L.scores = o;
        o += align_up(windows * 4 + 1);
        L.bins = L.ii = L.ws_ii = L.ws_ii_bytes = 0;
        if (!fused) {
            L.bins = o;
            o += align_up((size_t)W * H);
            L.ii = o;
            o += align_up((size_t)c.n_bins * W * H * (c.ii_dtype == HOG_U16 ? 2 : 4));
            L.ws_ii = o;
            L.ws_ii_bytes = hog_integral_workspace_bytes(W, H, c.n_bins);
            o += align_up(L.ws_ii_bytes);
        }
        L.total = o;
        return L;
    }

    // Enqueue one request's work on its slot's stream.
    hog_status enqueue(const Slot& sl, const Layout& L, const uint8_t* img, int W, int H, int channels,
                       int32_t* count_dev) {
        const hog_server_config& c = cfg;
        uint8_t* base = arena_base + sl.off;
        hog_stream_t st = reinterpret_cast<hog_stream_t>(sl.stream);
        const int windows = L.nx * L.ny;
        if (!fused && fasthog::integral_uses_sync(W, H, c.n_bins, c.ii_dtype)) {
            // The single pass reads a tag and flags from its workspace, which here is reused arena
            // memory: zero-fill that region first (ahead of the kernels, so the kernels still follow
            // one another directly).  The slot's detection workspace was zero-filled once, and every
            // call leaves it ready for the next, whatever the size.
            const cudaError_t e = cudaMemsetAsync(base + L.ws_ii, 0, fasthog::integral_sync_bytes(W, H), sl.stream);
            if (e != cudaSuccess) return cuda_fail(e);
        }
        if (windows > 0) {
            // the image the first kernel reads: in place where it is page-locked and mapped, else a copy
            const uint8_t* src = nullptr;
            if (c.image_in_place) {
                cudaPointerAttributes a{};
                if (cudaPointerGetAttributes(&a, img) == cudaSuccess && a.type == cudaMemoryTypeHost &&
                    a.devicePointer != nullptr)
                    src = static_cast<const uint8_t*>(a.devicePointer);
                cudaGetLastError();  // an unknown pointer leaves no error behind
            }
            if (src == nullptr) {
                const cudaError_t e = cudaMemcpyAsync(base + L.img, img, (size_t)W * H * channels,
                                                      cudaMemcpyHostToDevice, sl.stream);
                if (e != cudaSuccess) return cuda_fail(e);
                src = base + L.img;
            }
            hog_status s;
            if (fused) {
                s = hog_cell_hist_fused(src, W, H, channels, (size_t)W * channels, lut, c.n_bins, c.cell,
                                        c.stride, cell_dtype, base + L.cells, st);
            } else {
                s = hog_bin_map(src, W, H, channels, (size_t)W * channels, lut, c.n_bins, base + L.bins, st);
                if (s == HOG_OK)
                    s = hog_integral(base + L.bins, W, H, c.n_bins, c.ii_dtype, base + L.ii, base + L.ws_ii,
                                     L.ws_ii_bytes, st);
                if (s == HOG_OK)
                    s = hog_cell_hist(base + L.ii, W, H, c.n_bins, c.ii_dtype, c.cell, c.stride, cell_dtype,
                                      base + L.cells, st);
            }
            if (s != HOG_OK) return s;
            s = hog_window_score(base + L.cells, cell_dtype, L.ncx, L.ncy, c.n_bins, c.cells_x, c.cells_y, c.cell,
                                 c.stride, w, c.w_dtype, c.bias, base + L.scores, st);
            if (s != HOG_OK) return s;
        }
        // With no window position the list call still runs: it writes the count 0.
        return hog_detect(base + L.scores, score_dtype, L.nx, L.ny, c.stride, c.thr, sl.rid, 0, sl.dets_dev,
                          windows, count_dev, sl.ws_det, ws_det_bytes, st);
    }

    // Admit one request if a slot is free and its buffers fit (*admitted).
    hog_status submit_one(int32_t rid, const uint8_t* img, int W, int H, int channels, int* admitted) {
        *admitted = 0;
        if (!size_ok(W, H) || (channels != 1 && channels != 3)) return HOG_ERR_ARG;
        if (W > cfg.max_W || H > cfg.max_H) return HOG_ERR_ARG;
        const Layout L = plan(W, H, channels);
        if (L.total > cfg.budget_bytes) return HOG_ERR_ARG;
        if (free_slots.empty()) return HOG_OK;
        size_t off = 0;
        if (!arena.take(L.total, &off)) return HOG_OK;
        DeviceGuard g(device);
        if (g.error() != cudaSuccess) {
            arena.give(off, L.total);
            return cuda_fail(g.error());
        }
        const int i = free_slots.back();
        Slot& sl = slots[i];
        sl.off = off;
        sl.bytes = L.total;
        sl.rid = rid;
        sl.W = W;
        sl.H = H;
        counts_host[i * kCountStride] = -1;
        hog_status st = enqueue(sl, L, img, W, H, channels, counts_dev + i * kCountStride);
        if (st == HOG_OK) {
            const cudaError_t e = cudaEventRecord(sl.done, sl.stream);
            if (e != cudaSuccess) st = cuda_fail(e);
        }
        if (st != HOG_OK) {
            // Part of the work may be enqueued: let it finish before the block is reused.
            cudaStreamSynchronize(sl.stream);
            arena.give(off, L.total);
            return st;
        }
        free_slots.pop_back();
        sl.state = SlotState::kBusy;
        busy.push_back(i);
        *admitted = 1;
        return HOG_OK;
    }

    // Collect up to max_out finished requests (their arena blocks are free at once).
    hog_status poll_some(hog_server_result* out, int max_out, int* n_out, int64_t* t_done = nullptr) {
        *n_out = 0;
        DeviceGuard g(device);
        if (g.error() != cudaSuccess) return cuda_fail(g.error());
        int n = 0;
        size_t keep = 0;
        for (size_t k = 0; k < busy.size(); ++k) {
            const int i = busy[k];
            Slot& sl = slots[i];
            cudaError_t e = n < max_out ? cudaEventQuery(sl.done) : cudaErrorNotReady;
            if (e == cudaErrorNotReady) {
                busy[keep++] = i;
                continue;
            }
            std::atomic_thread_fence(std::memory_order_acquire);
            if (t_done) t_done[n] = clock_ns();
            hog_server_result& r = out[n++];
            r.rid = sl.rid;
            r.status = e == cudaSuccess ? HOG_OK : cuda_fail(e);
            r.count = e == cudaSuccess ? *static_cast<volatile int32_t*>(counts_host + i * kCountStride) : 0;
            r.token = i;
            r.W = sl.W;
            r.H = sl.H;
            r.dets = sl.dets_host;
            arena.give(sl.off, sl.bytes);
            sl.state = SlotState::kHeld;
        }
        busy.resize(keep);
        *n_out = n;
        return HOG_OK;
    }

    // The dispatcher thread: free released slots, collect finished requests,
    // admit queued ones in order; yield when nothing moved.
    void dispatch() {
        cudaSetDevice(device);
        std::vector<hog_server_result> got(slots.size());
        std::vector<int64_t> t_done(slots.size());
        int64_t last_turn = clock_ns();
        while (true) {
            {
                // a turn never blocks for long (every CUDA call here is asynchronous or a query):
                // a longer stretch means the thread was not running
                const int64_t now = clock_ns();
                if (now - last_turn > kPauseNs) {
                    std::lock_guard<std::mutex> lock(mu);
                    pauses.emplace_back(last_turn, now);
                    if (pauses.size() > kMaxPauses) pauses.pop_front();
                    ++n_pauses;
                }
                last_turn = now;
            }
            bool moved = false;
            {
                std::lock_guard<std::mutex> lock(mu);
                for (int tok : to_release) {
                    slots[tok].state = SlotState::kFree;
                    free_slots.push_back(tok);
                }
                moved = moved || !to_release.empty();
                to_release.clear();
            }
            int n = 0;
            if (!busy.empty() && poll_some(got.data(), (int)got.size(), &n, t_done.data()) == HOG_OK && n > 0) {
                std::lock_guard<std::mutex> lock(mu);
                for (int k = 0; k < n; ++k) {
                    const Slot& sl = slots[got[k].token];
                    finished.push_back(hog_server_timed_result{got[k], sl.t_enqueue, sl.t_admit, t_done[k]});
                }
                moved = true;
            }
            while (true) {
                Pending p;
                {
                    std::lock_guard<std::mutex> lock(mu);
                    if (queue.empty()) break;
                    p = queue.front();
                }
                int admitted = 0;
                const hog_status st = submit_one(p.rid, p.img, p.W, p.H, p.channels, &admitted);
                if (st == HOG_OK && !admitted) break;  // wait for a slot or for memory: first in, first out
                std::lock_guard<std::mutex> lock(mu);
                queue.pop_front();
                if (st != HOG_OK) {  // failed to enqueue on the GPU: report it as the request's result
                    hog_server_result r{p.rid, st, 0, -1, p.W, p.H, nullptr};
                    finished.push_back(hog_server_timed_result{r, p.t_enqueue, clock_ns(), clock_ns()});
                } else {
                    Slot& sl = slots[busy.back()];
                    sl.t_enqueue = p.t_enqueue;
                    sl.t_admit = clock_ns();
                }
                moved = true;
            }
            if (stopping.load(std::memory_order_acquire) && busy.empty()) {
                std::lock_guard<std::mutex> lock(mu);
                if (queue.empty()) break;
            }
            if (!moved) std::this_thread::yield();
        }
    }

    void stop_worker() {
        if (!running.load()) return;
        stopping.store(true, std::memory_order_release);
        worker.join();
        running.store(false);
        stopping.store(false);
    }

    void release_all() {
        stop_worker();
        for (Slot& sl : slots) {
            if (sl.state == SlotState::kBusy && sl.done) cudaEventSynchronize(sl.done);
            if (sl.done) cudaEventDestroy(sl.done);
            if (sl.stream) cudaStreamDestroy(sl.stream);
            if (sl.dets_host) cudaFreeHost(sl.dets_host);
            if (sl.ws_det) cudaFree(sl.ws_det);
        }
        slots.clear();
        if (counts_host) cudaFreeHost(counts_host);
        if (arena_base) cudaFree(arena_base);
        if (lut) cudaFree(lut);
        if (w) cudaFree(w);
        counts_host = nullptr;
        arena_base = lut = nullptr;
        w = nullptr;
    }
};

namespace {

hog_status check_config(const hog_server_config* c) {
    if (c->n_bins < 1 || c->n_bins > 64) return HOG_ERR_ARG;
    if (c->cell < 1 || c->cell > 64 || c->stride < 1 || c->cell % c->stride != 0) return HOG_ERR_ARG;
    if (c->cells_x < 1 || c->cells_y < 1 || c->cells_x > 64 || c->cells_y > 64) return HOG_ERR_ARG;
    if (c->w_dtype != HOG_F32 && c->w_dtype != HOG_BF16 && c->w_dtype != HOG_I8) return HOG_ERR_ARG;
    if (!std::isfinite(c->bias) || std::isnan(c->thr)) return HOG_ERR_ARG;
    if (c->fused < -1 || c->fused > 1) return HOG_ERR_ARG;
    if (c->image_in_place != 0 && c->image_in_place != 1) return HOG_ERR_ARG;
    if (c->ii_dtype != HOG_I32 && c->ii_dtype != HOG_U16) return HOG_ERR_ARG;
    if (c->n_slots < 1 || c->n_slots > kMaxSlots || c->budget_bytes == 0) return HOG_ERR_ARG;
    if (!size_ok(c->max_W, c->max_H)) return HOG_ERR_ARG;
    if (c->fused == 1 && !fasthog::cells_fused_supported(c->n_bins, c->cell, c->stride)) return HOG_ERR_UNSUPPORTED;
    return HOG_OK;
}

}  // namespace

extern "C" {

hog_status hog_server_create(const hog_server_config* cfg, const void* w, hog_server** out) {
    if (out == nullptr) return HOG_ERR_ARG;
    *out = nullptr;
    if (cfg == nullptr || w == nullptr) return HOG_ERR_ARG;
    hog_status st = check_config(cfg);
    if (st != HOG_OK) return st;
    hog_server* s = new (std::nothrow) hog_server();
    if (s == nullptr) return HOG_ERR_ARG;
    s->cfg = *cfg;
    const hog_server_config& c = s->cfg;
    // Histogram counts of cells up to 16 x 16 are exact in bf16; the tensor-core scores take bf16 cells
    // (with any weight type).
    s->cell_dtype = c.cell <= 16 ? HOG_BF16 : HOG_F32;
    s->score_dtype = c.w_dtype == HOG_I8 ? HOG_I32 : HOG_F32;
    s->fused = c.fused == 1 || (c.fused == -1 && fasthog::cells_fused_supported(c.n_bins, c.cell, c.stride));
    const int r = c.cell / c.stride;
    const long mx = n_pos(c.max_W, c.cell, c.stride) - (long)(c.cells_x - 1) * r;
    const long my = n_pos(c.max_H, c.cell, c.stride) - (long)(c.cells_y - 1) * r;
    s->max_windows = (size_t)(mx > 0 ? mx : 0) * (size_t)(my > 0 ? my : 0);
    s->ws_det_bytes = hog_detect_workspace_bytes(mx > 0 ? (int)mx : 0, my > 0 ? (int)my : 0);

    cudaError_t e = cudaGetDevice(&s->device);
    const size_t w_elems = (size_t)c.cells_x * c.cells_y * c.n_bins;
    const size_t w_bytes = w_elems * (c.w_dtype == HOG_F32 ? 4 : (c.w_dtype == HOG_BF16 ? 2 : 1));
    if (e == cudaSuccess) e = cudaMalloc(reinterpret_cast<void**>(&s->arena_base), c.budget_bytes);
    if (e == cudaSuccess) e = cudaMalloc(reinterpret_cast<void**>(&s->lut), HOG_LUT_BYTES);
    if (e == cudaSuccess) e = cudaMalloc(&s->w, w_bytes);
    if (e == cudaSuccess) e = cudaMemcpy(s->w, w, w_bytes, cudaMemcpyHostToDevice);
    if (e == cudaSuccess)
        e = cudaHostAlloc(reinterpret_cast<void**>(&s->counts_host), sizeof(int32_t) * kCountStride * c.n_slots,
                          cudaHostAllocMapped);
    if (e == cudaSuccess) e = cudaHostGetDevicePointer(reinterpret_cast<void**>(&s->counts_dev), s->counts_host, 0);
    s->slots.resize(c.n_slots);
    for (int i = 0; i < c.n_slots && e == cudaSuccess; ++i) {
        Slot& sl = s->slots[i];
        e = cudaStreamCreateWithFlags(&sl.stream, cudaStreamNonBlocking);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&sl.done, cudaEventDisableTiming);
        const size_t det_bytes = (s->max_windows > 0 ? s->max_windows : 1) * sizeof(hog_det);
        if (e == cudaSuccess) e = cudaHostAlloc(reinterpret_cast<void**>(&sl.dets_host), det_bytes, cudaHostAllocMapped);
        if (e == cudaSuccess) e = cudaHostGetDevicePointer(reinterpret_cast<void**>(&sl.dets_dev), sl.dets_host, 0);
        if (e == cudaSuccess) e = cudaMalloc(&sl.ws_det, s->ws_det_bytes);
        if (e == cudaSuccess) e = cudaMemset(sl.ws_det, 0, s->ws_det_bytes);  // zero once: the tags' start
    }
    if (e != cudaSuccess) {
        st = cuda_fail(e);
        s->release_all();
        delete s;
        return st;
    }
    st = hog_build_lut(c.n_bins, s->lut, reinterpret_cast<hog_stream_t>(s->slots[0].stream));
    if (st == HOG_OK) {
        e = cudaStreamSynchronize(s->slots[0].stream);
        if (e != cudaSuccess) st = cuda_fail(e);
    }
    if (st != HOG_OK) {
        s->release_all();
        delete s;
        return st;
    }
    s->arena.reset(c.budget_bytes);
    for (int i = c.n_slots - 1; i >= 0; --i) s->free_slots.push_back(i);
    s->busy.reserve(c.n_slots);
    *out = s;
    return HOG_OK;
}

hog_status hog_server_destroy(hog_server* s) {
    if (s == nullptr) return HOG_OK;
    DeviceGuard g(s->device);
    s->release_all();
    delete s;
    return g.error() == cudaSuccess ? HOG_OK : cuda_fail(g.error());
}

size_t hog_server_request_bytes(const hog_server* s, int W, int H, int channels) {
    if (s == nullptr || !size_ok(W, H) || (channels != 1 && channels != 3)) return 0;
    return s->plan(W, H, channels).total;
}

hog_status hog_server_submit(hog_server* s, int32_t rid, const uint8_t* img, int W, int H, int channels,
                             int* admitted) {
    if (s == nullptr || img == nullptr || admitted == nullptr) return HOG_ERR_ARG;
    *admitted = 0;
    if (s->running.load()) return HOG_ERR_UNSUPPORTED;  // the dispatcher thread owns admission
    return s->submit_one(rid, img, W, H, channels, admitted);
}

hog_status hog_server_poll(hog_server* s, hog_server_result* out, int max_out, int* n_out) {
    if (s == nullptr || n_out == nullptr || max_out < 0 || (out == nullptr && max_out > 0)) return HOG_ERR_ARG;
    *n_out = 0;
    if (s->running.load()) return HOG_ERR_UNSUPPORTED;
    return s->poll_some(out, max_out, n_out);
}

hog_status hog_server_release(hog_server* s, int32_t token) {
    if (s == nullptr || token < 0 || token >= (int32_t)s->slots.size()) return HOG_ERR_ARG;
    if (s->running.load()) {
        std::lock_guard<std::mutex> lock(s->mu);
        if (s->slots[token].state != SlotState::kHeld) return HOG_ERR_ARG;
        for (int t : s->to_release)
            if (t == token) return HOG_ERR_ARG;
        s->to_release.push_back(token);
        return HOG_OK;
    }
    Slot& sl = s->slots[token];
    if (sl.state != SlotState::kHeld) return HOG_ERR_ARG;
    sl.state = SlotState::kFree;
    s->free_slots.push_back(token);
    return HOG_OK;
}

hog_status hog_server_start(hog_server* s) {
    if (s == nullptr) return HOG_ERR_ARG;
    if (s->running.load()) return HOG_ERR_ARG;
    s->stopping.store(false);
    {
        std::lock_guard<std::mutex> lock(s->mu);
        s->pauses.clear();
        s->n_pauses = 0;
    }
    s->running.store(true);
    try {
        s->worker = std::thread([s] { s->dispatch(); });
    } catch (...) {
        s->running.store(false);
        return HOG_ERR_UNSUPPORTED;
    }
    return HOG_OK;
}

hog_status hog_server_stop(hog_server* s) {
    if (s == nullptr) return HOG_ERR_ARG;
    s->stop_worker();
    return HOG_OK;
}

hog_status hog_server_pauses(hog_server* s, int64_t* start_ns, int64_t* end_ns, int max_n, int* n) {
    if (s == nullptr || n == nullptr || max_n < 0 || (max_n > 0 && (start_ns == nullptr || end_ns == nullptr)))
        return HOG_ERR_ARG;
    std::lock_guard<std::mutex> lock(s->mu);
    const int kept = (int)s->pauses.size();
    const int first = kept > max_n ? kept - max_n : 0;  // the most recent max_n
    for (int i = first; i < kept; ++i) {
        start_ns[i - first] = s->pauses[i].first;
        end_ns[i - first] = s->pauses[i].second;
    }
    *n = (int)(s->n_pauses < 2147483647L ? s->n_pauses : 2147483647L);
    return HOG_OK;
}

hog_status hog_server_enqueue(hog_server* s, int32_t rid, const uint8_t* img, int W, int H, int channels) {
    if (s == nullptr || img == nullptr) return HOG_ERR_ARG;
    if (!size_ok(W, H) || (channels != 1 && channels != 3)) return HOG_ERR_ARG;
    if (W > s->cfg.max_W || H > s->cfg.max_H) return HOG_ERR_ARG;
    if (s->plan(W, H, channels).total > s->cfg.budget_bytes) return HOG_ERR_ARG;
    if (!s->running.load() || s->stopping.load()) return HOG_ERR_UNSUPPORTED;
    std::lock_guard<std::mutex> lock(s->mu);
    s->queue.push_back(Pending{rid, img, W, H, channels, clock_ns()});
    return HOG_OK;
}

hog_status hog_server_collect(hog_server* s, hog_server_timed_result* out, int max_out, int* n_out) {
    if (s == nullptr || n_out == nullptr || max_out < 0 || (out == nullptr && max_out > 0)) return HOG_ERR_ARG;
    std::lock_guard<std::mutex> lock(s->mu);
    int n = 0;
    while (n < max_out && !s->finished.empty()) {
        out[n++] = s->finished.front();
        s->finished.pop_front();
    }
    *n_out = n;
    return HOG_OK;
}

int64_t hog_server_clock_ns(void) { return clock_ns(); }

hog_status hog_server_stats(const hog_server* s, int* in_flight, size_t* bytes_in_use, int* free_slots) {
    if (s == nullptr) return HOG_ERR_ARG;
    if (s->running.load()) return HOG_ERR_UNSUPPORTED;  // the dispatcher thread owns these counts
    if (in_flight) *in_flight = (int)s->busy.size();
    if (bytes_in_use) *bytes_in_use = s->arena.used();
    if (free_slots) *free_slots = (int)s->free_slots.size();
    return HOG_OK;
}

}  // extern "C"
