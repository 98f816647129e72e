"""Benchmark of the fast-HOG detection path (one JSON line on stdout).

Workload: one 800x600 RGB image per GPU per step (seeded smooth noise plus
shapes), N_b = 8, 8x8 cells, 64x128 window, stride 4, float32 weights
N(0, 0.01), threshold 0.5.  A step is the whole path on that image: bin map,
integral images, cell histograms, window scores, detection list.  The
gradient table is built once per N_b before timing, as the paper builds it
once and only reads it afterwards.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

`value` is Mpixel/s over all ranks (device time, inputs resident, L2 flushed
between steps by writing 256 MB); `e2e` is the same metric through the public
Python API from pinned host memory, including the copies.  The reference arm
(--impl reference) times the CPU oracle, the only other implementation of
this method here.
"""

from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

METRIC = "Mpixel/s & windows/s (800×600, 1080p batch), % HBM peak; served p50/p99 latency"
WORKLOAD = "800x600 RGB uint8, N_b=8, 8x8 cells, 64x128 window, stride 4, f32 weights, thr 0.5"
L2_FLUSH_BYTES = 256 << 20
FALLBACK_HBM_GBS = 6800.0
FALLBACK_BF16_TFLOPS = 1900.0


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--cpu-seconds", type=float, default=10.0, help="CPU-baseline sample length")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-extras", action="store_true",
                    help="skip every extra figure (the main line is unchanged)")
    ap.add_argument("--extras",
                    default="ii_other,fused,stages_4k,batch_1080p,batch_pyramid,multi_filter,blocks,soft,serving",
                    help="comma-separated extra figures to run (default: all)")
    ap.add_argument("--image", default="800x600", help="WxH of the RGB image (same recipe as 800x600)")
    ap.add_argument("--serve-requests", type=int, default=10000, help="requests in the served stream (0: skip)")
    ap.add_argument("--no-tune", action="store_true", help="keep the library's default launch shapes")
    ap.add_argument("--ii", choices=["i32", "u16"], default="i32",
                    help="integral images of the main step: int32, or uint16 modulo 2^16 (exact box sums for "
                         "boxes below 65536 pixels; every result of the path is the same)")
    return ap.parse_args()


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return FALLBACK_HBM_GBS, "fallback"


def bf16_peak():
    """Measured dense bf16 peak (TFLOP/s, burst: the score is timed alone), or the fallback."""
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return float(json.load(f)["bf16_tflops"])
    except Exception:
        return FALLBACK_BF16_TFLOPS


def profiled_traffic(stage: str, workload: str):
    """DRAM bytes per launch of `stage` from the committed ncu capture, or None
    when there is none for this workload or the kernel source has changed
    since it was taken (profiles/traffic.txt records a hash of the source)."""
    import hashlib

    path = os.path.join(ROOT, "profiles", "traffic.txt")
    try:
        lines = open(path).read().splitlines()
    except OSError:
        return None
    for ln in lines:
        if ln.startswith("#") or not ln.strip():
            continue
        st, wl_, nbytes, src, sha = ln.split()
        if st == stage and wl_ == workload:
            try:
                cur = hashlib.sha256(open(os.path.join(ROOT, src), "rb").read()).hexdigest()[:16]
            except OSError:
                return None
            return int(nbytes) if cur == sha else None
    return None


def measured_precision():
    """The bf16 score's measured error on the 32 x 1920x1080 precision workload
    (profiles/precision_1080p.txt, written from the precision test's output),
    or None once the score kernel's source has changed since."""
    import hashlib

    path = os.path.join(ROOT, "profiles", "precision_1080p.txt")
    try:
        lines = [ln for ln in open(path).read().splitlines() if ln.strip() and not ln.startswith("#")]
    except OSError:
        return None
    out = {}
    for ln in lines:
        key, val = ln.split(None, 1)
        if key == "source":
            src, sha = val.split()
            cur = hashlib.sha256(open(os.path.join(ROOT, src), "rb").read()).hexdigest()[:16]
            if cur != sha:
                return None
            out["source"] = "profiles/precision_1080p.txt (python -m pytest tests/test_gpu_precision.py -s)"
        elif key == "windows":
            out[key] = int(val)
        elif key.startswith("int8"):
            out[key] = val
        else:
            out[key] = float(val)
    out["workload"] = "32 RGB 1920x1080, N_b=8, stride 4, bf16 cells x bf16 weights (tensor cores), FP32 accumulation"
    out["tolerance"] = "weight rounding <= 2^-8, FP32 accumulation <= 1e-5, of sum_k |w_k| h_k + |bias| per window"
    return out


class ClockSampler:
    """nvidia-smi clocks and throttle reasons, sampled every 200 ms."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.t.join(timeout=2)
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for n, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(n)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "sm_min_mhz": min(sm) if sm else None, "reasons": sorted(reasons), "samples": len(sm)}


def host_cores() -> int:
    try:
        return len(os.sched_getaffinity(0))
    except Exception:
        return os.cpu_count() or 1


def oracle_images(img, c, threads: int, per_thread: int):
    """`threads` host threads each run the C oracle on `per_thread` whole
    images (ctypes releases the GIL for the duration of each C call, so the
    threads run on separate cores); returns the wall time."""
    import concurrent.futures as cf

    import oracle

    def work(_):
        for _ in range(per_thread):
            oracle.pipeline(img, c["n_bins"], c["w"], c["bias"], c["stride"], c["thr"])

    t0 = time.perf_counter()
    if threads == 1:
        work(0)
    else:
        with cf.ThreadPoolExecutor(max_workers=threads) as ex:
            list(ex.map(work, range(threads)))
    return time.perf_counter() - t0


def cpu_baseline(img, c, seconds):
    """The oracle as it stands (plain FP64 C) on whole 800x600 images: one
    host thread, then one thread per host core (images spread over the
    threads).  Each leg runs for about `seconds` / 2."""
    import oracle

    oracle.build()
    px = img.shape[0] * img.shape[1]
    legs = {}
    cores = host_cores()
    for threads in (1, cores):
        oracle_images(img, c, threads, 1)  # warm-up: every thread's first image
        # size the sample from one timed round, then time the sample
        t1 = oracle_images(img, c, threads, 1)
        per = max(1, int(seconds / 2 / max(t1, 1e-3)))
        el = oracle_images(img, c, threads, per)
        n = per * threads
        legs[threads] = {"value": round(px * n / el / 1e6, 3), "unit": "Mpixel/s", "cores": threads,
                         "images": n, "seconds": round(el, 2)}
    top = legs[cores]
    return {"value": top["value"], "unit": "Mpixel/s", "cores": cores, "kind": "oracle",
            "sample": (f"{top['images']} full 800x600 images through the FP64 C oracle (bins, ii, Eq. 6 "
                       f"histograms, scores, list), one image per thread at a time on {cores} host threads, "
                       f"in {top['seconds']} s"),
            "single_thread": dict(legs[1], sample=f"{legs[1]['images']} images on one thread")}


def run_reference(args, rank, world):
    """The reference arm: the CPU oracle, the only other implementation of
    this method, on every host core (one 800x600 image per thread per step)."""
    if rank != 0:
        return
    import workloads as wl

    c = wl.config1()
    img = c["images"][0]
    import oracle

    oracle.build()
    cores = host_cores()
    for _ in range(args.warmup):
        oracle_images(img, c, cores, 1)
    el = sum(oracle_images(img, c, cores, 1) for _ in range(args.steps))
    px = img.shape[0] * img.shape[1] * cores
    value = px * args.steps / el / 1e6
    print(json.dumps({
        "impl": "reference", "metric": METRIC, "value": round(value, 3), "unit": "Mpixel/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(el / args.steps * 1e3, 4),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": WORKLOAD},
        "cpu_baseline": {"value": round(value, 3), "unit": "Mpixel/s", "cores": cores, "kind": "oracle",
                         "sample": f"{args.steps} steps of {cores} full 800x600 images, one per host thread, "
                                   "FP64 C oracle"},
        "e2e": {"value": round(value, 3), "unit": "Mpixel/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }), flush=True)


def algorithmic_bytes(W, H, nb, ncx, ncy, windows, cell_bytes=2, ii_bytes=4):
    """Bytes each stage must move (RGB image, integral images of `ii_bytes`
    per entry, cells of `cell_bytes` per count, f32 scores): the figures the
    rooflines divide by."""
    px = W * H
    return {
        "bin_map": px * (3 + 1),              # RGB in, bins out
        "integral": px * (1 + ii_bytes * nb),  # bins in, planes out
        # Eq. 6 per cell position and bin: one integral-image sample in (each
        # sample of the stride grid is a corner of up to four cells, read once)
        # and one count out
        "cell_hist": ncx * ncy * nb * (ii_bytes + cell_bytes),
        "score": ncx * ncy * nb * cell_bytes + windows * 4,  # cell map in, score out
        "detect": windows * 4,
    }


def graph_step(torch, fns, between: bool):
    """Record the five stages as one CUDA graph with timing events recorded
    inside it: at the two ends only (between=False; the kernels keep their
    programmatic dependent launches across stage boundaries), or also between
    the stages (between=True; each event is a graph node, so the stages
    serialise).  Falls back to one graph per stage with events between the
    replays where events cannot be recorded inside a graph."""
    n = len(fns)
    try:
        evs = [torch.cuda.Event(enable_timing=True, external=True) for _ in range(n + 1 if between else 2)]
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g):
            evs[0].record()
            for i, fn in enumerate(fns):
                fn()
                if between:
                    evs[i + 1].record()
            if not between:
                evs[1].record()

        def step():
            g.replay()
        mode = "one CUDA graph per step, events recorded inside it"
    except TypeError:
        evs = [torch.cuda.Event(enable_timing=True) for _ in range(n + 1 if between else 2)]
        graphs = []
        for fn in fns:
            gi = torch.cuda.CUDAGraph()
            with torch.cuda.graph(gi):
                fn()
            graphs.append(gi)

        def step():
            evs[0].record()
            for i, gi in enumerate(graphs):
                gi.replay()
                if between:
                    evs[i + 1].record()
            if not between:
                evs[1].record()
        mode = "one CUDA graph per stage, events between replays"

    def read_times():
        if between:
            return [evs[i].elapsed_time(evs[i + 1]) for i in range(n)], evs[0].elapsed_time(evs[-1])
        return None, evs[0].elapsed_time(evs[1])

    return step, read_times, mode


def time_steps(torch, step, read, flush, steps, warmup):
    """Mean device time (ms) of `steps` replays, each after an L2 flush."""
    for _ in range(max(warmup, 3)):
        flush.fill_(1)
        step()
    torch.cuda.synchronize()
    total = 0.0
    for k in range(steps):
        flush.fill_(k)
        step()
        torch.cuda.synchronize()
        total += read()[1]
    return total / steps


def batch_1080p(torch, fh, wl, replicas, flush, args, world):
    """The 1080p batch: 32 RGB 1920x1080 images per step (N_b = 8, stride 4),
    bf16 cell maps and bf16 weights, so the score runs on the tensor cores.
    All 32 images' calls are recorded in one CUDA graph."""
    n_img, W, H = 32, 1920, 1080
    rng = wl.rng_for(3)
    w = wl.weights_f32(8, rng)
    pipes = []
    for i in range(n_img):
        p = fh.HogPipeline(W, H, 3, 8, 4, cell_dtype=fh.HOG_BF16, w_dtype=fh.HOG_BF16)
        p.set_weights(w, 0.0, 0.5)
        p.set_image(wl.rgb_smooth_shapes(W, H, rng))
        pipes.append(p)
    from paper_1703_06256_gb300.batch import HogBatch

    out = {}
    for label, fused in (("separate_calls", False), ("fused_cells", True)):
        b = HogBatch(pipes, n_streams=8, fused=fused)
        evs = [torch.cuda.Event(enable_timing=True, external=True) for _ in range(2)]
        b.capture(evs)
        ms = replicas.max_over_ranks(
            time_steps(torch, b.run, lambda: (None, evs[0].elapsed_time(evs[1])), flush, max(args.steps // 10, 5),
                       args.warmup), "cuda")
        windows = n_img * pipes[0].nx * pipes[0].ny
        out[label] = {"value": round(replicas.aggregate_rate(n_img * W * H, ms * 1e-3, world) / 1e6, 1),
                      "unit": "Mpixel/s", "ms_per_step": round(ms, 4),
                      "windows_per_s": round(replicas.aggregate_rate(windows, ms * 1e-3, world), 1)}
    out["workload"] = ("32 RGB 1920x1080 images per step, N_b=8, stride 4, bf16 cells x bf16 weights (tensor cores); "
                       "one CUDA graph, 8 concurrent streams")
    del pipes
    torch.cuda.empty_cache()
    return out


def serving(torch, wl, args):
    """Continuous batching against the plain per-image path.

    Requests: RGB images, width and height uniform over multiples of 8 in
    320..3840 x 240..2160, Poisson arrivals, N_b = 8, stride 4, bf16 weights.
    The images cycle through 128 pinned host images, cropped at random
    offsets from one generated 3840x2160 image at the sizes of the stream's first 128
    requests.  The plain path is the same server with one stream (one request
    on the GPU at a time, FIFO); its capacity is measured by a back-to-back
    run, and the Poisson stream arrives at 0.8 x that capacity for both.
    Latency is arrival to detections on the host."""
    from paper_1703_06256_gb300.serve import HogServer, Request, latency_summary
    import paper_1703_06256_gb300 as fh

    n_req = args.serve_requests
    rng = wl.rng_for(5)
    w = wl.weights_f32(8, rng)
    stream = wl.request_stream(n_req, rate_per_s=1.0)
    base = base_4k(wl)
    pool = []
    for k in range(min(128, n_req)):
        Wk, Hk = stream[k]["W"], stream[k]["H"]
        y, x = int(rng.integers(0, 2160 - Hk + 1)), int(rng.integers(0, 3840 - Wk + 1))
        pool.append(torch.from_numpy(np.ascontiguousarray(base[y:y + Hk, x:x + Wk])).pin_memory())
    kw = dict(n_bins=8, stride=4, thr=0.5, w_dtype=fh.HOG_BF16, budget_bytes=8 << 30, fused=True)
    served = HogServer(w, n_streams=16, **kw)
    plain = HogServer(w, n_streams=1, **kw)

    def run(srv, reqs):
        t0 = time.perf_counter()
        res, replay = srv.serve_native(reqs, keep=False)
        return res, time.perf_counter() - t0, replay

    burst = [Request(i, pool[i % len(pool)], 0.0) for i in range(min(1000, n_req))]
    # clocks over the whole comparison; the sampler (an nvidia-smi process) starts before the warm-up,
    # so that its start-up falls outside the measured streams
    sampler = ClockSampler(torch.cuda.current_device())
    sampler.start()
    for srv in (served, plain):  # warm-up: every kernel loaded, allocator pools filled
        run(srv, burst[: len(pool)])
    torch.cuda.synchronize()
    _, t_plain, _ = run(plain, burst)
    _, t_served, _ = run(served, burst)
    cap_plain, cap_served = len(burst) / t_plain, len(burst) / t_served
    rate = 0.8 * cap_plain
    reqs = [Request(i, pool[i % len(pool)], stream[i]["t"] / rate) for i in range(n_req)]
    out = {"workload": ("Poisson arrivals at 0.8 x the plain path's capacity; RGB images, W, H uniform over multiples "
                        "of 8 in 320..3840 x 240..2160 (128 distinct pinned host images, cycled); N_b=8, stride 4, "
                        "bf16 cells x bf16 weights; 8 GB device budget; admission and completion on the server's "
                        "native dispatcher thread; latency = enqueue to detections in host memory (native clock); "
                        "replay_late = how far behind its arrival time the replaying thread queued a request"),
           "requests": n_req, "rate_per_s": round(rate, 1),
           "mean_mpixel_per_request": round(sum(int(t.numel()) for t in pool) / 3 / len(pool) / 1e6, 3),
           "capacity_images_per_s": {"plain": round(cap_plain, 1), "served": round(cap_served, 1)}}
    for label, srv, streams in (("served", served, 16), ("plain", plain, 1)):
        res, wall, replay = run(srv, reqs)
        pauses = replay.pop("pauses_ns")
        out[label] = dict(latency_summary(res, wall, pauses), streams=streams, fused=srv.fused, **replay)
    out["clocks"] = sampler.stop()
    del served, plain, pool
    torch.cuda.empty_cache()
    return out


def batch_pyramid(torch, fh, wl, replicas, flush, args, world):
    """The mixed-size pyramid batch: 64 RGB images, sizes drawn from
    {640x480, 800x600, 1280x720, 1920x1080}, each with a 3-level 2:1 pyramid
    (192 items), stride 4.  Images are crops, at random offsets, of one
    generated 1920x1080 image (generating 64 images on the host would take
    longer than the whole benchmark).  Mpixel/s counts input pixels (level 0);
    windows/s counts windows over all levels.

      batched_nb8   one launch per stage for the whole batch (pyramids: one
                    per image), bf16 cells x bf16 weights on the tensor cores
      batched_nb16  the same with N_b = 16 (the score runs per item on CUDA cores)
      graph_nb8     per-item calls (fused cells, score, detect), one graph
                    over 8 streams
      unfused_i32 / unfused_u16   per-item five calls with int32 / uint16
                    integral images, one graph over 8 streams"""
    from paper_1703_06256_gb300.batch import HogBatch, HogPlanBatch

    rng = wl.rng_for(2)
    sizes = [wl.BATCH_SIZES[int(i)] for i in rng.integers(0, len(wl.BATCH_SIZES), size=64)]
    base = wl.rgb_smooth_shapes(1920, 1080, rng)
    imgs = []
    for (W, H) in sizes:
        y, x = int(rng.integers(0, 1080 - H + 1)), int(rng.integers(0, 1920 - W + 1))
        imgs.append(np.ascontiguousarray(base[y:y + H, x:x + W]))
    px = sum(W * H for (W, H) in sizes)
    steps = max(args.steps // 10, 5)
    out = {}

    def timed(label, run_fn, evs, windows, extra=None):
        ms = replicas.max_over_ranks(
            time_steps(torch, run_fn, lambda: (None, evs[0].elapsed_time(evs[1])), flush, steps, args.warmup),
            "cuda")
        out[label] = dict({"value": round(replicas.aggregate_rate(px, ms * 1e-3, world) / 1e6, 1),
                           "unit": "Mpixel/s", "ms_per_step": round(ms, 4),
                           "windows_per_s": round(replicas.aggregate_rate(windows, ms * 1e-3, world), 1)},
                          **(extra or {}))

    for nb in (8, 16):
        w = wl.weights_f32(nb, rng)
        b = HogPlanBatch(sizes, channels=3, levels=3, n_bins=nb, stride=4, w_dtype=fh.HOG_BF16)
        b.set_images(imgs)
        b.set_weights(w, 0.0, 0.5)
        evs = [torch.cuda.Event(enable_timing=True, external=True) for _ in range(2)]
        b.capture(evs)
        timed(f"batched_nb{nb}", b.run, evs, b.windows, {"items": len(b.items), "launches": b.launches()})
        windows = b.windows
        del b
    torch.cuda.empty_cache()
    # per-item pipelines over the same items (levels decimated on the host: every 2^l-th row and column)
    w = wl.weights_f32(8, rng)
    for label, fused, ii in (("graph_nb8", True, fh.HOG_I32), ("unfused_i32", False, fh.HOG_I32),
                             ("unfused_u16", False, fh.HOG_U16)):
        pipes = []
        for img in imgs:
            H, W = img.shape[:2]
            for lv in range(3):
                lvl = np.ascontiguousarray(img[:: 1 << lv, :: 1 << lv][: H >> lv, : W >> lv])
                p = fh.HogPipeline(W >> lv, H >> lv, 3, 8, 4, ii_dtype=ii, cell_dtype=fh.HOG_BF16,
                                   w_dtype=fh.HOG_BF16)
                p.set_weights(w, 0.0, 0.5)
                p.set_image(lvl)
                pipes.append(p)
        hb = HogBatch(pipes, n_streams=8, fused=fused)
        evs = [torch.cuda.Event(enable_timing=True, external=True) for _ in range(2)]
        hb.capture(evs)
        timed(label, hb.run, evs, windows)
        del hb, pipes
        torch.cuda.empty_cache()
    out["workload"] = ("64 RGB images, sizes from {640x480, 800x600, 1280x720, 1920x1080} (crops of one generated "
                       "1920x1080 image), 3-level 2:1 pyramid (192 items), stride 4, bf16 cells x bf16 weights, "
                       "thr 0.5; Mpixel/s over level-0 pixels")
    return out


def multi_filter(torch, fh, wl, flush, args, bf16_peak):
    """Several filters on one 1920x1080 RGB image (stride 4, N_b = 8, bf16
    cells x bf16 weights): the score call alone (hog_window_score_multi, one
    tensor-core launch per filter group), cells computed beforehand.  Reports
    the dense-equivalent FLOP rate 2 * 1024 * windows * F / t against the
    measured bf16 peak: the banded implicit GEMM spends N = Tc output rows per
    MMA per filter, so its ceiling is far below dense peak; the figure shows
    how several filters raise it."""
    W, H = 1920, 1080
    rng = wl.rng_for(3)
    img = wl.rgb_smooth_shapes(W, H, rng)
    p = fh.HogPipeline(W, H, 3, 8, 4, cell_dtype=fh.HOG_BF16, w_dtype=fh.HOG_BF16)
    p.set_image(img)
    p.stage_cells_fused()
    torch.cuda.synchronize()
    windows = p.nx * p.ny
    out = {"workload": "1920x1080 RGB, N_b=8, stride 4, bf16 cells x bf16 weights; score call only"}
    steps = max(args.steps // 4, 10)
    for F in (1, 4, 16):
        w = torch.from_numpy(rng.normal(0, 0.01, (F, 1024)).astype(np.float32)).to(torch.bfloat16).cuda()
        scores = torch.empty(F * windows, dtype=torch.float32, device="cuda")
        biases = [0.0] * F
        evs = [torch.cuda.Event(enable_timing=True, external=True) for _ in range(2)]
        call = lambda: fh.hog_window_score_multi(p.cells, fh.HOG_BF16, p.ncx, p.ncy, 8, 8, 16, 8, 4, w,  # noqa: E731
                                                 fh.HOG_BF16, F, biases, scores)
        call()
        torch.cuda.synchronize()
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g):
            evs[0].record()
            call()
            evs[1].record()
        ms = time_steps(torch, g.replay, lambda: (None, evs[0].elapsed_time(evs[1])), flush, steps, args.warmup)
        tflops = 2.0 * 1024 * windows * F / (ms * 1e-3) / 1e12
        out[f"filters_{F}"] = {"ms": round(ms, 5), "filter_windows_per_s": round(windows * F / (ms * 1e-3), 1),
                               "tflops": round(tflops, 2),
                               "frac_of_bf16_peak": round(tflops / bf16_peak, 4) if bf16_peak else None}
    del p
    torch.cuda.empty_cache()
    return out


_BASE_4K = None


def base_4k(wl):
    """One generated 3840x2160 RGB image, shared by the figures that crop from it."""
    global _BASE_4K
    if _BASE_4K is None:
        _BASE_4K = wl.rgb_smooth_shapes(3840, 2160, wl.rng_for(5))
    return _BASE_4K


def stage_rooflines(torch, fh, wl, flush, args, hbm):
    """The five-call step on one 3840x2160 RGB image (the size at which the
    memory-bound stages leave L2): each stage's algorithmic bytes over its
    mean time (events between the stages inside one graph), against the
    measured HBM peak.  N_b = 8, stride 4, int32 integral images and cells."""
    W, H = 3840, 2160
    p = fh.HogPipeline(W, H, 3, 8, 4, cell_dtype=fh.HOG_BF16)
    p.set_weights(wl.weights_f32(8, wl.rng_for(1)), 0.0, 0.5)
    p.set_image(base_4k(wl))
    fns = [p.stage_bin_map, p.stage_integral, p.stage_cell_hist, p.stage_score, p.stage_detect]
    names = ["bin_map", "integral", "cell_hist", "score", "detect"]
    p.run_eager()
    torch.cuda.synchronize()
    step, read, _ = graph_step(torch, fns, between=True)
    steps = max(args.steps // 10, 10)
    for _ in range(max(args.warmup, 3)):
        flush.fill_(1)
        step()
    torch.cuda.synchronize()
    ms = [0.0] * 5
    for k in range(steps):
        flush.fill_(k)
        step()
        torch.cuda.synchronize()
        st, _ = read()
        ms = [a + b for a, b in zip(ms, st)]
    ms = [m / steps for m in ms]
    px, nb = W * H, 8
    windows = p.nx * p.ny
    alg = algorithmic_bytes(W, H, nb, p.ncx, p.ncy, windows)
    out = {"workload": "3840x2160 RGB, N_b=8, stride 4, int32 integral images, bf16 cells (exact counts), "
                       "f32 weights",
           "peak_gbs": hbm}
    for n, t in zip(names, ms):
        gbs = alg[n] / (t * 1e-3) / 1e9
        traffic = profiled_traffic(n, f"{W}x{H}")
        out[n] = {"ms": round(t, 5), "algorithmic_bytes": alg[n], "gbs": round(gbs, 1), "frac": round(gbs / hbm, 4),
                  "dram_bytes": traffic,
                  "dram_over_algorithmic": round(traffic / alg[n], 3) if traffic else None}
    del p
    torch.cuda.empty_cache()
    return out


def soft_variant(torch, fh, wl, flush, args):
    """Two-bin soft votes on the benchmark image (800x600 RGB, N_b = 8,
    stride 4): hog_cell_hist_soft (one kernel from the image) and the window
    score over its f32 cells (f32 weights), as one graph."""
    c = wl.config1()
    img = c["images"][0]
    H, W = img.shape[:2]
    p = fh.HogPipeline(W, H, 3, 8, 4)
    p.set_weights(c["w"], 0.0, c["thr"])
    p.set_image(img)
    lut = torch.empty(fh.HOG_SOFT_LUT_BYTES // 2, dtype=torch.int16, device="cuda")
    fh.hog_build_soft_lut(8, lut)
    calls = [lambda: fh.hog_cell_hist_soft(p.img, W, H, 3, W * 3, lut, 8, 8, 4, fh.HOG_F32, p.cells),
             p.stage_score]
    for fn in calls:
        fn()
    torch.cuda.synchronize()
    step, read, _ = graph_step(torch, calls, between=False)
    ms = time_steps(torch, step, read, flush, max(args.steps // 4, 10), args.warmup)
    return {"workload": "800x600 RGB, N_b=8, stride 4, soft votes (64 units per pixel), f32 weights",
            "ms_per_step": round(ms, 5), "mpixel_per_s": round(W * H / (ms * 1e-3) / 1e6, 1)}


def blocks_variant(torch, fh, wl, flush, args):
    """Overlapping L2-normalised 2x2-cell blocks on the benchmark image
    (800x600 RGB, N_b = 8, stride 4, eps = 1): cells from the five-call path,
    then hog_block_norm and the 7 x 15-block window score (f32 weights, 3360
    per window).  Times the two block calls as one graph."""
    c = wl.config1()
    img = c["images"][0]
    H, W = img.shape[:2]
    p = fh.HogPipeline(W, H, 3, 8, 4)
    p.set_image(img)
    p.run_eager()
    torch.cuda.synchronize()
    r = 2
    nbx, nby = p.ncx - r, p.ncy - r
    k = 32
    blocks = torch.empty(nbx * nby * k, dtype=torch.float32, device="cuda")
    nx, ny = nbx - 6 * r, nby - 14 * r
    w = torch.from_numpy(wl.rng_for(14).normal(0, 0.01, 15 * 7 * k).astype(np.float32)).cuda()
    scores = torch.empty(max(nx * ny, 1), dtype=torch.float32, device="cuda")
    calls = [lambda: fh.hog_block_norm(p.cells, fh.HOG_F32, p.ncx, p.ncy, 8, r, 1.0, blocks),
             lambda: fh.hog_window_score(blocks, fh.HOG_F32, nbx, nby, k, 7, 15, 8, 4, w, fh.HOG_F32, 0.0, scores)]
    for fn in calls:  # load the kernels before the capture
        fn()
    torch.cuda.synchronize()
    step, read, _ = graph_step(torch, calls, between=True)
    steps = max(args.steps // 4, 10)
    ms = [0.0, 0.0]
    for _ in range(max(args.warmup, 3)):
        flush.fill_(1)
        step()
    torch.cuda.synchronize()
    for kk in range(steps):
        flush.fill_(kk)
        step()
        torch.cuda.synchronize()
        st, _ = read()
        ms = [a + b for a, b in zip(ms, st)]
    ms = [m / steps for m in ms]
    return {"workload": "800x600 RGB, N_b=8, stride 4, 2x2-cell blocks at one-cell steps, L2 norm (eps 1), "
                        "7x15-block window, f32 weights",
            "block_norm_ms": round(ms[0], 5), "block_score_ms": round(ms[1], 5), "blocks": nbx * nby,
            "windows": nx * ny, "windows_per_s": round(nx * ny / (sum(ms) * 1e-3), 1)}


def free_port() -> int:
    import socket

    with socket.socket() as sk:
        sk.bind(("127.0.0.1", 0))
        return sk.getsockname()[1]


def launch_ranks(n: int, argv: list[str]) -> int:
    """`--gpus N` outside a torchrun launch: run this same command as N ranks
    of one node (one process per GPU; torch.distributed.run sets RANK,
    LOCAL_RANK, WORLD_SIZE and the rendezvous on 127.0.0.1).  Rank 0 prints
    the JSON line; returns the launcher's exit code."""
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes=1", f"--nproc-per-node={n}",
           "--master-addr=127.0.0.1", f"--master-port={free_port()}", os.path.abspath(__file__), *argv]
    return subprocess.run(cmd).returncode


def timed_region(run_step, read_ms, steps: int, barrier, sync) -> float:
    """The timed region of every rank: a barrier and a device synchronise on
    both sides, `steps` steps (each read back by `read_ms` after its own
    synchronise), then the mean ms per step of this rank."""
    if barrier is not None:
        barrier()
    sync()
    total = 0.0
    for k in range(steps):
        run_step(k)
        sync()
        total += read_ms()
    sync()
    if barrier is not None:
        barrier()
    return total / steps


def main():
    args = parse()
    extras = set() if args.no_extras else {e.strip() for e in args.extras.split(",") if e.strip()}
    rank, world, local = dist_env()
    if args.gpus > 1 and "WORLD_SIZE" not in os.environ:
        return launch_ranks(args.gpus, sys.argv[1:])
    if args.impl == "reference":
        return run_reference(args, rank, world)

    import torch

    import paper_1703_06256_gb300 as fh
    import workloads as wl
    from paper_1703_06256_gb300 import replicas

    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist

        dist.init_process_group("nccl")
    c = wl.config1(seed=wl.BASE_SEED + 1 + rank)
    iw, ih = (int(v) for v in args.image.lower().split("x"))
    if (iw, ih) != (800, 600):
        c["images"] = [wl.rgb_smooth_shapes(iw, ih, wl.rng_for(1, wl.BASE_SEED + 1 + rank))]
    img = c["images"][0]
    H, W = img.shape[:2]
    # bf16 cells: counts <= 64 are exact in bf16, and the score's tensor-core kernel reads them as they lie
    ii_u16 = args.ii == "u16"
    pipe = fh.HogPipeline(W, H, 3, c["n_bins"], c["stride"], cell_dtype=fh.HOG_BF16,
                          ii_dtype=fh.HOG_U16 if ii_u16 else fh.HOG_I32)
    pipe.set_weights(c["w"], c["bias"], c["thr"])
    pipe.set_image(img)
    pipe.img_host.copy_(torch.from_numpy(img.reshape(-1)))
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.int32, device="cuda")
    names = ["bin_map", "integral", "cell_hist", "score", "detect"]
    fns = [pipe.stage_bin_map, pipe.stage_integral, pipe.stage_cell_hist, pipe.stage_score, pipe.stage_detect]

    # eager warm-up loads every kernel; then the step is recorded as CUDA graph(s)
    for _ in range(3):
        flush.fill_(1)
        pipe.run_eager()
    torch.cuda.synchronize()
    # launch shapes picked by the autotuner on this workload (results do not depend on them)
    from paper_1703_06256_gb300 import autotune

    tuned = None if args.no_tune else autotune.tune_pipeline(pipe, autotune.Autotuner(), reps=30)
    step, read_total, timing_mode = graph_step(torch, fns, between=False)
    step_st, read_stages, _ = graph_step(torch, fns, between=True)
    for _ in range(max(args.warmup, 3)):
        for fn in (step, step_st):
            flush.fill_(1)
            fn()
    torch.cuda.synchronize()

    sampler = ClockSampler(local)
    sampler.start()
    t_end = time.perf_counter() + 2.0  # soak, so the clock record covers steady state
    while time.perf_counter() < t_end:
        flush.fill_(1)
        step()
        torch.cuda.synchronize()

    # timed region: each step is replayed from its graph after an L2 flush;
    # the events are recorded by the GPU at the two ends of the step
    def run_step(k):
        flush.fill_(k)
        step()

    mine_ms = timed_region(run_step, lambda: read_total()[1], args.steps,
                           dist.barrier if dist is not None else None, torch.cuda.synchronize)
    clocks = sampler.stop()
    # the slowest replica sets the time; the rate counts every rank's pixels
    ms_per_step = replicas.max_over_ranks(mine_ms, device="cuda")

    # per-stage breakdown (same steps, events between the stages)
    stage_ms = {n: 0.0 for n in names}
    for k in range(args.steps):
        flush.fill_(k)
        step_st()
        torch.cuda.synchronize()
        st, _ = read_stages()
        for n, v in zip(names, st):
            stage_ms[n] += v
    px = W * H
    value = replicas.aggregate_rate(px, ms_per_step * 1e-3, world) / 1e6
    windows = pipe.nx * pipe.ny

    # the serving comparison first among the extras, on a GPU that has run only the main step so far
    # (the library's own launch shapes; the main step's tuned ones are put back afterwards)
    autotune.reset()
    serving_res = (serving(torch, wl, args) if "serving" in extras and world == 1 and args.serve_requests > 0
                   else None)
    if tuned:
        autotune.apply(tuned["config"])

    # the same five calls with the other integral-image type (uint16 modulo 2^16 beside int32, or the
    # reverse): every result of the path is the same, the planes take half (or twice) the bytes
    other_ii = None
    if "ii_other" in extras:
        op = fh.HogPipeline(W, H, 3, c["n_bins"], c["stride"], cell_dtype=fh.HOG_BF16,
                            ii_dtype=fh.HOG_I32 if ii_u16 else fh.HOG_U16)
        op.set_weights(c["w"], c["bias"], c["thr"])
        op.set_image(img)
        for _ in range(3):
            op.run_eager()
        ostep, oread, _ = graph_step(torch, [op.stage_bin_map, op.stage_integral, op.stage_cell_hist,
                                             op.stage_score, op.stage_detect], between=False)
        oms = time_steps(torch, ostep, oread, flush, args.steps, args.warmup)
        other_ii = {"integral_images": "int32" if ii_u16 else "uint16 modulo 2^16",
                    "value": round(replicas.aggregate_rate(W * H, replicas.max_over_ranks(oms, "cuda") * 1e-3,
                                                           world) / 1e6, 2),
                    "unit": "Mpixel/s", "ms_per_step": round(oms, 5),
                    "launch_shapes": "the main step's" if tuned else "library defaults"}
        del op

    # the same step with the fused image-to-cells kernel (no bin map or integral planes in HBM)
    fused = None
    if "fused" in extras:
        pipe.fused = True
        ftuned = None if args.no_tune else autotune.tune_pipeline(pipe, autotune.Autotuner(), reps=30)
        fstep, fread, _ = graph_step(torch, [pipe.stage_cells_fused, pipe.stage_score, pipe.stage_detect],
                                     between=False)
        fused_ms = time_steps(torch, fstep, fread, flush, args.steps, args.warmup)
        pipe.fused = False
        fused = {"value": round(replicas.aggregate_rate(W * H, replicas.max_over_ranks(fused_ms, "cuda") * 1e-3,
                                                        world) / 1e6, 2),
                 "unit": "Mpixel/s", "ms_per_step": round(fused_ms, 5),
                 "calls": "hog_cell_hist_fused + hog_window_score + hog_detect", "tuned": ftuned}

    # the end-to-end figures run with the library's own launch shapes, as a caller of the public API
    # gets them (the tuning above picks shapes for one image at a time, and leaves its choice applied)
    autotune.reset()

    # end to end through the public API, from pinned host memory (graph replay: image copy, five calls,
    # detections and count written by the GPU into pinned host memory, one synchronisation)
    def one_at_a_time(zero_copy):
        pipe.capture_host(zero_copy)
        for _ in range(3):
            pipe.detect_host()
        d2h_ = []
        t0 = time.perf_counter()
        for _ in range(args.steps):
            _, n = pipe.detect_host()
            d2h_.append(4 + min(n, pipe.max_out) * fh.DET_BYTES)
        return replicas.max_over_ranks((time.perf_counter() - t0) / args.steps, device="cuda"), d2h_

    e2e_s, d2h = one_at_a_time(False)
    e2e_zc_s, _ = one_at_a_time(True)

    # end to end through the request server (the public serving API): the same five calls on the same
    # image, each step one request -- its image copied in from pinned host memory, its detections written
    # to host memory -- with up to 16 requests on the GPU at once
    from paper_1703_06256_gb300.serve import HogServer, Request

    srv = HogServer(c["w"], c["bias"], c["thr"], n_bins=c["n_bins"], stride=c["stride"], w_dtype=fh.HOG_F32,
                    budget_bytes=2 << 30, n_streams=16, fused=False, max_wh=(W, H))
    img_pinned = torch.from_numpy(np.ascontiguousarray(img)).pin_memory()
    srv.serve_native([Request(k, img_pinned, 0.0) for k in range(64)], keep=False)  # warm-up
    n_req = max(args.steps * 5, 500)
    t0 = time.perf_counter()
    res, _ = srv.serve_native([Request(k, img_pinned, 0.0) for k in range(n_req)], keep=False)
    wall_s = replicas.max_over_ranks((time.perf_counter() - t0) / n_req, device="cuda")
    # the server's own clock: from the first request queued to the last one's detections in host memory
    span_ns = max(r.t_done_ns for r in res) - min(r.t_enqueue_ns for r in res)
    served_s = replicas.max_over_ranks(span_ns * 1e-9 / n_req, device="cuda")
    served_d2h = 4 + int(statistics.mean(r.count for r in res)) * fh.DET_BYTES
    srv.close()

    # roofline of the dominant stage
    stage_avg = {k: v / args.steps for k, v in stage_ms.items()}
    dom = max(stage_avg, key=stage_avg.get)
    nb = c["n_bins"]
    alg_bytes = algorithmic_bytes(W, H, nb, pipe.ncx, pipe.ncy, windows, ii_bytes=2 if ii_u16 else 4)
    hbm, src = peaks()
    achieved = alg_bytes[dom] / (stage_avg[dom] * 1e-3) / 1e9
    # bin map 1; integral 1 (single pass) or 3 per window of bins, under the knobs the step was captured
    # with; cell histograms 1; score 1; detection 1 (single pass)
    if tuned:
        autotune.apply(tuned["config"])
    launches_per_step = 1 + fh.hog_integral_launches(W, H, nb) + 1 + 1 + 1
    status = fh.hog_device_status()
    autotune.reset()  # the extras below run with the library's own launch shapes
    # the serving comparison runs right after the main measurement, before the heavier extras,
    # so that both of its paths see the GPU in the state the main step saw
    autotune.reset()  # the remaining figures run with the library's own launch shapes
    out = {
        "metric": METRIC, "value": round(value, 2), "unit": "Mpixel/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": round(ms_per_step, 5), "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "u16+f32" if ii_u16 else "int32+f32", "data": "synthetic",
        "config": {"workload": WORKLOAD.replace("800x600", f"{W}x{H}"), "image": f"{W}x{H}x3", "windows_per_image": windows,
                   "integral_images": "uint16 modulo 2^16" if ii_u16 else "int32",
                   "l2": "flushed between steps (256 MB write, outside the timed events)",
                   "lut": "built once before timing", "timing": timing_mode,
                   "launch_shapes": "autotuned" if tuned else "library defaults", "tuned": tuned},
        "windows_per_s": round(world * windows / (ms_per_step * 1e-3), 1),
        "stages_ms": {k: round(v, 5) for k, v in stage_avg.items()},
        "roofline": {"kernel": dom, "bound": "hbm", "achieved": round(achieved, 1), "peak": hbm, "unit": "GB/s",
                     "frac": round(achieved / hbm, 4),
                     "traffic": profiled_traffic(dom, f"{W}x{H}" + ("-u16" if ii_u16 else "")),
                     "peak_source": src, "algorithmic_bytes_per_launch": alg_bytes[dom],
                     "traffic_source": "profiles/traffic.txt (ncu, summed over the stage's kernels)"},
        "e2e": {"value": round(replicas.aggregate_rate(px, served_s, world) / 1e6, 2), "unit": "Mpixel/s",
                "h2d_bytes_per_step": pipe.h2d_bytes(), "d2h_bytes_per_step": served_d2h,
                "api": "HogServer (native dispatcher: hog_server_enqueue / hog_server_collect), five calls per "
                       "request, 16 in flight",
                "requests": n_req,
                "timing": "server clock, first request queued to the last request's detections in host memory",
                "wall_value": round(replicas.aggregate_rate(px, wall_s, world) / 1e6, 2),
                "one_at_a_time": {"value": round(replicas.aggregate_rate(px, e2e_s, world) / 1e6, 2),
                                  "unit": "Mpixel/s",
                                  "api": "HogPipeline.detect_host (one graph: image copy, five calls, list into pinned "
                                         "host memory; one synchronisation per image)",
                                  "d2h_bytes_per_step": int(statistics.mean(d2h)),
                                  "zero_copy": {"value": round(replicas.aggregate_rate(px, e2e_zc_s, world) / 1e6, 2),
                                                "unit": "Mpixel/s",
                                                "api": "HogPipeline.detect_host after capture_host(zero_copy=True): "
                                                       "the bin map reads the pinned image in place (its bytes "
                                                       "cross to the GPU inside that kernel), no copy node"}}},
        "gpu_launches": launches_per_step * args.steps,
        "clocks": clocks,
        "device_status": status,
        "fused": fused,
        "ii_other": other_ii,
        "stages_4k": stage_rooflines(torch, fh, wl, flush, args, hbm) if "stages_4k" in extras else None,
        "batch_1080p": batch_1080p(torch, fh, wl, replicas, flush, args, world) if "batch_1080p" in extras else None,
        "precision": measured_precision(),
        "batch_pyramid": (batch_pyramid(torch, fh, wl, replicas, flush, args, world) if "batch_pyramid" in extras
                          else None),
        "multi_filter": (multi_filter(torch, fh, wl, flush, args, bf16_peak()) if "multi_filter" in extras
                         else None),
        "blocks": blocks_variant(torch, fh, wl, flush, args) if "blocks" in extras else None,
        "soft": soft_variant(torch, fh, wl, flush, args) if "soft" in extras else None,
        "serving": serving_res,
    }
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        out["cpu_baseline"] = cpu_baseline(img, c, args.cpu_seconds)
    if rank == 0:
        print(json.dumps(out), flush=True)
    if dist is not None:
        dist.destroy_process_group()


if __name__ == "__main__":
    sys.exit(main() or 0)
