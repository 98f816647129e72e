"""HogServer: continuous batching of detection requests on one GPU.

A thin Python face on the library's native request server
(include/fasthog_server.h).  Requests (RGB or gray images of any size) are
admitted as they arrive, subject to a free slot (one CUDA stream each) and a
device-memory budget; the gradient table and the weights stay resident, and
every admitted request gets buffers of its own carved from one device arena,
so requests that overlap on the GPU never share memory and a request's result
does not depend on what else is running.  The GPU writes each request's
detection list straight into page-locked host memory; completion is
collected without blocking.  Python here only replays arrivals, polls, and
copies the detections out.
"""

from __future__ import annotations

import collections
import ctypes
import gc
import time
from dataclasses import dataclass, field

import numpy as np
import torch

from . import (DET_BYTES, HOG_BF16, HOG_F32, HOG_I8, HOG_I32, HogServerConfig, HogServerResult,
               HogServerTimedResult, dets_to_numpy, hog_server_clock_ns, hog_server_collect, hog_server_create,
               hog_server_destroy, hog_server_enqueue, hog_server_poll, hog_server_release, hog_server_request_bytes,
               hog_server_pauses, hog_server_start, hog_server_stats, hog_server_stop, hog_server_submit)

_MAX_POLL = 64


def _weights_host(w, w_dtype: int) -> np.ndarray:
    t = torch.as_tensor(np.asarray(w)).reshape(-1)
    if w_dtype == HOG_F32:
        return t.to(torch.float32).numpy().copy()
    if w_dtype == HOG_BF16:
        return t.to(torch.bfloat16).view(torch.int16).numpy().copy()
    if w_dtype == HOG_I8:
        return t.to(torch.int8).numpy().copy()
    raise ValueError(f"weight dtype {w_dtype}")


@dataclass
class Request:
    rid: int
    image: object              # (H, W) or (H, W, 3) uint8: numpy array or (pinned) CPU tensor
    arrival: float = 0.0       # seconds, on the server's clock


@dataclass
class Result:
    rid: int
    detections: np.ndarray | None
    count: int
    latency: float             # completion - arrival, seconds
    shape: tuple = field(default=())
    t_enqueue_ns: int = 0      # native stamps (serve_native only): queued, put on the GPU, seen complete
    t_done_ns: int = 0
    t_admit_ns: int = 0


class HogServer:
    def __init__(self, w, bias: float = 0.0, thr: float = 0.5, n_bins: int = 8, stride: int = 4, cell: int = 8,
                 cells_x: int = 8, cells_y: int = 16, w_dtype: int = HOG_BF16, budget_bytes: int = 8 << 30,
                 n_streams: int = 16, fused: bool | None = None, ii_dtype: int = HOG_I32,
                 max_wh: tuple = (3840, 2160), image_in_place: bool = False, device=None):
        self.device = torch.device("cuda") if device is None else torch.device(device)
        cfg = HogServerConfig(n_bins=n_bins, cell=cell, stride=stride, cells_x=cells_x, cells_y=cells_y,
                              w_dtype=w_dtype, bias=float(bias), thr=float(thr),
                              fused=-1 if fused is None else int(bool(fused)), ii_dtype=ii_dtype,
                              n_slots=n_streams, budget_bytes=int(budget_bytes), max_W=max_wh[0], max_H=max_wh[1],
                              image_in_place=int(bool(image_in_place)))
        self.n_streams = n_streams
        self.fused = fused  # None: fused wherever hog_cell_hist_fused supports the parameters
        self._w = _weights_host(w, w_dtype)
        with torch.cuda.device(self.device):
            torch.cuda.init()
            self._h = hog_server_create(cfg, self._w)
        self._out = (HogServerResult * _MAX_POLL)()
        self._inflight: dict[int, tuple] = {}

    def close(self) -> None:
        if getattr(self, "_h", None) is not None:
            hog_server_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # ---- sizes and state
    def working_set(self, W: int, H: int, channels: int) -> int:
        """Device bytes a request of this size holds while on the GPU."""
        return hog_server_request_bytes(self._h, W, H, channels)

    @property
    def used(self) -> int:
        return hog_server_stats(self._h)[1]

    def idle(self) -> bool:
        return hog_server_stats(self._h)[0] == 0 and not self._inflight

    # ---- admission and completion
    def try_submit(self, req: Request, now: float = 0.0) -> bool:
        img = req.image
        if isinstance(img, torch.Tensor):
            img = img if img.is_contiguous() else img.contiguous()
        else:
            img = np.ascontiguousarray(img, dtype=np.uint8)
        H, W = img.shape[:2]
        ch = 1 if img.ndim == 2 else 3
        if req.rid in self._inflight:
            raise ValueError(f"request id {req.rid} is already on the GPU")
        if not hog_server_submit(self._h, req.rid, img, W, H, ch):
            return False
        self._inflight[req.rid] = (req, img)  # the image must outlive the request
        return True

    def poll(self, now_fn, keep: bool = True) -> list[Result]:
        n = hog_server_poll(self._h, self._out, _MAX_POLL)
        done = []
        t = now_fn()
        for k in range(n):
            r = self._out[k]
            if r.status != 0:
                raise RuntimeError(f"request {r.rid} failed on the GPU (status {r.status})")
            dets = None
            if keep:
                raw = ctypes.string_at(r.dets, r.count * DET_BYTES) if r.count else b""
                dets = dets_to_numpy(raw, r.count)
            hog_server_release(self._h, r.token)
            req, _ = self._inflight.pop(r.rid)
            done.append(Result(r.rid, dets, r.count, t - req.arrival, (r.H, r.W)))
        return done

    # ---- drivers
    def serve(self, requests: list[Request], keep: bool = True) -> list[Result]:
        """Replay `requests` at their arrival times (seconds from now),
        admitting each as soon as it has arrived and fits; returns the
        results in completion order."""
        queue = collections.deque(sorted(requests, key=lambda r: r.arrival))
        results: list[Result] = []
        gc_was_on = gc.isenabled()
        gc.disable()  # a collection pause would land in some request's latency
        try:
            t0 = time.perf_counter()
            clock = lambda: time.perf_counter() - t0  # noqa: E731
            while queue or self._inflight:
                now = clock()
                while queue and queue[0].arrival <= now and self.try_submit(queue[0], now):
                    queue.popleft()
                results += self.poll(clock, keep)
        finally:
            if gc_was_on:
                gc.enable()
        return results

    def serve_native(self, requests: list[Request], keep: bool = True) -> tuple[list[Result], dict]:
        """Replay `requests` at their arrival times through the server's own
        dispatcher thread (hog_server_start): this thread only queues each
        request when it arrives and collects results; admission and
        completion run natively.  Latency is the native enqueue-to-done
        time.  Returns the results in completion order and the replay's own
        lateness (how far behind its arrival time a request was queued)."""
        queue = sorted(requests, key=lambda r: r.arrival)
        # the images as the C ABI takes them (contiguous), kept alive until their results are in
        imgs = []
        for req in queue:
            img = req.image
            img = (img if img.is_contiguous() else img.contiguous()) if isinstance(img, torch.Tensor) \
                else np.ascontiguousarray(img, dtype=np.uint8)
            imgs.append(img)
        arrivals = [req.arrival for req in queue]
        out = (HogServerTimedResult * _MAX_POLL)()
        raw = []  # per completed request: its stamps and, with keep, its detections
        late = []
        n_total, n_done = len(queue), 0
        gc_was_on = gc.isenabled()
        gc.disable()
        hog_server_start(self._h)
        try:
            t0 = hog_server_clock_ns()
            i = 0
            while n_done < n_total:
                if i < n_total:
                    now = (hog_server_clock_ns() - t0) * 1e-9
                    while i < n_total and arrivals[i] <= now:
                        img = imgs[i]
                        H, W = img.shape[:2]
                        hog_server_enqueue(self._h, queue[i].rid, img, W, H, 1 if img.ndim == 2 else 3)
                        late.append(now - arrivals[i])
                        i += 1
                n = hog_server_collect(self._h, out, _MAX_POLL)
                for k in range(n):
                    t = out[k]
                    r = t.r
                    if r.status != 0:
                        raise RuntimeError(f"request {r.rid} failed on the GPU (status {r.status})")
                    dets = None
                    if keep:
                        dets = ctypes.string_at(r.dets, r.count * DET_BYTES) if r.count else b""
                    hog_server_release(self._h, r.token)  # the slot is free again before any other work
                    raw.append((r.rid, dets, r.count, r.H, r.W, t.t_enqueue_ns, t.t_done_ns, t.t_admit_ns))
                n_done += n
        finally:
            hog_server_stop(self._h)
            if gc_was_on:
                gc.enable()
        results = [Result(rid, dets_to_numpy(d, cnt) if keep else None, cnt, (td - te) * 1e-9, (h, w), te, td, ta)
                   for rid, d, cnt, h, w, te, td, ta in raw]
        n_pauses, pauses = hog_server_pauses(self._h)
        lat = np.array(late) * 1e3 if late else np.zeros(1)
        return results, {"replay_late_p50_ms": round(float(np.percentile(lat, 50)), 3),
                         "replay_late_p99_ms": round(float(np.percentile(lat, 99)), 3),
                         "dispatcher_pauses": n_pauses, "pauses_ns": pauses}

    def run_one(self, image, rid: int = 0) -> Result:
        """The plain per-image path: submit one request and wait for it."""
        t0 = time.perf_counter()
        clock = lambda: time.perf_counter() - t0  # noqa: E731
        req = Request(rid, image, 0.0)
        while not self.try_submit(req, clock()):
            self.poll(clock)
        while True:
            got = [r for r in self.poll(clock) if r.rid == rid]
            if got:
                return got[0]


def latency_summary(results: list[Result], wall: float, pauses_ns=None, long_pause_ms: float = 5.0) -> dict:
    """p50/p99 over every request.  With the dispatcher's pause record
    (serve_native), also the pauses of at least `long_pause_ms` (the process
    was not running: whatever was queued or on the GPU then waited) and p99
    over the requests whose enqueue-to-done span overlaps none of them."""
    lat = np.array([r.latency for r in results]) * 1e3
    px = sum(int(np.prod(r.shape[:2])) for r in results)
    out = {"requests": len(results), "p50_ms": round(float(np.percentile(lat, 50)), 3),
           "p99_ms": round(float(np.percentile(lat, 99)), 3), "images_per_s": round(len(results) / wall, 1),
           "mpixel_per_s": round(px / wall / 1e6, 1)}
    if pauses_ns is not None:
        long_ = [(a, b) for a, b in pauses_ns if (b - a) * 1e-6 >= long_pause_ms]
        hit = np.array([any(a < r.t_done_ns and b > r.t_enqueue_ns for a, b in long_) for r in results], bool)
        clear = lat[~hit] if (~hit).any() else lat
        out.update({"long_pauses": len(long_),
                    "longest_pause_ms": round(max(((b - a) * 1e-6 for a, b in pauses_ns), default=0.0), 3),
                    "requests_in_long_pauses": int(hit.sum()),
                    "p99_ms_outside_long_pauses": round(float(np.percentile(clear, 99)), 3)})
        # where the slowest requests spent their time: waiting for a slot or memory, or on the GPU
        t0 = min(r.t_enqueue_ns for r in results)
        slow = sorted(results, key=lambda r: -r.latency)[:5]
        out["slowest"] = [{"W": r.shape[1], "H": r.shape[0], "at_ms": round((r.t_enqueue_ns - t0) * 1e-6, 2),
                           "wait_ms": round((r.t_admit_ns - r.t_enqueue_ns) * 1e-6, 3),
                           "gpu_ms": round((r.t_done_ns - r.t_admit_ns) * 1e-6, 3)} for r in slow]
    return out
