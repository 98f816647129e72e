"""HogServer: continuous batching of detection requests on one GPU.

Requests (RGB or gray images of any size) are admitted as they arrive,
subject to two limits: a device-memory budget (the sum of the working sets
of the requests on the GPU) and a pool of CUDA streams.  The gradient table
and the weights are built once and stay resident; every admitted request
gets its own buffers and stream, so requests that overlap on the GPU never
share memory, and a request's result does not depend on what else is
running.  Completion is collected without blocking: a request's count
arrives first (event 1), then the list of exactly that many detections is
copied out (event 2).

The per-request path is the fused one (hog_cell_hist_fused, hog_window_score,
hog_detect) when the parameters allow it, otherwise the five separate calls.
"""

from __future__ import annotations

import collections
import time
from dataclasses import dataclass, field

import numpy as np
import torch

from . import (DET_BYTES, HOG_BF16, HOG_F32, HOG_I8, HOG_I32, HOG_LUT_BYTES, TORCH_DTYPE, dets_to_numpy,
               grid_shapes, hog_bin_map, hog_build_lut, hog_cell_hist, hog_cell_hist_fused, hog_detect,
               hog_detect_workspace_bytes, hog_integral, hog_integral_workspace_bytes, hog_window_score)

_W_DTYPE = {HOG_F32: torch.float32, HOG_BF16: torch.bfloat16, HOG_I8: torch.int8}


def _fused_ok(n_bins, cell, stride):
    return n_bins in (8, 16) and stride in (4, 8) and cell % stride == 0 and cell // stride <= 4


@dataclass
class Request:
    rid: int
    image: object              # (H, W) or (H, W, 3) uint8: numpy array or (pinned) CPU tensor
    arrival: float = 0.0       # seconds, on the server's clock


@dataclass
class _Flight:
    req: Request
    stream: torch.cuda.Stream
    bufs: dict
    nbytes: int
    ev_count: torch.cuda.Event
    ev_list: torch.cuda.Event | None = None
    count: int = -1
    t_submit: float = 0.0


@dataclass
class Result:
    rid: int
    detections: np.ndarray
    count: int
    latency: float             # completion - arrival, seconds
    shape: tuple = field(default=())


class HogServer:
    def __init__(self, w, bias: float = 0.0, thr: float = 0.5, n_bins: int = 8, stride: int = 4, cell: int = 8,
                 cells_x: int = 8, cells_y: int = 16, w_dtype: int = HOG_BF16, budget_bytes: int = 8 << 30,
                 n_streams: int = 16, fused: bool | None = None, device="cuda"):
        self.n_bins, self.stride, self.cell = n_bins, stride, cell
        self.cells_x, self.cells_y = cells_x, cells_y
        self.bias, self.thr = float(bias), float(thr)
        self.w_dtype = w_dtype
        self.score_dtype = HOG_I32 if w_dtype == HOG_I8 else HOG_F32
        self.cell_dtype = HOG_BF16 if w_dtype in (HOG_BF16, HOG_I8) and cell <= 16 else HOG_F32
        self.fused = _fused_ok(n_bins, cell, stride) if fused is None else fused
        self.budget = int(budget_bytes)
        self.device = torch.device(device)
        self.lut = torch.empty(HOG_LUT_BYTES, dtype=torch.uint8, device=self.device)
        hog_build_lut(n_bins, self.lut)
        t = torch.as_tensor(np.asarray(w)).reshape(-1)
        self.w = t.to(_W_DTYPE[w_dtype]).to(self.device)
        self.free_streams = collections.deque(torch.cuda.Stream(self.device) for _ in range(n_streams))
        self.flights: list[_Flight] = []
        self.used = 0
        torch.cuda.synchronize(self.device)

    # ---- sizes
    def working_set(self, W: int, H: int, channels: int) -> int:
        """Device bytes a request of this size holds while on the GPU."""
        ncx, ncy, nx, ny = grid_shapes(W, H, self.cell, self.stride, self.cells_x, self.cells_y)
        esz = {HOG_I32: 4, HOG_F32: 4, HOG_BF16: 2}
        b = W * H * channels + ncx * ncy * self.n_bins * esz[self.cell_dtype] + max(nx * ny, 1) * 4
        b += max(nx * ny, 1) * DET_BYTES + hog_detect_workspace_bytes(nx, ny) + 256
        if not self.fused:
            b += W * H + self.n_bins * W * H * 4 + hog_integral_workspace_bytes(W, H, self.n_bins)
        return b

    # ---- admission
    def try_submit(self, req: Request, now: float) -> bool:
        img = req.image
        H, W = img.shape[:2]
        ch = 1 if img.ndim == 2 else 3
        need = self.working_set(W, H, ch)
        if not self.free_streams or (self.flights and self.used + need > self.budget):
            return False
        s = self.free_streams.popleft()
        ncx, ncy, nx, ny = grid_shapes(W, H, self.cell, self.stride, self.cells_x, self.cells_y)
        dev = self.device
        with torch.cuda.stream(s):
            bufs = {
                "img": torch.empty(H * W * ch, dtype=torch.uint8, device=dev),
                "cells": torch.empty(max(ncx * ncy * self.n_bins, 1), dtype=TORCH_DTYPE[self.cell_dtype], device=dev),
                "scores": torch.empty(max(nx * ny, 1), dtype=TORCH_DTYPE[self.score_dtype], device=dev),
                "det": torch.empty(max(nx * ny, 1) * DET_BYTES, dtype=torch.uint8, device=dev),
                "count": torch.zeros(1, dtype=torch.int32, device=dev),
                "ws_det": torch.empty(max(hog_detect_workspace_bytes(nx, ny), 256), dtype=torch.uint8, device=dev),
                "count_host": torch.zeros(1, dtype=torch.int32, pin_memory=True),
                # a pinned request image is copied from directly; anything else is staged once
                "img_host": (img.reshape(-1) if isinstance(img, torch.Tensor) and img.is_pinned()
                             else torch.from_numpy(np.ascontiguousarray(img, dtype=np.uint8).reshape(-1)).pin_memory()),
            }
            if not self.fused:
                bufs["bins"] = torch.empty(H * W, dtype=torch.uint8, device=dev)
                bufs["ii"] = torch.empty(self.n_bins * H * W, dtype=torch.int32, device=dev)
                wsb = hog_integral_workspace_bytes(W, H, self.n_bins)
                bufs["ws_ii"] = torch.empty(max(wsb, 256), dtype=torch.uint8, device=dev)
            bufs["img"].copy_(bufs["img_host"], non_blocking=True)
            if self.fused:
                hog_cell_hist_fused(bufs["img"], W, H, ch, W * ch, self.lut, self.n_bins, self.cell, self.stride,
                                    self.cell_dtype, bufs["cells"], s)
            else:
                hog_bin_map(bufs["img"], W, H, ch, W * ch, self.lut, self.n_bins, bufs["bins"], s)
                hog_integral(bufs["bins"], W, H, self.n_bins, HOG_I32, bufs["ii"], bufs["ws_ii"],
                             bufs["ws_ii"].numel(), s)
                hog_cell_hist(bufs["ii"], W, H, self.n_bins, HOG_I32, self.cell, self.stride, self.cell_dtype,
                              bufs["cells"], s)
            hog_window_score(bufs["cells"], self.cell_dtype, ncx, ncy, self.n_bins, self.cells_x, self.cells_y,
                             self.cell, self.stride, self.w, self.w_dtype, self.bias, bufs["scores"], s)
            hog_detect(bufs["scores"], self.score_dtype, nx, ny, self.stride, self.thr, req.rid, 0, bufs["det"],
                       max(nx * ny, 1), bufs["count"], bufs["ws_det"], bufs["ws_det"].numel(), s)
            bufs["count_host"].copy_(bufs["count"], non_blocking=True)
            ev = torch.cuda.Event()
            ev.record(s)
        self.flights.append(_Flight(req, s, bufs, need, ev, t_submit=now))
        self.used += need
        return True

    # ---- completion
    def poll(self, now_fn) -> list[Result]:
        done: list[Result] = []
        keep: list[_Flight] = []
        for f in self.flights:
            if f.ev_list is None:
                if not f.ev_count.query():
                    keep.append(f)
                    continue
                f.count = int(f.bufs["count_host"][0])
                n = min(f.count, f.bufs["det"].numel() // DET_BYTES)
                f.bufs["n"] = n
                f.bufs["det_host"] = torch.empty(max(n, 1) * DET_BYTES, dtype=torch.uint8, pin_memory=True)
                with torch.cuda.stream(f.stream):
                    if n:
                        f.bufs["det_host"][: n * DET_BYTES].copy_(f.bufs["det"][: n * DET_BYTES], non_blocking=True)
                    f.ev_list = torch.cuda.Event()
                    f.ev_list.record(f.stream)
                keep.append(f)
                continue
            if not f.ev_list.query():
                keep.append(f)
                continue
            n = f.bufs["n"]
            dets = dets_to_numpy(f.bufs["det_host"], n)
            done.append(Result(f.req.rid, dets, f.count, now_fn() - f.req.arrival, f.req.image.shape))
            self.used -= f.nbytes
            self.free_streams.append(f.stream)
        self.flights = keep
        return done

    def idle(self) -> bool:
        return not self.flights

    # ---- drivers
    def serve(self, requests: list[Request], poll_sleep: float = 0.0) -> list[Result]:
        """Replay `requests` at their arrival times (seconds from now),
        admitting each as soon as it has arrived and fits; returns the
        results in completion order."""
        t0 = time.perf_counter()
        clock = lambda: time.perf_counter() - t0  # noqa: E731
        queue = collections.deque(sorted(requests, key=lambda r: r.arrival))
        results: list[Result] = []
        while queue or self.flights:
            now = clock()
            while queue and queue[0].arrival <= now and self.try_submit(queue[0], now):
                queue.popleft()
            got = self.poll(clock)
            results += got
            if not got and poll_sleep:
                time.sleep(poll_sleep)
        return results

    def run_one(self, image: np.ndarray, rid: int = 0) -> Result:
        """The plain per-image path: submit one request and wait for it."""
        t0 = time.perf_counter()
        clock = lambda: time.perf_counter() - t0  # noqa: E731
        req = Request(rid, image, 0.0)
        while not self.try_submit(req, clock()):
            self.poll(clock)
        while True:
            got = self.poll(clock)
            if got:
                return got[0]


def latency_summary(results: list[Result], wall: float) -> dict:
    lat = np.array([r.latency for r in results]) * 1e3
    px = sum(int(np.prod(r.shape[:2])) for r in results)
    return {"requests": len(results), "p50_ms": round(float(np.percentile(lat, 50)), 3),
            "p99_ms": round(float(np.percentile(lat, 99)), 3), "images_per_s": round(len(results) / wall, 1),
            "mpixel_per_s": round(px / wall / 1e6, 1)}
