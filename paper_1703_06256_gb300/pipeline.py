"""HogPipeline: device buffers for one image size plus the five per-image
calls of the C ABI, in the paper's order (bin map -> integral images -> cell
histograms -> window scores -> detections).

Buffers are allocated once with PyTorch (the C ABI never allocates); the
gradient table is built once per N_b at construction (the paper builds it a
single time and only reads it afterwards).  ``run`` enqueues the five calls
on a stream; ``detect_host`` is the end-to-end path a caller with a host
image uses: copy in, run, copy the detections out.
"""

from __future__ import annotations

import numpy as np
import torch

from . import (DET_BYTES, HOG_BF16, HOG_F32, HOG_I8, HOG_I32, HOG_LUT_BYTES, HOG_U16, TORCH_DTYPE,
               dets_to_numpy, grid_shapes, hog_bin_map, hog_build_lut, hog_cell_hist, hog_cell_hist_fused,
               hog_detect, hog_detect_workspace_bytes, hog_integral, hog_integral_workspace_bytes,
               hog_window_score)

_W_DTYPE = {HOG_F32: torch.float32, HOG_BF16: torch.bfloat16, HOG_I8: torch.int8}


class HogPipeline:
    def __init__(self, W: int, H: int, channels: int = 3, n_bins: int = 8, stride: int = 8, cell: int = 8,
                 cells_x: int = 8, cells_y: int = 16, ii_dtype: int = HOG_I32, cell_dtype: int = HOG_F32,
                 w_dtype: int = HOG_F32, max_out: int | None = None, device: str | torch.device = "cuda"):
        self.W, self.H, self.channels, self.n_bins = W, H, channels, n_bins
        self.stride, self.cell, self.cells_x, self.cells_y = stride, cell, cells_x, cells_y
        self.ii_dtype, self.cell_dtype, self.w_dtype = ii_dtype, cell_dtype, w_dtype
        self.device = torch.device(device)
        self.ncx, self.ncy, self.nx, self.ny = grid_shapes(W, H, cell, stride, cells_x, cells_y)
        self.max_out = max(self.nx * self.ny, 1) if max_out is None else max_out
        dev = self.device
        self.lut = torch.empty(HOG_LUT_BYTES, dtype=torch.uint8, device=dev)
        self.img = torch.empty(H * W * channels, dtype=torch.uint8, device=dev)
        self.bins = torch.empty(H * W, dtype=torch.uint8, device=dev)
        self.ii = torch.empty(n_bins * H * W, dtype=TORCH_DTYPE[ii_dtype], device=dev)
        self.ws_ii_bytes = hog_integral_workspace_bytes(W, H, n_bins)
        # workspaces start zero-filled (the single-pass kernels' contract) and are never cleared again
        self.ws_ii = torch.zeros(max(self.ws_ii_bytes, 256), dtype=torch.uint8, device=dev)
        self.cells = torch.empty(max(self.ncx * self.ncy * n_bins, 1), dtype=TORCH_DTYPE[cell_dtype], device=dev)
        self.score_dtype = HOG_I32 if w_dtype == HOG_I8 else HOG_F32
        self.scores = torch.empty(max(self.nx * self.ny, 1), dtype=TORCH_DTYPE[self.score_dtype], device=dev)
        self.det = torch.empty(self.max_out * DET_BYTES, dtype=torch.uint8, device=dev)
        self.count = torch.zeros(1, dtype=torch.int32, device=dev)
        self.ws_det_bytes = hog_detect_workspace_bytes(self.nx, self.ny)
        self.ws_det = torch.zeros(max(self.ws_det_bytes, 256), dtype=torch.uint8, device=dev)
        self.w = torch.zeros(cells_x * cells_y * n_bins, dtype=_W_DTYPE[w_dtype], device=dev)
        self.bias = 0.0
        self.thr = 0.0
        with torch.cuda.device(dev):
            hog_build_lut(n_bins, self.lut)
        # pinned host staging for the end-to-end path
        self.img_host = torch.empty(H * W * channels, dtype=torch.uint8, pin_memory=True)
        self.count_host = torch.zeros(1, dtype=torch.int32, pin_memory=True)
        self.det_host = torch.empty(self.max_out * DET_BYTES, dtype=torch.uint8, pin_memory=True)
        # numpy views of the same page-locked memory: reading them costs no torch dispatch
        self._count_np = self.count_host.numpy()
        self._det_np = self.det_host.numpy()

    def set_weights(self, w, bias: float = 0.0, thr: float = 0.0) -> None:
        t = torch.as_tensor(np.asarray(w)).reshape(-1)
        if t.numel() != self.w.numel():
            raise ValueError(f"expected {self.w.numel()} weights, got {t.numel()}")
        self.w.copy_(t.to(self.w.dtype))
        self.bias, self.thr = float(bias), float(thr)
        self.graph = None  # bias and threshold are launch arguments: recapture

    def set_image(self, img: np.ndarray) -> None:
        a = np.ascontiguousarray(img, dtype=np.uint8).reshape(-1)
        self.img.copy_(torch.from_numpy(a))

    # -- the five per-image calls (`img`: where the bin map reads the image, by default the device copy)
    def stage_bin_map(self, stream=None, img=None):
        hog_bin_map(self.img if img is None else img, self.W, self.H, self.channels, self.W * self.channels, self.lut,
                    self.n_bins, self.bins, stream)

    def stage_integral(self, stream=None):
        hog_integral(self.bins, self.W, self.H, self.n_bins, self.ii_dtype, self.ii, self.ws_ii, self.ws_ii_bytes,
                     stream)

    def stage_cell_hist(self, stream=None):
        hog_cell_hist(self.ii, self.W, self.H, self.n_bins, self.ii_dtype, self.cell, self.stride, self.cell_dtype,
                      self.cells, stream)

    def stage_score(self, stream=None):
        hog_window_score(self.cells, self.cell_dtype, self.ncx, self.ncy, self.n_bins, self.cells_x, self.cells_y,
                         self.cell, self.stride, self.w, self.w_dtype, self.bias, self.scores, stream)

    def stage_detect(self, stream=None):
        hog_detect(self.scores, self.score_dtype, self.nx, self.ny, self.stride, self.thr, 0, 0, self.det,
                   self.max_out, self.count, self.ws_det, self.ws_det_bytes, stream)

    def stage_cells_fused(self, stream=None, img=None):
        """Bin map, integral images and cell histograms in one call (the bin
        map and the integral planes are not written)."""
        hog_cell_hist_fused(self.img if img is None else img, self.W, self.H, self.channels, self.W * self.channels,
                            self.lut, self.n_bins, self.cell, self.stride, self.cell_dtype, self.cells, stream)

    fused = False

    def run_eager(self, stream=None) -> None:
        """Enqueue the calls for the image already in ``self.img``: the five
        separate stages, or (fused=True) the fused image-to-cells call, the
        score and the list."""
        if self.fused:
            self.stage_cells_fused(stream)
        else:
            self.stage_bin_map(stream)
            self.stage_integral(stream)
            self.stage_cell_hist(stream)
        self.stage_score(stream)
        self.stage_detect(stream)

    def capture(self) -> None:
        """Record the five calls once as a CUDA graph; ``run`` then replays it
        (one launch instead of eight, no host work between the kernels).  The
        calls allocate nothing and never synchronise, so they capture as is.
        Weights, bias and threshold must be set before capturing."""
        with torch.cuda.device(self.device):
            s = torch.cuda.Stream(self.device)
            s.wait_stream(torch.cuda.current_stream(self.device))
            with torch.cuda.stream(s):
                self.run_eager(s)  # first launches load the kernels outside the capture
            torch.cuda.current_stream(self.device).wait_stream(s)
            g = torch.cuda.CUDAGraph()
            with torch.cuda.graph(g):
                self.run_eager()
            self.graph = g

    graph = None

    def run(self, stream=None) -> None:
        """Enqueue the whole path: the captured graph if there is one."""
        if self.graph is not None:
            if stream is None:
                self.graph.replay()
            else:
                with torch.cuda.stream(stream):
                    self.graph.replay()
        else:
            self.run_eager(stream)

    def _enqueue_host(self, zero_copy: bool = False) -> None:
        """The whole path from the page-locked image to page-locked results:
        the image's host-to-device copy (or, with zero_copy, none: the first
        kernel reads the page-locked image in place, which is mapped into
        the device's address space, so its bytes cross to the GPU inside that
        kernel), the calls, and the detection list and its count written by
        hog_detect straight into page-locked host memory."""
        src = self.img_host if zero_copy else self.img
        if not zero_copy:
            self.img.copy_(self.img_host, non_blocking=True)
        if self.fused:
            self.stage_cells_fused(img=src)
        else:
            self.stage_bin_map(img=src)
            self.stage_integral()
            self.stage_cell_hist()
        self.stage_score()
        hog_detect(self.scores, self.score_dtype, self.nx, self.ny, self.stride, self.thr, 0, 0, self.det_host,
                   self.max_out, self.count_host, self.ws_det, self.ws_det_bytes)

    host_graph = None

    def capture_host(self, zero_copy: bool = False) -> None:
        """Record _enqueue_host as one CUDA graph (copy node + kernels, or the
        kernels alone with zero_copy); after it, detect_host is one replay
        and one synchronisation."""
        with torch.cuda.device(self.device):
            s = torch.cuda.Stream(self.device)
            s.wait_stream(torch.cuda.current_stream(self.device))
            with torch.cuda.stream(s):
                self._enqueue_host(zero_copy)  # first launches load the kernels outside the capture
            s.synchronize()
            g = torch.cuda.CUDAGraph()
            with torch.cuda.graph(g):
                self._enqueue_host(zero_copy)
            self.host_graph = g

    def detect_host(self, img_host: torch.Tensor | None = None, stream=None):
        """End to end from pinned host memory: the image is copied in, the
        path runs, and the GPU writes the count and the detections straight
        into pinned host memory; one synchronisation.  Returns the
        detections as a numpy record array and the count."""
        if img_host is not None:
            self.img_host.copy_(img_host.reshape(-1))
        if stream is None:
            s = torch.cuda.current_stream(self.device)
            if self.host_graph is not None:
                self.host_graph.replay()
            else:
                self._enqueue_host()
        else:
            s = stream
            with torch.cuda.stream(s):
                if self.host_graph is not None:
                    self.host_graph.replay()
                else:
                    self._enqueue_host()
        s.synchronize()
        n_all = int(self._count_np[0])
        n = min(n_all, self.max_out)
        return dets_to_numpy(self._det_np, n), n_all

    def h2d_bytes(self) -> int:
        return self.img.numel()

    def results(self) -> dict:
        """Copy every intermediate to host numpy arrays (for tests)."""
        torch.cuda.synchronize(self.device)
        ii = self.ii.view(torch.int16) if self.ii_dtype == HOG_U16 else self.ii
        ii_np = ii.cpu().numpy()
        if self.ii_dtype == HOG_U16:
            ii_np = ii_np.view(np.uint16)
        cells = self.cells.float() if self.cell_dtype == HOG_BF16 else self.cells
        n = int(self.count.item())
        return {
            "bins": self.bins.cpu().numpy().reshape(self.H, self.W),
            "ii": ii_np.reshape(self.n_bins, self.H, self.W),
            "cells": cells.cpu().numpy().reshape(self.ncy, self.ncx, self.n_bins).astype(np.int64),
            "scores": self.scores[: self.nx * self.ny].cpu().numpy().reshape(self.ny, self.nx),
            "count": n,
            "detections": dets_to_numpy(self.det.cpu(), min(n, self.max_out)),
        }
