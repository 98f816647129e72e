"""Batches of images of any sizes through the detection path.

HogBatch: many images in one CUDA graph of per-image calls.

Each image keeps its own HogPipeline (buffers sized for it, its own table
copy and workspaces), so images never share scratch.  The images are dealt
round-robin to `n_streams` streams; each stream runs its images' calls in
order (with programmatic dependent launch between consecutive kernels), and
the streams are independent branches of one graph, so the GPU overlaps the
images' kernels.  One replay runs the whole batch with one launch.

HogPlanBatch: images and their pyramid levels through the batch calls of
include/fasthog_batch.h, one kernel launch per stage for the whole batch.
"""

from __future__ import annotations

import numpy as np
import torch

from .pipeline import HogPipeline


class HogBatch:
    def __init__(self, pipes: list[HogPipeline], n_streams: int = 4, fused: bool = False):
        if not pipes:
            raise ValueError("empty batch")
        self.pipes = pipes
        self.n_streams = max(1, min(n_streams, len(pipes)))
        self.fused = fused
        self.graph = None

    def _calls(self, pipe: HogPipeline):
        pipe.fused = self.fused
        if self.fused:
            return [pipe.stage_cells_fused, pipe.stage_score, pipe.stage_detect]
        return [pipe.stage_bin_map, pipe.stage_integral, pipe.stage_cell_hist, pipe.stage_score, pipe.stage_detect]

    def enqueue(self, events=None) -> None:
        """Enqueue the batch on the current stream (forking to side streams and
        joining back); usable eagerly or under graph capture.  `events`, if
        given, is a pair recorded at the start and at the end."""
        main = torch.cuda.current_stream()
        if events is not None:
            events[0].record(main)
        streams = [torch.cuda.Stream() for _ in range(self.n_streams)]
        for s in streams:
            s.wait_stream(main)
        for k, pipe in enumerate(self.pipes):
            s = streams[k % self.n_streams]
            with torch.cuda.stream(s):
                for call in self._calls(pipe):
                    call(s)
        for s in streams:
            main.wait_stream(s)
        if events is not None:
            events[1].record(main)

    def capture(self, events=None) -> None:
        """Record the batch as one graph (after one eager pass, which loads
        every kernel)."""
        self.enqueue()
        torch.cuda.synchronize()
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g):
            self.enqueue(events)
        self.graph = g

    def run(self) -> None:
        if self.graph is None:
            self.enqueue()
        else:
            self.graph.replay()


class HogPlanBatch:
    """Images of uneven sizes, each with its 2:1 pyramid levels, through the
    batch calls of include/fasthog_batch.h: one launch per stage over every
    (image, level) item of the batch -- fused cells, tensor-core (or
    CUDA-core) score, and one detection list for the whole batch -- after one
    hog_pyramid launch per image.

    Buffers are allocated once for the given sizes; ``set_images`` fills
    them, ``capture`` records the stages as one CUDA graph and ``run``
    replays it.  Each detection carries its image index and pyramid level."""

    def __init__(self, sizes, channels: int = 3, levels: int = 1, n_bins: int = 8, stride: int = 4, cell: int = 8,
                 cells_x: int = 8, cells_y: int = 16, cell_dtype: int | None = None, w_dtype: int | None = None,
                 device="cuda"):
        from . import (DET_BYTES, HOG_BF16, HOG_I8, HOG_I32, HOG_F32, HOG_LUT_BYTES, TORCH_DTYPE, HogBatchItem,
                       grid_shapes, hog_batch_plan, hog_build_lut, hog_detect_batch_workspace_bytes,
                       hog_pyramid_bytes)

        self.device = torch.device(device)
        self.sizes = [tuple(s) for s in sizes]
        self.channels, self.levels, self.n_bins = channels, levels, n_bins
        self.stride, self.cell, self.cells_x, self.cells_y = stride, cell, cells_x, cells_y
        self.w_dtype = HOG_BF16 if w_dtype is None else w_dtype
        # counts of cells up to 16 x 16 are exact in bf16, and the tensor-core scores read bf16 cells
        # (with any weight type)
        self.cell_dtype = (HOG_BF16 if cell <= 16 else HOG_F32) if cell_dtype is None else cell_dtype
        self.score_dtype = HOG_I32 if self.w_dtype == HOG_I8 else HOG_F32
        dev = self.device
        self.lut = torch.empty(HOG_LUT_BYTES, dtype=torch.uint8, device=dev)
        with torch.cuda.device(dev):
            hog_build_lut(n_bins, self.lut)
        self.imgs, self.pyr, self.items, self.item_meta = [], [], [], []
        self.cells, self.scores = [], []
        for k, (W, H) in enumerate(self.sizes):
            img = torch.zeros(H * W * channels, dtype=torch.uint8, device=dev)
            pyr = torch.zeros(max(hog_pyramid_bytes(W, H, channels, levels), 16), dtype=torch.uint8, device=dev)
            self.imgs.append(img)
            self.pyr.append(pyr)
            off = 0
            for lv in range(levels):
                Wl, Hl = W >> lv, H >> lv
                if Wl < 1 or Hl < 1:
                    break
                base = img.data_ptr() if lv == 0 else pyr.data_ptr() + off
                if lv > 0:
                    off += Wl * Hl * channels
                ncx, ncy, nx, ny = grid_shapes(Wl, Hl, cell, stride, cells_x, cells_y)
                c = torch.zeros(max(ncx * ncy * n_bins, 8), dtype=TORCH_DTYPE[self.cell_dtype], device=dev)
                sc = torch.zeros(max(nx * ny, 1), dtype=TORCH_DTYPE[self.score_dtype], device=dev)
                self.cells.append(c)
                self.scores.append(sc)
                self.items.append(HogBatchItem(base, Wl * channels, Wl, Hl, c.data_ptr(), sc.data_ptr(), k, lv))
                self.item_meta.append(dict(image=k, level=lv, W=Wl, H=Hl, ncx=ncx, ncy=ncy, nx=nx, ny=ny))
        self.plan = hog_batch_plan(self.items, channels, n_bins, cell, stride, cells_x, cells_y)
        self.plan_dev = torch.frombuffer(bytearray(bytes(self.plan)), dtype=torch.uint8).to(dev)
        self.windows = sum(m["nx"] * m["ny"] for m in self.item_meta)
        self.max_out = max(self.windows, 1)
        self.det = torch.empty(self.max_out * DET_BYTES, dtype=torch.uint8, device=dev)
        self.count = torch.zeros(1, dtype=torch.int32, device=dev)
        self.item_counts = torch.zeros(len(self.items), dtype=torch.int32, device=dev)
        self.ws_bytes = hog_detect_batch_workspace_bytes(self.plan)
        self.ws = torch.empty(self.ws_bytes, dtype=torch.uint8, device=dev)
        self.w = None
        self.bias, self.thr = 0.0, 0.0
        self.graph = None
        self.pixels = sum(m["W"] * m["H"] for m in self.item_meta)

    def set_images(self, images) -> None:
        for img, buf in zip(images, self.imgs):
            buf.copy_(torch.from_numpy(np.ascontiguousarray(img, dtype=np.uint8).reshape(-1)))

    def set_weights(self, w, bias: float = 0.0, thr: float = 0.0) -> None:
        from . import HOG_BF16, HOG_F32, HOG_I8

        t = torch.as_tensor(np.asarray(w)).reshape(-1)
        dt = {HOG_F32: torch.float32, HOG_BF16: torch.bfloat16, HOG_I8: torch.int8}[self.w_dtype]
        self.w = t.to(dt).to(self.device)
        self.bias, self.thr = float(bias), float(thr)
        self.graph = None

    def enqueue(self, stream=None) -> None:
        from . import (hog_cell_hist_fused_batch, hog_detect_batch, hog_pyramid, hog_window_score_batch)

        if self.levels > 1:
            for (W, H), img, pyr in zip(self.sizes, self.imgs, self.pyr):
                hog_pyramid(img, W, H, self.channels, W * self.channels, self.levels, pyr, stream)
        hog_cell_hist_fused_batch(self.plan, self.plan_dev, self.lut, self.cell_dtype, stream)
        hog_window_score_batch(self.plan, self.plan_dev, self.cell_dtype, self.w, self.w_dtype, self.bias, stream)
        hog_detect_batch(self.plan, self.plan_dev, self.score_dtype, self.thr, self.det, self.max_out, self.count,
                         self.item_counts, self.ws, self.ws_bytes, stream)

    def capture(self, events=None) -> None:
        s = torch.cuda.Stream(self.device)
        s.wait_stream(torch.cuda.current_stream(self.device))
        with torch.cuda.stream(s):
            self.enqueue(s)  # first launches load the kernels outside the capture
        torch.cuda.current_stream(self.device).wait_stream(s)
        torch.cuda.synchronize(self.device)
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g):
            if events is not None:
                events[0].record()
            self.enqueue()
            if events is not None:
                events[1].record()
        self.graph = g

    def run(self) -> None:
        if self.graph is None:
            self.enqueue()
        else:
            self.graph.replay()

    def launches(self) -> int:
        """Kernels one pass launches: pyramids, fused cells, score, and the
        detection count, scan and scatter."""
        from . import HOG_BF16

        n_pyr = len(self.sizes) if self.levels > 1 else 0
        tc = (self.cell_dtype == HOG_BF16 and self.n_bins in (8, 16)
              and (self.cells_x, self.cells_y) == (8, 16) and self.cell // self.stride in (1, 2, 4))
        score = 1 if tc else sum(1 for m in self.item_meta if m["nx"] * m["ny"] > 0)
        return n_pyr + 1 + score + (3 if self.windows > 0 else 1)

    def results(self) -> dict:
        """Per item cells, scores and detections, plus the whole list (for tests)."""
        from . import dets_to_numpy

        torch.cuda.synchronize(self.device)
        n = int(self.count.item())
        out = {"count": n, "item_counts": self.item_counts.cpu().numpy(),
               "detections": dets_to_numpy(self.det.cpu(), min(n, self.max_out)), "items": []}
        for m, c, sc in zip(self.item_meta, self.cells, self.scores):
            cf = c.float() if c.dtype == torch.bfloat16 else c
            out["items"].append(dict(m, cells=cf.cpu().numpy()[: m["ncx"] * m["ncy"] * self.n_bins].reshape(
                m["ncy"], m["ncx"], self.n_bins).astype(np.int64),
                scores=sc.cpu().numpy()[: m["nx"] * m["ny"]].reshape(m["ny"], m["nx"])))
        return out
