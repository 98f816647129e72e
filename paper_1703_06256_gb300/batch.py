"""HogBatch: many images, of any sizes, through the detection path in one
CUDA graph.

Each image keeps its own HogPipeline (buffers sized for it, its own table
copy and workspaces), so images never share scratch.  The images are dealt
round-robin to `n_streams` streams; each stream runs its images' calls in
order (with programmatic dependent launch between consecutive kernels), and
the streams are independent branches of one graph, so the GPU overlaps the
images' kernels.  One replay runs the whole batch with one launch.
"""

from __future__ import annotations

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
