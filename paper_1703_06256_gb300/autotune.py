"""Autotuner for the library's launch-shape knobs (``hog_tune_*`` in
include/fasthog.h): the integral-image scan's band height (rows per tile),
the bin-map and fused-cells grid caps, where those two kernels read the
gradient table, the cell-histogram kernel's tile height (or its per-cell
form), the score's engine (CUDA or tensor cores) and the tensor-core score's
rows per CTA.  None of them changes a result; they change only how the work is cut.

The tuner times each candidate on the caller's own workload through the
library's calls -- the per-image path captured as a CUDA graph, CUDA events
around each replay, the L2 flushed between replays -- and keeps the fastest.
The search is coordinate descent from the library's defaults (value 0 for
every knob): one knob at a time over its candidates, the others held at the
best so far, repeated until a sweep changes nothing.  The defaults and the
winner are then measured once more, side by side, and the winner is kept only
if it still beats the defaults (the first configuration a process measures
can read slow).  Results are cached in a JSON file per device and workload.
"""

from __future__ import annotations

import json
import os
import statistics

from . import (HOG_TUNE_BINMAP_CTAS_PER_SM, HOG_TUNE_CELL_ROWS, HOG_TUNE_FUSED_CTAS_PER_SM, HOG_TUNE_TABLE,
               HOG_TUNE_INTEGRAL_BAND_ROWS, HOG_TUNE_INTEGRAL_PATH, HOG_TUNE_INTEGRAL_WARP_ROWS, HOG_TUNE_SCORE_PATH,
               HOG_TUNE_SCORE_TC_ROWS, HOG_TUNE_BINMAP_SCHEDULE, HOG_TUNE_FUSED_TILE_ROWS,
               HOG_TUNE_SLIDE_WINDOWS, hog_tune_get, hog_tune_set)

# knob name -> (hog_tune_knob, candidate values; 0 = the library's own choice)
KNOBS = {
    "integral_band_rows": (HOG_TUNE_INTEGRAL_BAND_ROWS, (0, 4, 8, 16, 32)),
    "binmap_ctas_per_sm": (HOG_TUNE_BINMAP_CTAS_PER_SM, (0, 1, 2, 4)),
    "binmap_schedule": (HOG_TUNE_BINMAP_SCHEDULE, (0, 1, 2)),
    "fused_ctas_per_sm": (HOG_TUNE_FUSED_CTAS_PER_SM, (0, 1)),
    "fused_tile_rows": (HOG_TUNE_FUSED_TILE_ROWS, (0, 4, 8, 16)),
    "score_tc_rows": (HOG_TUNE_SCORE_TC_ROWS, (0, 2, 4, 8, 16, 32)),
    "table": (HOG_TUNE_TABLE, (0, 1, 2)),
    "cell_rows": (HOG_TUNE_CELL_ROWS, (0, 1, 4, 8, 16)),
    "score_path": (HOG_TUNE_SCORE_PATH, (0, 1, 2, 3)),
    "slide_windows": (HOG_TUNE_SLIDE_WINDOWS, (0, 8, 16)),
    "integral_path": (HOG_TUNE_INTEGRAL_PATH, (0, 1, 2, 3)),
    "integral_warp_rows": (HOG_TUNE_INTEGRAL_WARP_ROWS, (0, 2, 4, 8)),
}
# the knobs each path's launches read
PATH_KNOBS = {
    "separate": ("integral_path", "integral_warp_rows", "integral_band_rows", "binmap_schedule", "binmap_ctas_per_sm", "cell_rows", "score_path",
                 "score_tc_rows", "slide_windows", "table"),
    "fused": ("fused_ctas_per_sm", "fused_tile_rows", "score_path", "score_tc_rows", "slide_windows", "table"),
}


def apply(config: dict) -> None:
    """Set every knob named in `config` (others keep their value)."""
    for name, value in config.items():
        hog_tune_set(KNOBS[name][0], int(value))


def current() -> dict:
    return {name: hog_tune_get(k) for name, (k, _) in KNOBS.items()}


def reset() -> None:
    apply({name: 0 for name in KNOBS})


def search(candidates: dict, measure, max_sweeps: int = 3):
    """Coordinate descent over `candidates` (name -> values) with `measure`
    (config -> time, lower is better).  Starts from the first value of every
    knob.  Returns (best config, best time, {config key: time} of every
    measurement)."""
    best = {name: vals[0] for name, vals in candidates.items()}
    seen: dict = {}

    def timed(cfg):
        key = json.dumps(cfg, sort_keys=True)
        if key not in seen:
            seen[key] = measure(dict(cfg))
        return seen[key]

    best_t = timed(best)
    for _ in range(max_sweeps):
        changed = False
        for name, vals in candidates.items():
            for v in vals:
                if v == best[name]:
                    continue
                cfg = dict(best, **{name: v})
                t = timed(cfg)
                if t < best_t:
                    best, best_t, changed = cfg, t, True
        if not changed:
            break
    return best, best_t, seen


class Autotuner:
    """Cached tuning: ``tune(workload, measure, knobs)`` returns the best
    knob values for `workload` (a dict naming it), measuring only on a cache
    miss."""

    def __init__(self, cache_path: str | None = None, device_name: str | None = None):
        self.cache_path = cache_path
        self.device_name = device_name or _device_name()
        self.cache: dict = {}
        if cache_path and os.path.exists(cache_path):
            with open(cache_path) as f:
                self.cache = json.load(f)

    def key(self, workload: dict) -> str:
        return json.dumps({"device": self.device_name, **workload}, sort_keys=True)

    def tune(self, workload: dict, measure, knobs) -> dict:
        k = self.key(workload)
        hit = self.cache.get(k)
        if hit is not None:
            return hit
        cand = {name: KNOBS[name][1] for name in knobs}
        best, best_t, seen = search(cand, measure)
        # the first configuration measured (the defaults) may have run slow;
        # measure the defaults and the winner once more, side by side, and
        # keep the defaults unless the winner still beats them
        default = {name: 0 for name in knobs}
        default_t = measure(dict(default))
        if best != default:
            best_t = measure(dict(best))
            if best_t >= default_t:
                best, best_t = default, default_t
        else:
            best_t = default_t
        entry = {"config": best, "ms": best_t, "default_ms": default_t, "measured": len(seen) + 2}
        self.cache[k] = entry
        if self.cache_path:
            tmp = self.cache_path + ".tmp"
            with open(tmp, "w") as f:
                json.dump(self.cache, f, indent=1, sort_keys=True)
            os.replace(tmp, self.cache_path)
        return entry


def _device_name() -> str:
    import torch

    return torch.cuda.get_device_name(0) if torch.cuda.is_available() else "cpu"


def pipeline_measure(pipe, reps: int = 20, flush_bytes: int = 256 << 20, warm_s: float = 0.5):
    """A `measure` for `search`: apply the knobs, recapture `pipe`'s graph
    (launch shapes are fixed at capture), and return the mean device time
    (ms) of `reps` replays, each after an L2 flush, without the fastest and
    slowest tenth (event times come in steps of about a microsecond, so a
    mean separates launch shapes that a median would tie).  Before its first
    measurement it replays the step for `warm_s` seconds: the first steps
    after a pause run slower, and the first configuration measured (the
    defaults) would otherwise carry that."""
    import time

    import torch

    flush = torch.empty(flush_bytes // 4, dtype=torch.int32, device=pipe.device)
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
    warmed = [False]

    def measure(cfg: dict) -> float:
        apply(cfg)
        pipe.graph = None
        pipe.capture()
        if not warmed[0]:
            t_end = time.perf_counter() + warm_s
            while time.perf_counter() < t_end:
                for _ in range(50):
                    flush.fill_(0)
                    pipe.run()
                torch.cuda.synchronize(pipe.device)
            warmed[0] = True
        times = []
        for k in range(reps + 3):
            flush.fill_(k)
            ev[0].record()
            pipe.run()
            ev[1].record()
            torch.cuda.synchronize(pipe.device)
            if k >= 3:
                times.append(ev[0].elapsed_time(ev[1]))
        times.sort()
        cut = len(times) // 10
        return statistics.fmean(times[cut: len(times) - cut])

    return measure


def tune_pipeline(pipe, tuner: Autotuner | None = None, reps: int = 20) -> dict:
    """Tune the knobs of `pipe`'s path (HogPipeline, image and weights set)
    and leave the best values applied.  Returns the cache entry."""
    tuner = tuner or Autotuner()
    path = "fused" if pipe.fused else "separate"
    workload = {"W": pipe.W, "H": pipe.H, "channels": pipe.channels, "n_bins": pipe.n_bins, "stride": pipe.stride,
                "cell": pipe.cell, "ii_dtype": pipe.ii_dtype, "cell_dtype": pipe.cell_dtype,
                "w_dtype": pipe.w_dtype, "path": path}
    entry = tuner.tune(workload, pipeline_measure(pipe, reps), PATH_KNOBS[path])
    apply(entry["config"])
    pipe.graph = None
    return entry


__all__ = ["KNOBS", "PATH_KNOBS", "Autotuner", "apply", "current", "reset", "search", "pipeline_measure",
           "tune_pipeline"]
