"""Python binding of libfasthog, the GB300 (sm_103a) fast-HOG detection library.

The functions below carry the names of the C ABI in ``include/fasthog.h`` and
do argument marshalling only: every step runs in the library's CUDA kernels.
Tensors are PyTorch CUDA tensors (PyTorch provides device memory and streams);
each call enqueues work on the given stream (default: the current stream) and
returns.  A non-OK status raises :class:`HogError`.

There is no CPU path: if the library has not been built, importing this
package raises.  Build it with ``python paper_1703_06256_gb300/build.py``.
"""

from __future__ import annotations

import ctypes
import os

import torch

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_build", "libfasthog.so")

HOG_OK, HOG_ERR_ARG, HOG_ERR_UNSUPPORTED, HOG_ERR_CUDA, HOG_ERR_TIMEOUT = range(5)
HOG_U8, HOG_I32, HOG_BF16, HOG_F32, HOG_I8, HOG_U16 = range(6)
HOG_NO_BIN = 0xFF
HOG_LUT_SIDE = 511
HOG_LUT_PITCH = 512
HOG_LUT_QUAD_OFFSET = HOG_LUT_SIDE * HOG_LUT_PITCH
HOG_LUT_BYTES = HOG_LUT_QUAD_OFFSET + 256 * 256
HOG_STATUS_TIMEOUT = 1
HOG_SOFT_Q = 64
HOG_SOFT_LUT_BYTES = HOG_LUT_SIDE * HOG_LUT_PITCH * 2
(HOG_TUNE_INTEGRAL_BAND_ROWS, HOG_TUNE_BINMAP_CTAS_PER_SM, HOG_TUNE_FUSED_CTAS_PER_SM,
 HOG_TUNE_SCORE_TC_ROWS, HOG_TUNE_TABLE, HOG_TUNE_CELL_ROWS, HOG_TUNE_SCORE_PATH, HOG_TUNE_SLIDE_WINDOWS,
 HOG_TUNE_INTEGRAL_PATH, HOG_TUNE_INTEGRAL_WARP_ROWS, HOG_TUNE_BINMAP_SCHEDULE, HOG_TUNE_FUSED_TILE_ROWS) = range(12)
HOG_TUNE_KNOBS = 12

TORCH_DTYPE = {HOG_U8: torch.uint8, HOG_I32: torch.int32, HOG_BF16: torch.bfloat16, HOG_F32: torch.float32,
               HOG_I8: torch.int8, HOG_U16: torch.uint16 if hasattr(torch, "uint16") else torch.int16}


class HogDet(ctypes.Structure):
    _fields_ = [("x", ctypes.c_int32), ("y", ctypes.c_int32), ("score", ctypes.c_float),
                ("image", ctypes.c_int32), ("level", ctypes.c_int32)]


DET_BYTES = ctypes.sizeof(HogDet)  # 20


class HogBatchItem(ctypes.Structure):
    """hog_batch_item of include/fasthog_batch.h."""
    _fields_ = [("img", ctypes.c_void_p), ("pitch", ctypes.c_size_t), ("W", ctypes.c_int), ("H", ctypes.c_int),
                ("cells", ctypes.c_void_p), ("scores", ctypes.c_void_p), ("image", ctypes.c_int),
                ("level", ctypes.c_int)]


class HogServerConfig(ctypes.Structure):
    """hog_server_config of include/fasthog_server.h."""
    _fields_ = [("n_bins", ctypes.c_int), ("cell", ctypes.c_int), ("stride", ctypes.c_int),
                ("cells_x", ctypes.c_int), ("cells_y", ctypes.c_int), ("w_dtype", ctypes.c_int),
                ("bias", ctypes.c_float), ("thr", ctypes.c_float), ("fused", ctypes.c_int),
                ("ii_dtype", ctypes.c_int), ("n_slots", ctypes.c_int), ("budget_bytes", ctypes.c_size_t),
                ("max_W", ctypes.c_int), ("max_H", ctypes.c_int), ("image_in_place", ctypes.c_int)]


class HogServerResult(ctypes.Structure):
    """hog_server_result of include/fasthog_server.h."""
    _fields_ = [("rid", ctypes.c_int32), ("status", ctypes.c_int32), ("count", ctypes.c_int32),
                ("token", ctypes.c_int32), ("W", ctypes.c_int32), ("H", ctypes.c_int32),
                ("dets", ctypes.c_void_p)]


class HogServerTimedResult(ctypes.Structure):
    """hog_server_timed_result of include/fasthog_server.h."""
    _fields_ = [("r", HogServerResult), ("t_enqueue_ns", ctypes.c_int64), ("t_admit_ns", ctypes.c_int64),
                ("t_done_ns", ctypes.c_int64)]


class HogError(RuntimeError):
    def __init__(self, fn: str, status: int, cuda_error: int = 0):
        self.status = status
        self.cuda_error = cuda_error
        names = ["HOG_OK", "HOG_ERR_ARG", "HOG_ERR_UNSUPPORTED", "HOG_ERR_CUDA", "HOG_ERR_TIMEOUT"]
        name = names[status] if 0 <= status < len(names) else str(status)
        extra = f" (cudaError {cuda_error})" if status == HOG_ERR_CUDA else ""
        super().__init__(f"{fn} failed: {name}{extra}")


def _load() -> ctypes.CDLL:
    if not os.path.exists(LIB_PATH):
        raise ImportError(f"libfasthog is not built ({LIB_PATH} missing); run "
                          "`python paper_1703_06256_gb300/build.py` (needs nvcc)")
    lib = ctypes.CDLL(LIB_PATH)
    P, I, Z, F = ctypes.c_void_p, ctypes.c_int, ctypes.c_size_t, ctypes.c_float
    sig = {
        "hog_status_string": (ctypes.c_char_p, [I]),
        "hog_last_cuda_error": (I, []),
        "hog_version": (I, []),
        "hog_device_status": (I, [P, I]),
        "hog_selftest_wait_timeout": (I, [I, I, P]),
        "hog_build_lut": (I, [I, P, P]),
        "hog_bin_map": (I, [P, I, I, I, Z, P, I, P, P]),
        "hog_integral_workspace_bytes": (Z, [I, I, I]),
        "hog_integral_launches": (I, [I, I, I]),
        "hog_integral": (I, [P, I, I, I, I, P, P, Z, P]),
        "hog_cell_hist": (I, [P, I, I, I, I, I, I, I, P, P]),
        "hog_window_score": (I, [P, I, I, I, I, I, I, I, I, P, I, F, P, P]),
        "hog_detect_workspace_bytes": (Z, [I, I]),
        "hog_detect": (I, [P, I, I, I, I, F, I, I, P, I, P, P, Z, P]),
        "hog_detect_noalloc": (I, [P, I, I, I, I, F, I, I, P, I, P, P]),
        "hog_cell_hist_fused": (I, [P, I, I, I, Z, P, I, I, I, I, P, P]),
        "hog_build_soft_lut": (I, [I, P, P]),
        "hog_cell_hist_soft": (I, [P, I, I, I, Z, P, I, I, I, I, P, P]),
        "hog_block_norm": (I, [P, I, I, I, I, I, F, P, P]),
        "hog_window_score_multi": (I, [P, I, I, I, I, I, I, I, I, P, I, I, P, P, P]),
        "hog_tune_set": (I, [I, I]),
        "hog_tune_get": (I, [I]),
        "hog_batch_plan_bytes": (Z, [I]),
        "hog_batch_plan": (I, [P, I, I, I, I, I, I, I, P, Z]),
        "hog_cell_hist_fused_batch": (I, [P, P, P, I, P]),
        "hog_window_score_batch": (I, [P, P, I, P, I, F, P]),
        "hog_detect_batch_workspace_bytes": (Z, [P]),
        "hog_detect_batch": (I, [P, P, I, F, P, I, P, P, P, Z, P]),
        "hog_pyramid_bytes": (Z, [I, I, I, I]),
        "hog_pyramid": (I, [P, I, I, I, Z, I, P, P]),
        "hog_server_create": (I, [P, P, P]),
        "hog_server_destroy": (I, [P]),
        "hog_server_request_bytes": (Z, [P, I, I, I]),
        "hog_server_submit": (I, [P, ctypes.c_int32, P, I, I, I, P]),
        "hog_server_poll": (I, [P, P, I, P]),
        "hog_server_release": (I, [P, ctypes.c_int32]),
        "hog_server_stats": (I, [P, P, P, P]),
        "hog_server_start": (I, [P]),
        "hog_server_stop": (I, [P]),
        "hog_server_enqueue": (I, [P, ctypes.c_int32, P, I, I, I]),
        "hog_server_collect": (I, [P, P, I, P]),
        "hog_server_clock_ns": (ctypes.c_int64, []),
        "hog_server_pauses": (I, [P, P, P, I, P]),
    }
    for name, (res, args) in sig.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    return lib


_lib = _load()
EXPORTED = ("hog_status_string", "hog_last_cuda_error", "hog_version", "hog_device_status",
            "hog_selftest_wait_timeout", "hog_build_lut",
            "hog_bin_map", "hog_integral_workspace_bytes", "hog_integral_launches", "hog_integral", "hog_cell_hist", "hog_window_score",
            "hog_detect_workspace_bytes", "hog_detect", "hog_detect_noalloc", "hog_cell_hist_fused",
            "hog_build_soft_lut", "hog_cell_hist_soft", "hog_block_norm", "hog_window_score_multi", "hog_tune_set", "hog_tune_get", "hog_batch_plan_bytes", "hog_batch_plan", "hog_cell_hist_fused_batch", "hog_window_score_batch",
            "hog_detect_batch_workspace_bytes", "hog_detect_batch", "hog_pyramid_bytes", "hog_pyramid",
            "hog_server_create", "hog_server_destroy", "hog_server_request_bytes", "hog_server_submit",
            "hog_server_poll", "hog_server_release", "hog_server_stats", "hog_server_start", "hog_server_stop",
            "hog_server_enqueue", "hog_server_collect", "hog_server_clock_ns", "hog_server_pauses")


def lib() -> ctypes.CDLL:
    return _lib


def _ptr(x) -> int | None:
    if x is None:
        return None
    if isinstance(x, torch.Tensor):
        if x.device.type != "cuda" and not x.is_pinned():
            # page-locked host memory is mapped into the device's address space (same address)
            raise ValueError("libfasthog takes CUDA tensors or page-locked CPU tensors; got pageable host memory")
        return x.data_ptr()
    return int(x)


def _host_ptr(x) -> int:
    """Address of a contiguous HOST buffer (numpy array or CPU tensor)."""
    if isinstance(x, torch.Tensor):
        if x.device.type != "cpu" or not x.is_contiguous():
            raise ValueError("expected a contiguous CPU tensor (host memory)")
        return x.data_ptr()
    if not x.flags["C_CONTIGUOUS"]:
        raise ValueError("expected a C-contiguous numpy array")
    return x.ctypes.data


def _stream(stream) -> int | None:
    if stream is None:
        return torch.cuda.current_stream().cuda_stream
    if isinstance(stream, torch.cuda.Stream):
        return stream.cuda_stream
    return int(stream)


def _check(fn: str, status: int) -> None:
    if status != HOG_OK:
        raise HogError(fn, status, _lib.hog_last_cuda_error() if status == HOG_ERR_CUDA else 0)


# ---- entry points (same names and argument order as the C ABI) -------------

def hog_version() -> int:
    return _lib.hog_version()


def hog_device_status(clear: bool = False) -> int:
    v = ctypes.c_uint32(0)
    _check("hog_device_status", _lib.hog_device_status(ctypes.addressof(v), int(clear)))
    return v.value


def hog_selftest_wait_timeout(mode: int, limit_us: int, stream=None) -> None:
    """Run one bounded device-side wait that runs out (mode 0: an mbarrier,
    mode 1: a device-memory flag); the kernel sets HOG_STATUS_TIMEOUT."""
    _check("hog_selftest_wait_timeout", _lib.hog_selftest_wait_timeout(mode, limit_us, _stream(stream)))


def hog_build_lut(n_bins: int, lut, stream=None) -> None:
    _check("hog_build_lut", _lib.hog_build_lut(n_bins, _ptr(lut), _stream(stream)))


def hog_bin_map(img, W: int, H: int, channels: int, pitch_bytes: int, lut, n_bins: int, bins,
                stream=None) -> None:
    _check("hog_bin_map", _lib.hog_bin_map(_ptr(img), W, H, channels, pitch_bytes, _ptr(lut), n_bins,
                                           _ptr(bins), _stream(stream)))


def hog_integral_launches(W: int, H: int, n_bins: int) -> int:
    return _lib.hog_integral_launches(W, H, n_bins)


def hog_integral_workspace_bytes(W: int, H: int, n_bins: int) -> int:
    return _lib.hog_integral_workspace_bytes(W, H, n_bins)


def hog_integral(bins, W: int, H: int, n_bins: int, ii_dtype: int, ii, workspace, workspace_bytes: int,
                 stream=None) -> None:
    _check("hog_integral", _lib.hog_integral(_ptr(bins), W, H, n_bins, ii_dtype, _ptr(ii), _ptr(workspace),
                                             workspace_bytes, _stream(stream)))


def hog_cell_hist(ii, W: int, H: int, n_bins: int, ii_dtype: int, cell: int, stride: int, cell_dtype: int,
                  cells, stream=None) -> None:
    _check("hog_cell_hist", _lib.hog_cell_hist(_ptr(ii), W, H, n_bins, ii_dtype, cell, stride, cell_dtype,
                                               _ptr(cells), _stream(stream)))


def hog_cell_hist_fused(img, W: int, H: int, channels: int, pitch_bytes: int, lut, n_bins: int, cell: int,
                        stride: int, cell_dtype: int, cells, stream=None) -> None:
    _check("hog_cell_hist_fused", _lib.hog_cell_hist_fused(_ptr(img), W, H, channels, pitch_bytes, _ptr(lut), n_bins,
                                                           cell, stride, cell_dtype, _ptr(cells), _stream(stream)))


def hog_window_score(cells, cell_dtype: int, ncx: int, ncy: int, n_bins: int, cells_x: int, cells_y: int,
                     cell: int, stride: int, w, w_dtype: int, bias: float, scores, stream=None) -> None:
    _check("hog_window_score", _lib.hog_window_score(_ptr(cells), cell_dtype, ncx, ncy, n_bins, cells_x, cells_y,
                                                     cell, stride, _ptr(w), w_dtype, float(bias), _ptr(scores),
                                                     _stream(stream)))


def hog_build_soft_lut(n_bins: int, lut, stream=None) -> None:
    _check("hog_build_soft_lut", _lib.hog_build_soft_lut(n_bins, _ptr(lut), _stream(stream)))


def hog_cell_hist_soft(img, W: int, H: int, channels: int, pitch_bytes: int, soft_lut, n_bins: int, cell: int,
                       stride: int, cell_dtype: int, cells, stream=None) -> None:
    _check("hog_cell_hist_soft", _lib.hog_cell_hist_soft(_ptr(img), W, H, channels, pitch_bytes, _ptr(soft_lut),
                                                         n_bins, cell, stride, cell_dtype, _ptr(cells),
                                                         _stream(stream)))


def hog_block_norm(cells, cell_dtype: int, ncx: int, ncy: int, n_bins: int, r: int, eps: float, blocks,
                   stream=None) -> None:
    _check("hog_block_norm", _lib.hog_block_norm(_ptr(cells), cell_dtype, ncx, ncy, n_bins, r, float(eps),
                                                 _ptr(blocks), _stream(stream)))


def hog_window_score_multi(cells, cell_dtype: int, ncx: int, ncy: int, n_bins: int, cells_x: int, cells_y: int,
                           cell: int, stride: int, w, w_dtype: int, n_filters: int, biases, scores,
                           stream=None) -> None:
    """Several filters: `w` [n_filters][K] on the device, `biases` host
    floats (a sequence), `scores` [n_filters][ny][nx] on the device."""
    b = (ctypes.c_float * n_filters)(*[float(x) for x in biases])
    _check("hog_window_score_multi", _lib.hog_window_score_multi(_ptr(cells), cell_dtype, ncx, ncy, n_bins, cells_x,
                                                                 cells_y, cell, stride, _ptr(w), w_dtype, n_filters,
                                                                 b, _ptr(scores), _stream(stream)))


def hog_detect_workspace_bytes(nx: int, ny: int) -> int:
    return _lib.hog_detect_workspace_bytes(nx, ny)


def hog_detect(scores, score_dtype: int, nx: int, ny: int, stride: int, thr: float, image: int, level: int, out,
               max_out: int, d_count, workspace, workspace_bytes: int, stream=None) -> None:
    _check("hog_detect", _lib.hog_detect(_ptr(scores), score_dtype, nx, ny, stride, float(thr), image, level,
                                         _ptr(out), max_out, _ptr(d_count), _ptr(workspace), workspace_bytes,
                                         _stream(stream)))


def hog_detect_noalloc(scores, score_dtype: int, nx: int, ny: int, stride: int, thr: float, image: int, level: int,
                       out, max_out: int, d_count, stream=None) -> None:
    """hog_detect for callers that cannot allocate scratch: the library uses
    a fixed array of its own (see include/fasthog.h for the limits)."""
    _check("hog_detect_noalloc", _lib.hog_detect_noalloc(_ptr(scores), score_dtype, nx, ny, stride, float(thr),
                                                         image, level, _ptr(out), max_out, _ptr(d_count),
                                                         _stream(stream)))


HOG_DETECT_NOALLOC_MAX_SCORES = 16384 * 2048


# ---- launch-shape knobs -------------------------------------------------------

def hog_tune_set(knob: int, value: int) -> None:
    _check("hog_tune_set", _lib.hog_tune_set(knob, value))


def hog_tune_get(knob: int) -> int:
    return _lib.hog_tune_get(knob)


# ---- batches of images and pyramid levels (include/fasthog_batch.h) ---------

def hog_batch_plan_bytes(n_items: int) -> int:
    return _lib.hog_batch_plan_bytes(n_items)


def hog_batch_plan(items, channels: int, n_bins: int, cell: int, stride: int, cells_x: int, cells_y: int):
    """Plan of a batch of HogBatchItem (a sequence).  Returns the host copy (a
    ctypes buffer; ``bytes(plan)`` are the bytes to copy to device memory)."""
    arr = (HogBatchItem * len(items))(*items)
    nbytes = _lib.hog_batch_plan_bytes(len(items))
    buf = (ctypes.c_uint64 * ((nbytes + 7) // 8))()
    _check("hog_batch_plan", _lib.hog_batch_plan(arr, len(items), channels, n_bins, cell, stride, cells_x, cells_y,
                                                 buf, nbytes))
    return buf


def hog_cell_hist_fused_batch(plan, plan_dev, lut, cell_dtype: int, stream=None) -> None:
    _check("hog_cell_hist_fused_batch", _lib.hog_cell_hist_fused_batch(_plan_ptr(plan), _ptr(plan_dev), _ptr(lut),
                                                                       cell_dtype, _stream(stream)))


def hog_window_score_batch(plan, plan_dev, cell_dtype: int, w, w_dtype: int, bias: float,
                           stream=None) -> None:
    _check("hog_window_score_batch", _lib.hog_window_score_batch(_plan_ptr(plan), _ptr(plan_dev), cell_dtype, _ptr(w),
                                                                 w_dtype, float(bias), _stream(stream)))


def hog_detect_batch_workspace_bytes(plan) -> int:
    return _lib.hog_detect_batch_workspace_bytes(_plan_ptr(plan))


def hog_detect_batch(plan, plan_dev, score_dtype: int, thr: float, out, max_out: int, d_count, item_counts,
                     workspace, workspace_bytes: int, stream=None) -> None:
    _check("hog_detect_batch", _lib.hog_detect_batch(_plan_ptr(plan), _ptr(plan_dev), score_dtype, float(thr),
                                                     _ptr(out), max_out, _ptr(d_count), _ptr(item_counts),
                                                     _ptr(workspace), workspace_bytes, _stream(stream)))


def hog_pyramid_bytes(W: int, H: int, channels: int, levels: int) -> int:
    return _lib.hog_pyramid_bytes(W, H, channels, levels)


def hog_pyramid(img, W: int, H: int, channels: int, pitch: int, levels: int, out, stream=None) -> None:
    _check("hog_pyramid", _lib.hog_pyramid(_ptr(img), W, H, channels, pitch, levels, _ptr(out), _stream(stream)))


def _plan_ptr(plan) -> int:
    return ctypes.addressof(plan)


# ---- request server (include/fasthog_server.h) -------------------------------

def hog_server_create(cfg: HogServerConfig, w_host) -> ctypes.c_void_p:
    """`w_host`: a contiguous host numpy array (or CPU tensor) of the
    weights, of the type cfg.w_dtype names.  Returns the server handle."""
    h = ctypes.c_void_p()
    _check("hog_server_create", _lib.hog_server_create(ctypes.byref(cfg), _host_ptr(w_host), ctypes.byref(h)))
    return h


def hog_server_destroy(handle) -> None:
    _check("hog_server_destroy", _lib.hog_server_destroy(handle))


def hog_server_request_bytes(handle, W: int, H: int, channels: int) -> int:
    return _lib.hog_server_request_bytes(handle, W, H, channels)


def hog_server_submit(handle, rid: int, img_host, W: int, H: int, channels: int) -> bool:
    """True if the request was admitted; `img_host` must stay alive and
    unchanged until its result has been polled."""
    ok = ctypes.c_int(0)
    _check("hog_server_submit", _lib.hog_server_submit(handle, rid, _host_ptr(img_host), W, H, channels,
                                                       ctypes.byref(ok)))
    return bool(ok.value)


def hog_server_poll(handle, out, max_out: int) -> int:
    """Fill `out` (a ctypes array of HogServerResult) and return how many."""
    n = ctypes.c_int(0)
    _check("hog_server_poll", _lib.hog_server_poll(handle, out, max_out, ctypes.byref(n)))
    return n.value


def hog_server_release(handle, token: int) -> None:
    _check("hog_server_release", _lib.hog_server_release(handle, token))


def hog_server_start(handle) -> None:
    _check("hog_server_start", _lib.hog_server_start(handle))


def hog_server_stop(handle) -> None:
    _check("hog_server_stop", _lib.hog_server_stop(handle))


def hog_server_enqueue(handle, rid: int, img_host, W: int, H: int, channels: int) -> None:
    """Queue a request for the dispatcher thread; `img_host` must stay alive
    and unchanged until its result has been collected."""
    _check("hog_server_enqueue", _lib.hog_server_enqueue(handle, rid, _host_ptr(img_host), W, H, channels))


def hog_server_collect(handle, out, max_out: int) -> int:
    """Fill `out` (a ctypes array of HogServerTimedResult) and return how many."""
    n = ctypes.c_int(0)
    _check("hog_server_collect", _lib.hog_server_collect(handle, out, max_out, ctypes.byref(n)))
    return n.value


def hog_server_clock_ns() -> int:
    return _lib.hog_server_clock_ns()


def hog_server_pauses(handle, max_n: int = 4096) -> tuple[int, list[tuple[int, int]]]:
    """(pauses since hog_server_start, [(start_ns, end_ns)] of the most recent
    up to max_n of them, oldest first)."""
    starts = (ctypes.c_int64 * max(max_n, 1))()
    ends = (ctypes.c_int64 * max(max_n, 1))()
    n = ctypes.c_int(0)
    _check("hog_server_pauses", _lib.hog_server_pauses(handle, starts, ends, max_n, ctypes.byref(n)))
    kept = min(n.value, max_n)
    return n.value, [(starts[i], ends[i]) for i in range(kept)]


def hog_server_stats(handle) -> tuple[int, int, int]:
    """(requests on the GPU, arena bytes in use, free slots)."""
    a, b, c = ctypes.c_int(0), ctypes.c_size_t(0), ctypes.c_int(0)
    _check("hog_server_stats", _lib.hog_server_stats(handle, ctypes.byref(a), ctypes.byref(b), ctypes.byref(c)))
    return a.value, b.value, c.value


# ---- shapes (host arithmetic only) --------------------------------------------

def n_positions(extent: int, box: int, stride: int) -> int:
    return 0 if extent < box else (extent - box) // stride + 1


def grid_shapes(W: int, H: int, cell: int = 8, stride: int = 8, cells_x: int = 8, cells_y: int = 16):
    """(ncx, ncy, nx, ny): cell-map and window-grid sizes of a W x H image."""
    ncx, ncy = n_positions(W, cell, stride), n_positions(H, cell, stride)
    r = cell // stride
    nx, ny = max(0, ncx - (cells_x - 1) * r), max(0, ncy - (cells_y - 1) * r)
    return ncx, ncy, nx, ny


_DET_DTYPE = None


def dets_to_numpy(raw, count: int):
    """Unpack `count` hog_det records from a uint8 tensor (host or device), a
    uint8 numpy array or a bytes object (host memory is viewed, not copied)."""
    import numpy as np

    global _DET_DTYPE
    if _DET_DTYPE is None:
        _DET_DTYPE = np.dtype([("x", "<i4"), ("y", "<i4"), ("score", "<f4"), ("image", "<i4"), ("level", "<i4")])
    dt = _DET_DTYPE
    if isinstance(raw, (bytes, bytearray)):
        return np.frombuffer(raw, dtype=np.uint8, count=count * DET_BYTES).view(dt)
    if isinstance(raw, np.ndarray):
        return raw[: count * DET_BYTES].view(dt)
    return raw[: count * DET_BYTES].cpu().numpy().view(dt)


from .pipeline import HogPipeline  # noqa: E402  (after the entry points it calls)

__all__ = [n for n in EXPORTED] + ["HogPipeline", "HogError", "grid_shapes", "n_positions", "dets_to_numpy"]
