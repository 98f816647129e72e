"""CPU oracle for the fast-HOG detection path (Huang & Huang, "A Fast HOG
Descriptor Using Lookup Table and Integral Image").

TEST INFRASTRUCTURE ONLY.  Only the test-suite, ``__graft_entry__.smoke()`` and
the CPU-baseline leg of ``bench.py`` may import this package.  The product path
(the CUDA library and its Python binding) never imports, links or runs it, and
this package never imports the product path: the two share no code.  The only
module both sides use is ``workloads`` (seeded input generators, none of the
method's arithmetic).

The arithmetic lives in ``fasthog_oracle.c`` (plain C, FP64, one function per
step of the paper, each citing its section and equation).  This module builds
it with gcc and marshals numpy arrays into it; it adds no arithmetic of its own
apart from exact dtype widening of the weights.
"""

from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "fasthog_oracle.c")
_BUILD_DIR = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD_DIR, "liboracle.so")
_lock = threading.Lock()
_lib = None

NO_BIN = 0xFF
LUT_SIDE = 511
DMAX = 255


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (FP contraction off, so x86 and Arm agree)."""
    os.makedirs(_BUILD_DIR, exist_ok=True)
    stale = (not os.path.exists(_LIB_PATH)) or os.path.getmtime(_LIB_PATH) < os.path.getmtime(_SRC)
    if force or stale:
        tmp = _LIB_PATH + f".tmp{os.getpid()}"
        cmd = ["gcc", "-std=c99", "-O2", "-ffp-contract=off", "-fno-fast-math", "-D_DEFAULT_SOURCE",
               "-shared", "-fPIC", "-o", tmp, _SRC, "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    with _lock:
        if _lib is None:
            # ORACLE_LIB names another build of fasthog_oracle.c (the mutation tests load
            # deliberately broken copies this way); by default the one built here
            path = os.environ.get("ORACLE_LIB") or build()
            lib = ctypes.CDLL(path)
            P = ctypes.c_void_p
            I = ctypes.c_int
            L = ctypes.c_long
            D = ctypes.c_double
            sig = {
                "oracle_min_margin": (D, []),
                "oracle_margin_violation": (I, []),
                "oracle_reset_margin": (None, []),
                "oracle_sector_bin": (I, [I, I, I]),
                "oracle_lut": (I, [I, P]),
                "oracle_bin_map": (I, [P, I, I, I, L, I, P]),
                "oracle_integral_brute": (I, [P, I, I, I, P]),
                "oracle_integral": (I, [P, I, I, I, P]),
                "oracle_cell_hist_direct": (I, [P, I, I, I, I, I, P]),
                "oracle_cell_hist_ii": (I, [P, I, I, I, I, I, P]),
                "oracle_window_score": (I, [P, I, I, I, I, I, I, I, P, D, P]),
                "oracle_window_score_from_bins": (I, [P, I, I, I, I, I, I, I, P, D, P]),
                "oracle_detect": (L, [P, I, I, I, D, P, P, P, L]),
                "oracle_decimate": (I, [P, I, I, I, L, P]),
                "oracle_block_norm": (I, [P, I, I, I, I, D, P]),
                "oracle_soft_lut": (I, [I, I, P, P]),
                "oracle_soft_votes": (I, [P, I, I, I, L, I, I, P]),
            }
            for name, (res, args) in sig.items():
                fn = getattr(lib, name)
                fn.restype = res
                fn.argtypes = args
            _lib = lib
    return _lib


def _ptr(a: np.ndarray):
    assert a.flags["C_CONTIGUOUS"]
    return a.ctypes.data_as(ctypes.c_void_p)


def _check(rc, what):
    if rc != 0:
        raise ValueError(f"oracle {what} rejected its arguments (rc={rc})")


def n_positions(extent: int, box: int, stride: int) -> int:
    """Positions 0, s, 2s, ... of a box of `box` pixels inside `extent` pixels."""
    return 0 if extent < box else (extent - box) // stride + 1


# --- Section 2 --------------------------------------------------------------

def min_margin() -> float:
    return _load().oracle_min_margin()


def margin_violation() -> bool:
    return bool(_load().oracle_margin_violation())


def reset_margin() -> None:
    _load().oracle_reset_margin()


def sector_bin(dx: int, dy: int, n_bins: int) -> int:
    """Orientation bin of one gradient (0xFF for dx = dy = 0)."""
    return _load().oracle_sector_bin(int(dx), int(dy), int(n_bins))


def lut(n_bins: int) -> np.ndarray:
    """The 511 x 511 table, flat, index (dy + 255) * 511 + (dx + 255)."""
    out = np.empty(LUT_SIDE * LUT_SIDE, np.uint8)
    _check(_load().oracle_lut(int(n_bins), _ptr(out)), "lut")
    return out


def bin_map(img: np.ndarray, n_bins: int) -> np.ndarray:
    """Eq. 1 + sector binning.  img: (H, W) gray or (H, W, 3) RGB uint8."""
    img = np.ascontiguousarray(img, dtype=np.uint8)
    H, W = img.shape[:2]
    ch = 1 if img.ndim == 2 else img.shape[2]
    out = np.empty((H, W), np.uint8)
    _check(_load().oracle_bin_map(_ptr(img), W, H, ch, W * ch, int(n_bins), _ptr(out)), "bin_map")
    return out


# --- Section 3.2 -------------------------------------------------------------

def integral_brute(bins: np.ndarray, n_bins: int) -> np.ndarray:
    bins = np.ascontiguousarray(bins, dtype=np.uint8)
    H, W = bins.shape
    out = np.empty((n_bins, H, W), np.int32)
    _check(_load().oracle_integral_brute(_ptr(bins), W, H, int(n_bins), _ptr(out)), "integral_brute")
    return out


def integral(bins: np.ndarray, n_bins: int) -> np.ndarray:
    bins = np.ascontiguousarray(bins, dtype=np.uint8)
    H, W = bins.shape
    out = np.empty((n_bins, H, W), np.int32)
    _check(_load().oracle_integral(_ptr(bins), W, H, int(n_bins), _ptr(out)), "integral")
    return out


# --- Section 3.3 -------------------------------------------------------------

def cell_hist_direct(bins: np.ndarray, n_bins: int, cell: int = 8, stride: int = 8) -> np.ndarray:
    bins = np.ascontiguousarray(bins, dtype=np.uint8)
    H, W = bins.shape
    ncx, ncy = n_positions(W, cell, stride), n_positions(H, cell, stride)
    out = np.zeros((ncy, ncx, n_bins), np.int32)
    _check(_load().oracle_cell_hist_direct(_ptr(bins), W, H, int(n_bins), cell, stride, _ptr(out)),
           "cell_hist_direct")
    return out


def cell_hist_ii(ii: np.ndarray, n_bins: int, cell: int = 8, stride: int = 8) -> np.ndarray:
    ii = np.ascontiguousarray(ii, dtype=np.int32)
    _, H, W = ii.shape
    ncx, ncy = n_positions(W, cell, stride), n_positions(H, cell, stride)
    out = np.zeros((ncy, ncx, n_bins), np.int32)
    _check(_load().oracle_cell_hist_ii(_ptr(ii), W, H, int(n_bins), cell, stride, _ptr(out)),
           "cell_hist_ii")
    return out


# --- Sections 1 and 4 ---------------------------------------------------------

def window_score_multi(cells: np.ndarray, w: np.ndarray, biases, cells_x: int = 8, cells_y: int = 16,
                       cell: int = 8, stride: int = 8) -> np.ndarray:
    """Several independent linear filters scored over the same windows (the
    paper scores one): `w` is [F][cells_y * cells_x * nb], `biases` [F];
    returns [F][ny][nx], filter f being window_score with w[f], bias f."""
    w = np.asarray(w)
    return np.stack([window_score(cells, w[f], float(biases[f]), cells_x, cells_y, cell, stride)
                     for f in range(w.shape[0])])


def window_score(cells: np.ndarray, w: np.ndarray, bias: float = 0.0, cells_x: int = 8,
                 cells_y: int = 16, cell: int = 8, stride: int = 8) -> np.ndarray:
    """FP64 score map S[ny][nx].  `w` is widened exactly to float64."""
    cells = np.ascontiguousarray(cells, dtype=np.int32)
    ncy, ncx, nb = cells.shape
    w64 = np.ascontiguousarray(np.asarray(w, dtype=np.float64).reshape(-1))
    assert w64.size == cells_x * cells_y * nb
    r = cell // stride
    nx, ny = ncx - (cells_x - 1) * r, ncy - (cells_y - 1) * r
    S = np.zeros((max(ny, 0), max(nx, 0)), np.float64)
    _check(_load().oracle_window_score(_ptr(cells), ncx, ncy, nb, cells_x, cells_y, cell, stride,
                                       _ptr(w64), float(bias), _ptr(S)), "window_score")
    return S


def window_score_from_bins(bins: np.ndarray, n_bins: int, w: np.ndarray, bias: float = 0.0,
                           cells_x: int = 8, cells_y: int = 16, cell: int = 8,
                           stride: int = 8) -> np.ndarray:
    bins = np.ascontiguousarray(bins, dtype=np.uint8)
    H, W = bins.shape
    w64 = np.ascontiguousarray(np.asarray(w, dtype=np.float64).reshape(-1))
    nx = n_positions(W, cells_x * cell, stride)
    ny = n_positions(H, cells_y * cell, stride)
    S = np.zeros((ny, nx), np.float64)
    _check(_load().oracle_window_score_from_bins(_ptr(bins), W, H, int(n_bins), cells_x, cells_y,
                                                 cell, stride, _ptr(w64), float(bias), _ptr(S)),
           "window_score_from_bins")
    return S


def detect(S: np.ndarray, stride: int, thr: float):
    """Row-major list of windows with score >= thr: (xs, ys, scores)."""
    S = np.ascontiguousarray(S, dtype=np.float64)
    ny, nx = S.shape if S.size else (0, 0)
    cap = max(S.size, 1)
    xs = np.empty(cap, np.int32)
    ys = np.empty(cap, np.int32)
    sc = np.empty(cap, np.float64)
    n = _load().oracle_detect(_ptr(S), nx, ny, int(stride), float(thr), _ptr(xs), _ptr(ys),
                              _ptr(sc), cap)
    return xs[:n].copy(), ys[:n].copy(), sc[:n].copy()


SOFT_Q = 64  # vote units per pixel


def soft_lut(nb: int, q: int = SOFT_Q):
    """Soft-vote table [511][511] uint16 (k0 | a << 8, 0xFFFF at (0, 0)) and
    the smallest distance of q * alpha from a rounding tie over the table."""
    out = np.empty(511 * 511, np.uint16)
    m = ctypes.c_double(0.0)
    _check(_load().oracle_soft_lut(nb, q, _ptr(out), ctypes.addressof(m)), "soft_lut")
    return out.reshape(511, 511), m.value


def soft_votes(img: np.ndarray, nb: int, q: int = SOFT_Q) -> np.ndarray:
    """Per-pixel two-bin votes [H][W][nb] int32 (q units per voting pixel)."""
    img = np.ascontiguousarray(img, dtype=np.uint8)
    H, W = img.shape[:2]
    ch = 1 if img.ndim == 2 else img.shape[2]
    out = np.empty((H, W, nb), np.int32)
    _check(_load().oracle_soft_votes(_ptr(img), W, H, ch, W * ch, nb, q, _ptr(out)), "soft_votes")
    return out


def soft_cells(img: np.ndarray, nb: int, cell: int = 8, stride: int = 8, q: int = SOFT_Q) -> np.ndarray:
    """Soft-vote cell histograms [ncy][ncx][nb] by direct summation of each
    cell's pixel votes."""
    v = soft_votes(img, nb, q)
    H, W = v.shape[:2]
    ncx = 0 if W < cell else (W - cell) // stride + 1
    ncy = 0 if H < cell else (H - cell) // stride + 1
    out = np.zeros((ncy, ncx, nb), np.int64)
    for j in range(ncy):
        for i in range(ncx):
            out[j, i] = v[j * stride: j * stride + cell, i * stride: i * stride + cell].sum(axis=(0, 1))
    return out


def block_norm(cells: np.ndarray, r: int, eps: float) -> np.ndarray:
    """Overlapping 2x2-cell blocks, L2-normalised: [ncy-r][ncx-r][4 nb] FP64
    (quadrant q = 2 cy + cx of the block holds cell (i + cx r, j + cy r))."""
    cells = np.ascontiguousarray(cells, dtype=np.int32)
    ncy, ncx, nb = cells.shape
    out = np.zeros((max(ncy - r, 0), max(ncx - r, 0), 4 * nb), np.float64)
    _check(_load().oracle_block_norm(_ptr(cells), ncx, ncy, nb, r, float(eps), _ptr(out)), "block_norm")
    return out


def block_window_score(blocks: np.ndarray, w: np.ndarray, bias: float = 0.0, blocks_x: int = 7,
                       blocks_y: int = 15, r: int = 2) -> np.ndarray:
    """Linear score over windows of blocks_x x blocks_y blocks, block step r
    positions (one cell): the window score of the block map with 4 nb
    'bins' per entry, in FP64."""
    blocks = np.ascontiguousarray(blocks, dtype=np.float64)
    nby, nbx, k = blocks.shape
    w64 = np.asarray(w, dtype=np.float64).reshape(blocks_y, blocks_x, k)
    ny, nx = nby - (blocks_y - 1) * r, nbx - (blocks_x - 1) * r
    S = np.full((max(ny, 0), max(nx, 0)), float(bias))
    for by in range(blocks_y):
        for bx in range(blocks_x):
            S += blocks[by * r: by * r + ny, bx * r: bx * r + nx, :] @ w64[by, bx]
    return S


def decimate(img: np.ndarray) -> np.ndarray:
    """2:1 decimation of a (H, W) or (H, W, C) uint8 image."""
    img = np.ascontiguousarray(img, dtype=np.uint8)
    H, W = img.shape[:2]
    ch = 1 if img.ndim == 2 else img.shape[2]
    shape = (H // 2, W // 2) if img.ndim == 2 else (H // 2, W // 2, ch)
    out = np.empty(shape, np.uint8)
    _check(_load().oracle_decimate(_ptr(img), W, H, ch, W * ch, _ptr(out)), "decimate")
    return out


def pipeline(img: np.ndarray, n_bins: int, w: np.ndarray, bias: float = 0.0, stride: int = 8,
             thr: float | None = None, cell: int = 8, cells_x: int = 8, cells_y: int = 16):
    """Whole path, in the paper's order: bins -> ii -> cell histograms (Eq. 6)
    -> scores -> detections.  Returns a dict of every intermediate."""
    bins = bin_map(img, n_bins)
    ii = integral(bins, n_bins)
    cells = cell_hist_ii(ii, n_bins, cell, stride)
    S = window_score(cells, w, bias, cells_x, cells_y, cell, stride)
    out = {"bins": bins, "ii": ii, "cells": cells, "scores": S}
    if thr is not None:
        out["detections"] = detect(S, stride, thr)
    return out
