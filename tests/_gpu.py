"""Helpers for the GPU parity tests: move numpy arrays through one C-ABI call
at a time.  The expected values always come from the oracle."""

import numpy as np
import torch

import paper_1703_06256_gb300 as fh


def dev(a: np.ndarray) -> torch.Tensor:
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def gpu_lut(nb: int) -> torch.Tensor:
    lut = torch.empty(fh.HOG_LUT_BYTES, dtype=torch.uint8, device="cuda")
    fh.hog_build_lut(nb, lut)
    return lut


def gpu_bins(img: np.ndarray, nb: int, lut=None, pitch_pad: int = 0, offset: int = 0) -> np.ndarray:
    """Bin map of a (H, W) or (H, W, 3) image; pitch_pad adds bytes after
    every row, offset shifts the image start (unaligned base)."""
    H, W = img.shape[:2]
    ch = 1 if img.ndim == 2 else 3
    pitch = W * ch + pitch_pad
    host = np.zeros(offset + H * pitch + 16, np.uint8)
    rows = host[offset: offset + H * pitch].reshape(H, pitch)
    rows[:, : W * ch] = img.reshape(H, W * ch)
    d = dev(host)
    bins = torch.empty(H * W, dtype=torch.uint8, device="cuda")
    lut = gpu_lut(nb) if lut is None else lut
    fh.hog_bin_map(d.data_ptr() + offset, W, H, ch, pitch, lut, nb, bins)
    return bins.cpu().numpy().reshape(H, W)


def gpu_integral(bins: np.ndarray, nb: int, ii_dtype=fh.HOG_I32, ws=None) -> np.ndarray:
    """`ws`: a zero-filled workspace to reuse (at least
    hog_integral_workspace_bytes), else a fresh one."""
    H, W = bins.shape
    b = dev(bins.reshape(-1))
    ws_bytes = fh.hog_integral_workspace_bytes(W, H, nb)
    if ws is None:
        ws = torch.zeros(ws_bytes, dtype=torch.uint8, device="cuda")  # zero-filled before its first use
    else:
        assert ws.numel() >= ws_bytes
        ws_bytes = ws.numel()
    # canaries around the output catch writes past either end
    pad = 64
    t = torch.int32 if ii_dtype == fh.HOG_I32 else torch.int16
    buf = torch.full((nb * H * W + 2 * pad,), 0x5A5A if t == torch.int16 else 0x5A5A5A5A, dtype=t, device="cuda")
    out = buf[pad: pad + nb * H * W]
    fh.hog_integral(b, W, H, nb, ii_dtype, out, ws, ws_bytes)
    host = buf.cpu().numpy()
    assert np.all(host[:pad] == host[0]) and np.all(host[-pad:] == host[0]), "write outside the ii planes"
    a = host[pad: pad + nb * H * W].reshape(nb, H, W)
    return a.view(np.uint16) if ii_dtype == fh.HOG_U16 else a


def gpu_cells(ii: np.ndarray, nb: int, cell: int, stride: int, ii_dtype=fh.HOG_I32, cell_dtype=fh.HOG_I32):
    _, H, W = ii.shape
    ncx, ncy = fh.n_positions(W, cell, stride), fh.n_positions(H, cell, stride)
    src = ii.astype(np.int32) if ii_dtype == fh.HOG_I32 else ii.astype(np.uint16).view(np.int16)
    d = dev(src.reshape(-1))
    n = max(ncx * ncy * nb, 1)
    out = torch.zeros(n, dtype=fh.TORCH_DTYPE[cell_dtype], device="cuda")
    fh.hog_cell_hist(d, W, H, nb, ii_dtype, cell, stride, cell_dtype, out)
    return out.float().cpu().numpy()[: ncx * ncy * nb].reshape(ncy, ncx, nb)


def gpu_scores(cells: np.ndarray, w: np.ndarray, w_dtype: int, bias: float, cell: int = 8, stride: int = 8,
               cells_x: int = 8, cells_y: int = 16, cell_dtype=fh.HOG_I32):
    ncy, ncx, nb = cells.shape
    r = cell // stride
    nx, ny = ncx - (cells_x - 1) * r, ncy - (cells_y - 1) * r
    if cell_dtype == fh.HOG_I32:
        c = dev(cells.astype(np.int32).reshape(-1))
    elif cell_dtype == fh.HOG_F32:
        c = dev(cells.astype(np.float32).reshape(-1))
    else:
        c = torch.from_numpy(cells.astype(np.float32).reshape(-1)).to(torch.bfloat16).cuda()
    if w_dtype == fh.HOG_F32:
        wd = dev(w.astype(np.float32))
    elif w_dtype == fh.HOG_BF16:
        wd = torch.from_numpy(w.astype(np.float32)).to(torch.bfloat16).cuda()
    else:
        wd = dev(w.astype(np.int8))
    out_t = torch.int32 if w_dtype == fh.HOG_I8 else torch.float32
    out = torch.zeros(max(nx * ny, 1), dtype=out_t, device="cuda")
    fh.hog_window_score(c, cell_dtype, ncx, ncy, nb, cells_x, cells_y, cell, stride, wd, w_dtype, bias, out)
    return out.cpu().numpy()[: max(nx, 0) * max(ny, 0)].reshape(max(ny, 0), max(nx, 0))


def gpu_detect(scores: np.ndarray, stride: int, thr: float, max_out: int | None = None, image=0, level=0):
    ny, nx = scores.shape
    dtype = fh.HOG_I32 if scores.dtype == np.int32 else fh.HOG_F32
    s = dev(scores.astype(np.int32 if dtype == fh.HOG_I32 else np.float32).reshape(-1)) if scores.size else \
        torch.zeros(1, dtype=torch.float32, device="cuda")
    cap = scores.size if max_out is None else max_out
    out = torch.zeros(max(cap, 1) * fh.DET_BYTES, dtype=torch.uint8, device="cuda")
    cnt = torch.full((1,), -7, dtype=torch.int32, device="cuda")
    ws_b = fh.hog_detect_workspace_bytes(nx, ny)
    ws = torch.zeros(ws_b, dtype=torch.uint8, device="cuda")  # zero-filled before its first use
    fh.hog_detect(s, dtype, nx, ny, stride, thr, image, level, out, cap, cnt, ws, ws_b)
    n = int(cnt.item())
    return fh.dets_to_numpy(out.cpu(), min(n, cap)), n


def score_tolerance(cells: np.ndarray, w: np.ndarray, bias: float, cell=8, stride=8, cells_x=8, cells_y=16):
    """1e-5 * (sum_k |w_k| h_k + |bias|) per window: the FP32-path bound."""
    import oracle

    return 1e-5 * (oracle.window_score(np.abs(cells), np.abs(np.asarray(w, np.float64)), abs(bias), cells_x,
                                       cells_y, cell, stride))


def check_detections(det, n, S_gpu, S64, tol, thr, stride):
    """The list must be exactly the row-major compaction of the GPU's own
    scores (same precision decides), and may differ from the FP64 decision
    only for windows whose FP64 score lies within `tol` of the threshold.
    Returns the number of such near-threshold windows."""
    ys, xs = np.nonzero(S_gpu >= np.float32(thr))
    assert n == len(xs)
    assert np.array_equal(det["x"], xs * stride) and np.array_equal(det["y"], ys * stride)
    assert np.array_equal(det["score"], S_gpu[ys, xs])
    near = np.abs(S64 - thr) <= tol
    assert np.array_equal((S_gpu >= np.float32(thr))[~near], (S64 >= thr)[~near])
    return int(near.sum())
