"""Pins for the oracle's window score and detection list (Sections 1 and 4:
objectness score per position as an inner product, then a threshold)."""

import json
import os

import numpy as np
import pytest

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def test_hand_worked_window(oracle_mod):
    g = json.load(open(os.path.join(GOLDEN, "hand_5x5.json")))
    bins = np.array(g["bins_rows_y"], np.uint8)
    wg = g["window"]
    K = wg["cells_x"] * wg["cells_y"] * 8
    w = np.arange(1, K + 1, dtype=np.float64)
    ii = oracle_mod.integral(bins, 8)
    cells = oracle_mod.cell_hist_ii(ii, 8, cell=wg["cell"], stride=wg["stride"])
    S = oracle_mod.window_score(cells, w, 0.0, wg["cells_x"], wg["cells_y"], wg["cell"], wg["stride"])
    assert S[0, 0] == wg["score_at_0_0"]
    S2 = oracle_mod.window_score_from_bins(bins, 8, w, 0.0, wg["cells_x"], wg["cells_y"],
                                           wg["cell"], wg["stride"])
    assert np.array_equal(S, S2)


@pytest.mark.parametrize("stride", [8, 4, 2])
def test_cell_route_equals_pixel_route(oracle_mod, stride):
    rng = np.random.default_rng(stride)
    img = rng.integers(0, 256, size=(150, 90), dtype=np.uint8)
    bins = oracle_mod.bin_map(img, 8)
    w = rng.normal(0, 0.01, 1024)
    cells = oracle_mod.cell_hist_ii(oracle_mod.integral(bins, 8), 8, 8, stride)
    S = oracle_mod.window_score(cells, w, 0.25, stride=stride)
    S2 = oracle_mod.window_score_from_bins(bins, 8, w, 0.25, stride=stride)
    assert S.shape == ((150 - 128) // stride + 1, (90 - 64) // stride + 1)
    assert np.array_equal(S, S2)


def test_unit_weights_count_binned_pixels(oracle_mod):
    """All-ones weights: the score is the number of binned pixels in the window.
    On a +x ramp every non-border pixel is binned (closed form)."""
    H, W = 136, 72
    img = (3 * np.mgrid[0:H, 0:W][1]).astype(np.uint8)
    bins = oracle_mod.bin_map(img, 8)
    cells = oracle_mod.cell_hist_direct(bins, 8, 8, 4)
    S = oracle_mod.window_score(cells, np.ones(1024), 0.0, stride=4)
    for py in range(S.shape[0]):
        for px in range(S.shape[1]):
            x0, y0 = 4 * px, 4 * py
            nxi = 64 - (x0 == 0) - (x0 + 64 == W)
            nyi = 128 - (y0 == 0) - (y0 + 128 == H)
            assert S[py, px] == nxi * nyi
    # one-hot weight on (cell row 3, cell column 5, bin 0): the count in that cell
    w = np.zeros(1024)
    w[(3 * 8 + 5) * 8 + 0] = 1.0
    S = oracle_mod.window_score(cells, w, 0.0, stride=4)
    assert np.all(S == 64)


def test_linearity_and_bias(oracle_mod):
    rng = np.random.default_rng(3)
    img = rng.integers(0, 256, size=(140, 80), dtype=np.uint8)
    cells = oracle_mod.cell_hist_direct(oracle_mod.bin_map(img, 8), 8, 8, 4)
    w1 = rng.integers(-127, 128, 1024).astype(np.float64)
    w2 = rng.integers(-127, 128, 1024).astype(np.float64)
    s1 = oracle_mod.window_score(cells, w1, 0.0, stride=4)
    s2 = oracle_mod.window_score(cells, w2, 0.0, stride=4)
    s12 = oracle_mod.window_score(cells, w1 + w2, 7.0, stride=4)
    assert np.array_equal(s1 + s2 + 7.0, s12)  # integers: exact in FP64


def test_detect_list(oracle_mod):
    S = np.array([[0.1, 0.5, 0.49999], [2.0, -1.0, 0.5]])
    xs, ys, sc = oracle_mod.detect(S, 4, 0.5)
    assert xs.tolist() == [4, 0, 8] and ys.tolist() == [0, 4, 4]
    assert sc.tolist() == [0.5, 2.0, 0.5]
    xs, ys, sc = oracle_mod.detect(np.zeros((0, 0)), 4, 0.5)
    assert len(xs) == 0


def test_decimate(oracle_mod):
    img = np.arange(7 * 9 * 3, dtype=np.uint8).reshape(7, 9, 3)
    d = oracle_mod.decimate(img)
    assert d.shape == (3, 4, 3)
    assert np.array_equal(d, img[0:6:2, 0:8:2])


def test_multi_filter_linearity_and_order(oracle_mod):
    """Several filters: filter f of the result is filter f's own score with
    bias f.  Checked by exact integer linearity (f2 = 3 f0 - 2 f1), one-hot
    filters that read single cell counts, and the all-ones filter, which
    counts the binned pixels of the window (closed form)."""
    rng = np.random.default_rng(31)
    img = rng.integers(0, 256, size=(200, 120), dtype=np.uint8)
    bins = oracle_mod.bin_map(img, 8)
    cells = oracle_mod.cell_hist_direct(bins, 8, 8, 4)
    K = 8 * 16 * 8
    w0 = rng.integers(-5, 6, K).astype(np.float64)
    w1 = rng.integers(-5, 6, K).astype(np.float64)
    onehot = np.zeros(K)
    onehot[(3 * 8 + 5) * 8 + 6] = 1.0  # cell (cx, cy) = (5, 3), bin 6
    W = np.stack([w0, w1, 3 * w0 - 2 * w1, onehot, np.ones(K)])
    B = np.array([0.5, -1.0, 3.5, 0.0, 0.0])
    S = oracle_mod.window_score_multi(cells, W, B, stride=4)
    assert S.shape[0] == 5
    assert np.array_equal(S[2] - 3.5, 3 * (S[0] - 0.5) - 2 * (S[1] + 1.0))
    ny, nx = S.shape[1:]
    assert np.array_equal(S[3], cells[3 * 2: 3 * 2 + ny, 5 * 2: 5 * 2 + nx, 6].astype(np.float64))
    for py in (0, ny // 2, ny - 1):
        for px in (0, nx - 1):
            win = bins[py * 4: py * 4 + 128, px * 4: px * 4 + 64]
            assert S[4, py, px] == np.count_nonzero(win < 8)


def test_block_norm_from_pixels(oracle_mod):
    """Overlapping 2x2-cell blocks counted straight from the bin map (16x16
    pixels at the scan stride, four 8x8 quadrants) and L2-normalised equal the
    oracle's blocks built from the cell map."""
    rng = np.random.default_rng(41)
    img = rng.integers(0, 256, size=(90, 70, 3), dtype=np.uint8)
    bins = oracle_mod.bin_map(img, 8)
    cells = oracle_mod.cell_hist_direct(bins, 8, 8, 4)
    eps = 0.7
    B = oracle_mod.block_norm(cells, 2, eps)
    nby, nbx, k = B.shape
    assert k == 32 and (nby, nbx) == (cells.shape[0] - 2, cells.shape[1] - 2)
    for j in range(0, nby, 3):
        for i in range(0, nbx, 2):
            v = []
            for q in range(4):
                y0, x0 = 4 * j + 8 * (q >> 1), 4 * i + 8 * (q & 1)
                blk = bins[y0: y0 + 8, x0: x0 + 8]
                v += [np.count_nonzero(blk == b) for b in range(8)]
            v = np.array(v, np.float64)
            assert np.allclose(B[j, i], v / np.sqrt(v @ v + eps * eps), rtol=0, atol=1e-15)


def test_block_norm_closed_forms(oracle_mod):
    """A ramp puts every interior pixel in one bin: each quadrant of an
    interior block holds 64 counts of that bin, so the block is
    64 / sqrt(4 * 64^2 + eps^2) at the four entries of that bin and 0
    elsewhere; with eps = 0 every non-empty block has unit norm, and a block
    without binned pixels is all zero."""
    _, xx = np.mgrid[0:64, 0:80]
    img = (3 * xx).astype(np.uint8)  # (dx, dy) = (6, 0) inside: bin 0
    bins = oracle_mod.bin_map(img, 8)
    cells = oracle_mod.cell_hist_direct(bins, 8, 8, 4)
    B = oracle_mod.block_norm(cells, 2, 2.0)
    v = B[5, 5].reshape(4, 8)
    want = 64 / np.sqrt(4 * 64.0 ** 2 + 4.0)
    assert np.allclose(v[:, 0], want, atol=1e-15) and np.all(v[:, 1:] == 0)
    B0 = oracle_mod.block_norm(cells, 2, 0.0)
    n = np.sqrt((B0 ** 2).sum(axis=2))
    assert np.allclose(n[n > 0], 1.0, atol=1e-15)
    empty = np.zeros_like(cells)
    assert np.all(oracle_mod.block_norm(empty, 2, 0.0) == 0)


def test_block_window_score_indexing(oracle_mod):
    """A one-hot weight on block (bx, by), entry k picks that block entry
    of every window; the bias is added once."""
    rng = np.random.default_rng(42)
    B = rng.random((50, 30, 32))
    w = np.zeros((15, 7, 32))
    w[11, 4, 19] = 1.0
    S = oracle_mod.block_window_score(B, w, 0.25, r=2)
    ny, nx = S.shape
    assert (ny, nx) == (50 - 28, 30 - 12)
    assert np.array_equal(S, B[22: 22 + ny, 8: 8 + nx, 19] + 0.25)
