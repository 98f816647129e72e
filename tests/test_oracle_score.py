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
