"""Pins for the oracle's per-bin integral images (Section 3.2, Eq. 4-5) and
box sums (Section 3.1 Eq. 3, Section 3.3 Eq. 6)."""

import json
import os

import numpy as np
import pytest

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def random_bins(H, W, nb, seed, p_none=0.2):
    rng = np.random.default_rng(seed)
    b = rng.integers(0, nb, size=(H, W)).astype(np.uint8)
    b[rng.random((H, W)) < p_none] = 255
    return b


@pytest.mark.parametrize("H,W", [(1, 1), (2, 3), (3, 3), (7, 5), (17, 33), (4, 1), (1, 6)])
def test_running_sums_equal_brute_force(oracle_mod, H, W):
    for nb, seed in [(8, 1), (3, 2), (16, 3)]:
        bins = random_bins(H, W, nb, seed)
        assert np.array_equal(oracle_mod.integral(bins, nb), oracle_mod.integral_brute(bins, nb))
    const = np.full((H, W), 2, np.uint8)
    ii = oracle_mod.integral(const, 4)
    yy, xx = np.mgrid[0:H, 0:W]
    assert np.array_equal(ii[2], (yy + 1) * (xx + 1))
    assert not ii[[0, 1, 3]].any()


def test_library_cumsum(oracle_mod):
    """Eq. 5 equals two library prefix sums of the one-hot images (Eq. 4)."""
    bins = random_bins(61, 87, 8, 11)
    onehot = (bins[None] == np.arange(8)[:, None, None]).astype(np.int64)
    ref = np.cumsum(np.cumsum(onehot, axis=1), axis=2)
    assert np.array_equal(oracle_mod.integral(bins, 8), ref)


def test_invariants(oracle_mod):
    bins = random_bins(45, 70, 8, 4)
    ii = oracle_mod.integral(bins, 8)
    assert ii[:, -1, -1].sum() == np.count_nonzero(bins != 255)
    assert np.all(np.diff(ii, axis=1) >= 0) and np.all(np.diff(ii, axis=2) >= 0)
    # with the border unbinned (as the bin map makes it) row 0 and column 0 are zero
    bins[0, :] = 255
    bins[:, 0] = 255
    ii = oracle_mod.integral(bins, 8)
    assert not ii[:, 0, :].any() and not ii[:, :, 0].any()


def test_hand_worked_5x5(oracle_mod):
    g = json.load(open(os.path.join(GOLDEN, "hand_5x5.json")))
    bins = np.array(g["bins_rows_y"], np.uint8)
    ii = oracle_mod.integral(bins, 8)
    for b, plane in g["ii"].items():
        assert ii[int(b)].tolist() == plane, b
    bx = g["box_eq3"]
    # a one-cell histogram whose cell is exactly that box
    cells = oracle_mod.cell_hist_ii(ii[:, :bx["y1"] + 1, :bx["x1"] + 1], 8,
                                    cell=bx["x1"] - bx["x0"] + 1, stride=1)
    assert cells[bx["y0"], bx["x0"], bx["bin"]] == bx["value"]


@pytest.mark.parametrize("stride", [1, 2, 4, 8])
def test_eq6_box_sums_equal_direct_counts(oracle_mod, stride):
    for H, W, seed in [(8, 8, 1), (37, 53, 2), (64, 96, 3)]:
        bins = random_bins(H, W, 8, seed)
        ii = oracle_mod.integral(bins, 8)
        a = oracle_mod.cell_hist_ii(ii, 8, cell=8, stride=stride)
        b = oracle_mod.cell_hist_direct(bins, 8, cell=8, stride=stride)
        assert a.shape == b.shape and np.array_equal(a, b)
        assert np.all(a.sum(axis=2) <= 64)


def test_cell_counts_closed_form(oracle_mod):
    """+x ramp: every interior pixel is bin 0, the border has no bin, so a cell
    holds 64 minus the border pixels it covers, all in bin 0."""
    H, W = 40, 48
    img = (3 * np.mgrid[0:H, 0:W][1]).astype(np.uint8)
    bins = oracle_mod.bin_map(img, 8)
    cells = oracle_mod.cell_hist_direct(bins, 8, cell=8, stride=4)
    ncy, ncx = cells.shape[:2]
    for j in range(ncy):
        for i in range(ncx):
            x0, y0 = 4 * i, 4 * j
            nxi = 8 - (x0 == 0) - (x0 + 8 == W)
            nyi = 8 - (y0 == 0) - (y0 + 8 == H)
            assert cells[j, i, 0] == nxi * nyi
            assert not cells[j, i, 1:].any()
