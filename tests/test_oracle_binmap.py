"""Pins for the oracle's oriented-gradient map (Section 2, Eq. 1).

Closed-form images whose every gradient is known by hand: ramps, a single
bright pixel, constant images, and colour images built so that a chosen
channel wins (or ties)."""

import json
import os

import numpy as np
import pytest

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")
NO = 255


def interior(a):
    return a[1:-1, 1:-1]


def border_mask(H, W):
    m = np.ones((H, W), bool)
    m[1:-1, 1:-1] = False
    return m


@pytest.mark.parametrize("nb", [4, 8, 16])
def test_ramps(oracle_mod, nb):
    H, W = 13, 17
    yy, xx = np.mgrid[0:H, 0:W]
    cases = [
        (3 * xx, 0),                 # +x: phi = 0
        (200 - 3 * xx, nb // 2),     # -x: phi = pi
        (5 * yy, nb // 4),           # +y (down): phi = pi/2
        (200 - 5 * yy, 3 * nb // 4),  # -y: phi = 3pi/2
    ]
    if nb % 8 == 0:
        cases.append((4 * xx + 4 * yy, nb // 8))  # phi = pi/4
    for img, expect in cases:
        bins = oracle_mod.bin_map(img.astype(np.uint8), nb)
        assert np.all(interior(bins) == expect)
        assert np.all(bins[border_mask(H, W)] == NO)


def test_single_bright_pixel(oracle_mod):
    H, W, x0, y0 = 9, 11, 5, 4
    img = np.zeros((H, W), np.uint8)
    img[y0, x0] = 200
    bins = oracle_mod.bin_map(img, 8)
    expect = np.full((H, W), NO, np.uint8)
    expect[y0, x0 - 1] = 0   # dx = +200
    expect[y0, x0 + 1] = 4   # dx = -200
    expect[y0 - 1, x0] = 2   # dy = +200 (the pixel below is brighter)
    expect[y0 + 1, x0] = 6   # dy = -200
    assert np.array_equal(bins, expect)


def test_constant_and_tiny(oracle_mod):
    for H, W in [(1, 1), (2, 2), (1, 9), (9, 1), (5, 5)]:
        img = np.full((H, W), 77, np.uint8)
        assert np.all(oracle_mod.bin_map(img, 8) == NO)
    img = np.array([[0, 0, 0], [0, 0, 9], [0, 0, 0]], np.uint8)
    assert oracle_mod.bin_map(img, 8).tolist() == [[NO] * 3, [NO, 0, NO], [NO] * 3]


def test_channel_choice(oracle_mod):
    H, W = 7, 8
    yy, xx = np.mgrid[0:H, 0:W]
    img = np.zeros((H, W, 3), np.uint8)
    img[..., 0] = 2 * xx          # R: weak +x   (|g| = 4)
    img[..., 1] = 10 * yy         # G: strong +y (|g| = 20)
    img[..., 2] = 100 - 5 * xx    # B: medium -x (|g| = 10)
    assert np.all(interior(oracle_mod.bin_map(img, 8)) == 2)
    img[..., 1] = 0
    assert np.all(interior(oracle_mod.bin_map(img, 8)) == 4)
    # tie between R (+x) and G (+y) at equal magnitude: the lower index (R) wins
    img[..., 0] = 6 * xx
    img[..., 1] = 6 * yy
    img[..., 2] = 0
    assert np.all(interior(oracle_mod.bin_map(img, 8)) == 0)
    # tie between G (-y) and B (+x): G wins
    img[..., 0] = 0
    img[..., 1] = 100 - 6 * yy
    img[..., 2] = 6 * xx
    assert np.all(interior(oracle_mod.bin_map(img, 8)) == 6)


def test_gray_equals_identical_rgb(oracle_mod):
    rng = np.random.default_rng(5)
    g = rng.integers(0, 256, size=(23, 31), dtype=np.uint8)
    rgb = np.repeat(g[..., None], 3, axis=2)
    assert np.array_equal(oracle_mod.bin_map(g, 8), oracle_mod.bin_map(rgb, 8))


def test_hand_worked_5x5(oracle_mod):
    g = json.load(open(os.path.join(GOLDEN, "hand_5x5.json")))
    img = np.array(g["image_rows_y"], np.uint8)
    assert oracle_mod.bin_map(img, g["n_bins"]).tolist() == g["bins_rows_y"]


def test_bins_match_table(oracle_mod):
    """The per-pixel bin is the table entry at that pixel's (dx, dy)."""
    rng = np.random.default_rng(7)
    img = rng.integers(0, 256, size=(40, 50), dtype=np.uint8).astype(np.int32)
    lut = oracle_mod.lut(8)
    bins = oracle_mod.bin_map(img.astype(np.uint8), 8)
    dx = img[1:-1, 2:] - img[1:-1, :-2]
    dy = img[2:, 1:-1] - img[:-2, 1:-1]
    assert np.array_equal(interior(bins), lut[(dy + 255) * 511 + dx + 255])
