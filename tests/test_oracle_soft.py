"""Pins of the oracle's soft votes (the two-bin vote of Section 2): closed
forms on the axes and diagonals, agreement of the larger vote with the exact
hard bin over the whole table, quarter-turn symmetry, a certified distance
from rounding ties (so any correctly rounded atan2 gives the same table),
the vote as the rounded linear interpolation weight over the whole table,
unit mass per pixel, and cells through weighted integral images (Eq. 5,
Eq. 6) equal to direct sums."""

import numpy as np
import pytest


def entry(tab, dx, dy):
    e = int(tab[dy + 255, dx + 255])
    return e & 0xFF, e >> 8


@pytest.mark.parametrize("nb", [4, 8, 9, 12, 16])
def test_tie_margin_certified(oracle_mod, nb):
    _, m = oracle_mod.soft_lut(nb)
    assert m > 1e-9, m  # FP64 atan2 errors are ~1e-16 in t: no entry is near a rounding tie


def test_closed_forms(oracle_mod):
    q = oracle_mod.SOFT_Q
    t8, _ = oracle_mod.soft_lut(8)
    # angles on bin boundaries split evenly between the two bins whose centres flank them
    assert entry(t8, 1, 0) == (7, q // 2)      # phi = 0: centres of bins 7 and 0
    assert entry(t8, 0, 1) == (1, q // 2)      # phi = pi/2: bins 1 and 2
    assert entry(t8, 1, 1) == (0, q // 2)      # phi = pi/4: bins 0 and 1
    assert entry(t8, -1, 0) == (3, q // 2)     # phi = pi: bins 3 and 4
    assert entry(t8, 0, 0) == (0xFF, 0xFF)
    t4, _ = oracle_mod.soft_lut(4)
    assert entry(t4, 1, 1) == (0, 0)           # phi = pi/4: the centre of bin 0, all votes there
    assert entry(t4, -1, 1) == (1, 0)          # phi = 3 pi/4: centre of bin 1
    assert entry(t4, -5, -5) == (2, 0)


@pytest.mark.parametrize("nb", [4, 8, 16])
def test_larger_vote_is_the_hard_bin(oracle_mod, nb):
    soft, _ = oracle_mod.soft_lut(nb)
    hard = oracle_mod.lut(nb).reshape(511, 511)
    q = oracle_mod.SOFT_Q
    k0 = (soft & 0xFF).astype(np.int64)
    a = (soft >> 8).astype(np.int64)
    ok = soft != 0xFFFF
    big = np.where(a > q - a, (k0 + 1) % nb, k0)
    tie = a * 2 == q
    assert np.all(hard[ok & ~tie] == big[ok & ~tie])
    assert np.all((hard[ok & tie] == k0[ok & tie]) | (hard[ok & tie] == (k0[ok & tie] + 1) % nb))


@pytest.mark.parametrize("nb", [8, 9, 16])
def test_vote_is_the_rounded_interpolation_weight(oracle_mod, nb):
    """The vote for the upper of the two flanking bins is the linear
    interpolation weight between their centres, in units of 1/q, rounded to
    the nearest unit: within 1/2 of q times the weight, for every gradient of
    the table.  The angle here comes from numpy's arctan2, independently of the
    oracle's libm call; the certified tie margin keeps the two from rounding
    differently."""
    soft, _ = oracle_mod.soft_lut(nb)
    q = oracle_mod.SOFT_Q
    dy, dx = np.mgrid[-255:256, -255:256]
    ok = (dx != 0) | (dy != 0)
    phi = np.mod(np.arctan2(dy, dx), 2 * np.pi)
    t = phi * nb / (2 * np.pi) - 0.5
    fl = np.floor(t)
    w = q * (t - fl)  # q times the weight of the upper bin
    k0 = (soft & 0xFF).astype(np.int64)
    a = (soft >> 8).astype(np.int64)
    lower = np.mod(fl, nb).astype(np.int64)
    # a vote of q for the upper bin is written as 0 for the next pair of bins
    wraps = ok & (np.abs(w - q) <= 0.5)
    plain = ok & ~wraps
    assert np.all(np.abs(a[plain] - w[plain]) <= 0.5)
    assert np.all(k0[plain] == lower[plain])
    assert np.all((a[wraps] == 0) & (k0[wraps] == (lower[wraps] + 1) % nb))


@pytest.mark.parametrize("nb", [4, 8, 16])
def test_quarter_turn(oracle_mod, nb):
    soft, _ = oracle_mod.soft_lut(nb)
    rng = np.random.default_rng(nb)
    for dx, dy in rng.integers(-255, 256, size=(4000, 2)):
        if dx == 0 and dy == 0:
            continue
        k, a = entry(soft, dx, dy)
        k2, a2 = entry(soft, -dy, dx)  # the gradient turned by +pi/2
        assert a2 == a and k2 == (k + nb // 4) % nb, (dx, dy)


def test_votes_mass_and_table(oracle_mod):
    rng = np.random.default_rng(3)
    img = rng.integers(0, 256, size=(40, 50, 3), dtype=np.uint8)
    q = oracle_mod.SOFT_Q
    v = oracle_mod.soft_votes(img, 8)
    bins = oracle_mod.bin_map(img, 8)
    s = v.sum(axis=2)
    assert np.array_equal(s, np.where(bins < 8, q, 0))  # q per pixel with a gradient, 0 elsewhere
    # a pixel's hard bin (exact sector predicate) receives at least half of its votes
    ys, xs = np.nonzero(bins < 8)
    assert np.all(v[ys, xs, bins[ys, xs]] * 2 >= q)
    assert np.all(np.count_nonzero(v, axis=2) <= 2)


@pytest.mark.parametrize("stride", [4, 8])
def test_cells_through_integral_images(oracle_mod, stride):
    rng = np.random.default_rng(11 + stride)
    img = rng.integers(0, 256, size=(70, 90, 3), dtype=np.uint8)
    v = oracle_mod.soft_votes(img, 8).astype(np.int64)
    ii = v.cumsum(axis=0).cumsum(axis=1)  # Eq. 5 on the weighted vote planes

    def at(y, x):
        return ii[y, x] if y >= 0 and x >= 0 else np.zeros(8, np.int64)

    direct = oracle_mod.soft_cells(img, 8, 8, stride)
    ncy, ncx, _ = direct.shape
    for j in range(ncy):
        for i in range(ncx):
            y0, x0, y1, x1 = j * stride, i * stride, j * stride + 7, i * stride + 7
            box = at(y1, x1) + at(y0 - 1, x0 - 1) - at(y0 - 1, x1) - at(y1, x0 - 1)  # Eq. 6
            assert np.array_equal(box, direct[j, i])
