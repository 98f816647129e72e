"""Pins for the oracle's gradient binning and 511 x 511 table (Section 2, Fig. 2).

Each check is fixed by something other than the oracle itself: hand-counted
closed forms, the rotation symmetry of half-open sectors, numpy's arctan2
away from sector boundaries, and hand-picked spot values.
"""

import json
import math
import os

import numpy as np
import pytest

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")
D = np.arange(-255, 256)
DX, DY = np.meshgrid(D, D)  # DX[dy+255, dx+255] = dx


def test_closed_form_counts(oracle_mod):
    g = json.load(open(os.path.join(GOLDEN, "lut_closed_forms.json")))
    for nb_s, counts in g["counts"].items():
        nb = int(nb_s)
        lut = oracle_mod.lut(nb)
        hist = np.bincount(lut, minlength=256)
        assert hist[:nb].tolist() == counts, nb
        assert hist[255] == g["no_bin_entries"]
        assert lut[255 * 511 + 255] == 255  # (0, 0)


def test_spot_values(oracle_mod):
    g = json.load(open(os.path.join(GOLDEN, "lut_closed_forms.json")))
    lut = oracle_mod.lut(8)
    for dx, dy, b in g["spot_values_nb8"]:
        assert oracle_mod.sector_bin(dx, dy, 8) == b, (dx, dy)
        assert lut[(dy + 255) * 511 + dx + 255] == b


@pytest.mark.parametrize("nb", [4, 8, 12, 16, 20, 32])
def test_rotation_by_quarter_turn(oracle_mod, nb):
    """(dx, dy) -> (-dy, dx) adds pi/2 to phi, so with 4 | N_b it adds N_b/4 to the bin."""
    lut = oracle_mod.lut(nb).reshape(511, 511)  # [dy+255, dx+255]
    # rotated entry for (dx, dy) is at (dx', dy') = (-dy, dx): row dx+255, col -dy+255
    rot = lut[DX + 255, -DY + 255]
    mask = ~((DX == 0) & (DY == 0))
    assert np.array_equal(rot[mask], (lut[mask].astype(int) + nb // 4) % nb)


@pytest.mark.parametrize("nb", list(range(1, 33)))
def test_matches_arctan2_off_boundary(oracle_mod, nb):
    """numpy's arctan2 gives phi; away from sector boundaries floor(phi*N_b/2pi) is the bin."""
    oracle_mod.reset_margin()
    lut = oracle_mod.lut(nb).reshape(511, 511).astype(int)
    assert not oracle_mod.margin_violation()
    phi = np.mod(np.arctan2(DY.astype(np.float64), DX.astype(np.float64)), 2 * math.pi)
    t = phi * nb / (2 * math.pi)
    frac_dist = np.abs(t - np.round(t))
    off = (frac_dist > 1e-9) & ~((DX == 0) & (DY == 0))
    expect = np.floor(t).astype(int) % nb
    assert np.array_equal(lut[off], expect[off])
    # On-boundary lattice points exist only on the rays at multiples of pi/4
    # (Niven's theorem); there the half-open sector starting at the ray wins.
    on = (~off) & ~((DX == 0) & (DY == 0))
    assert np.all((DX[on] == 0) | (DY[on] == 0) | (np.abs(DX[on]) == np.abs(DY[on])))
    assert np.array_equal(lut[on], np.round(t[on]).astype(int) % nb)


def test_margin_certificate(oracle_mod):
    """The FP64 sign tests against irrational boundaries keep a margin far above
    any fixed-point evaluation error (2^-40 scale): the smallest |cross| over
    all lattice points and all N_b <= 64 stays above 1e-6."""
    oracle_mod.reset_margin()
    for nb in range(1, 65):
        oracle_mod.lut(nb)
    assert not oracle_mod.margin_violation()
    assert oracle_mod.min_margin() > 1e-6


def test_axis_reflection_off_boundary(oracle_mod):
    """(dx, dy) -> (dx, -dy) maps phi to 2pi - phi; off boundaries bin -> N_b-1-bin."""
    nb = 9
    lut = oracle_mod.lut(nb).reshape(511, 511).astype(int)
    refl = lut[-DY + 255, DX + 255]
    phi = np.mod(np.arctan2(DY.astype(float), DX.astype(float)), 2 * math.pi)
    t = phi * nb / (2 * math.pi)
    off = (np.abs(t - np.round(t)) > 1e-9) & (DY != 0)
    assert np.array_equal(refl[off], nb - 1 - lut[off])
