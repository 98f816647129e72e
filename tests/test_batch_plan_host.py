"""hog_batch_plan is host arithmetic (no CUDA call), so its layout is checked
here without a GPU: every item's cell and window counts, and where each
stage's tiles of each item start, against the definitions written out below
(cell positions (extent - cell) / stride + 1, windows of cells_x x cells_y
cells at one-cell steps of r = cell / stride positions, fused tiles of 32 x 16
cell positions at stride 4 and 16 x 16 at stride 8, one detection tile per
2048 window positions, 128-window strips of the row-GEMM score)."""

import os
import struct

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

HEADER = struct.Struct("<I15i")          # magic, 13 fields, 2 of padding
ITEM = struct.Struct("<QQiiQQii12i")     # hog_batch_item (48 bytes), 10 fields, 2 of padding


@pytest.fixture(scope="module")
def fh():
    import importlib.util

    spec = importlib.util.spec_from_file_location("_fasthog_build", os.path.join(ROOT, "paper_1703_06256_gb300",
                                                                                  "build.py"))
    b = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(b)
    b.build()
    import paper_1703_06256_gb300 as m

    return m


def n_pos(extent, box, stride):
    return 0 if extent < box else (extent - box) // stride + 1


def ceil_div(a, b):
    return (a + b - 1) // b


@pytest.mark.parametrize("cell,stride", [(8, 4), (8, 8), (16, 4)])
def test_plan_layout(fh, cell, stride):
    sizes = [(640, 480), (7, 5), (60, 100), (1920, 1080), (64, 128), (800, 600), (129, 257), (8, 8)]
    cells_x, cells_y, channels, nb = 8, 16, 3, 8
    items = [fh.HogBatchItem(4096, W * channels, W, H, 4096, 8192, k, k % 3) for k, (W, H) in enumerate(sizes)]
    plan = bytes(fh.hog_batch_plan(items, channels, nb, cell, stride, cells_x, cells_y))
    assert len(plan) == HEADER.size + ITEM.size * len(sizes)
    h = HEADER.unpack_from(plan, 0)
    magic, n_items, ch, nbins, c, s, cx, cy, r, cells_tiles, score_tc, score_ctas, detect_tiles, score_rows = h[:14]
    assert magic != 0
    assert (n_items, ch, nbins, c, s, cx, cy, r) == (len(sizes), channels, nb, cell, stride, cells_x, cells_y,
                                                     cell // stride)
    assert score_rows == (1 if r in (1, 2, 4) else 0) and score_tc >= 1
    bx = 32 if stride == 4 else 16
    cells_t = score_c = detect_t = 0
    for k, (W, H) in enumerate(sizes):
        f = ITEM.unpack_from(plan, HEADER.size + k * ITEM.size)
        img, pitch, w, hh, cells, scores, image, level = f[:8]
        ncx, ncy, nx, ny, cells_t0, cells_tx, score_c0, score_tx, score_bands, detect_t0 = f[8:18]
        assert (img, pitch, w, hh, cells, scores, image, level) == (4096, W * channels, W, H, 4096, 8192, k, k % 3)
        assert (ncx, ncy) == (n_pos(W, cell, stride), n_pos(H, cell, stride)), (W, H)
        ex, ey = ncx - (cells_x - 1) * r, ncy - (cells_y - 1) * r
        assert (nx, ny) == ((ex, ey) if ex > 0 and ey > 0 else (0, 0)), (W, H)
        assert cells_t0 == cells_t and score_c0 == score_c and detect_t0 == detect_t, (W, H)
        assert cells_tx == (ceil_div(ncx, bx) if ncx > 0 else 1)
        cells_t += ceil_div(ncx, bx) * ceil_div(ncy, 16) if ncx > 0 and ncy > 0 else 0
        assert score_tx == ceil_div(nx, 128) and score_bands == ceil_div(ny, score_tc), (W, H)
        score_c += score_tx * score_bands
        detect_t += ceil_div(nx * ny, 2048)
    assert (cells_tiles, score_ctas, detect_tiles) == (cells_t, score_c, detect_t)
