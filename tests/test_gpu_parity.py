"""GPU parity: every stage of the CUDA path against the oracle, called through
the C ABI, on seeded inputs that span several tiles and ragged tails.

Bar: bit-exact for the table, bin map, integral images, cell histograms,
integer scores and detection lists; FP32 scores within
1e-5 * (sum_k |w_k| h_k + |bias|) of the FP64 oracle."""

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

import oracle  # noqa: E402
import workloads as wl  # noqa: E402


@pytest.fixture(scope="module")
def fh():
    import paper_1703_06256_gb300 as m

    assert torch.cuda.is_available()
    m.hog_device_status(clear=True)
    yield m
    assert m.hog_device_status() == 0, "a kernel reported a timed-out wait"


@pytest.fixture(scope="module")
def g(fh):
    import _gpu

    return _gpu


class score_engine:
    """Force the single-image score's engine (HOG_TUNE_SCORE_PATH) in a block."""

    def __init__(self, fh, path):
        self.fh, self.path = fh, path

    def __enter__(self):
        self.fh.hog_tune_set(self.fh.HOG_TUNE_SCORE_PATH, self.path)

    def __exit__(self, *exc):
        self.fh.hog_tune_set(self.fh.HOG_TUNE_SCORE_PATH, 0)


def rand_img(H, W, ch, seed):
    rng = np.random.default_rng(seed)
    shape = (H, W) if ch == 1 else (H, W, 3)
    return rng.integers(0, 256, size=shape, dtype=np.uint8)


# ---------------------------------------------------------------- table
@pytest.mark.parametrize("nb", [1, 2, 3, 4, 5, 6, 7, 8, 9, 12, 16, 17, 31, 32, 64])
def test_lut_exhaustive(fh, g, nb):
    buf = g.gpu_lut(nb).cpu().numpy()
    lut = buf[: fh.HOG_LUT_QUAD_OFFSET].reshape(511, 512)
    assert np.all(lut[:, 511] == 255)  # pad column
    assert np.array_equal(lut[:, :511].reshape(-1), oracle.lut(nb))
    quad = buf[fh.HOG_LUT_QUAD_OFFSET:].reshape(256, 256)  # row dy, column dx - 1
    assert np.array_equal(quad[:, :255], lut[255:, 256:511]) and np.all(quad[:, 255] == 255)


# ---------------------------------------------------------------- bin map
SHAPES = [(1, 1), (2, 2), (3, 3), (1, 100), (100, 1), (17, 129), (35, 131), (7, 1000), (240, 320), (33, 257)]


@pytest.mark.parametrize("nb", [8, 9, 16, 6])
@pytest.mark.parametrize("ch", [1, 3])
def test_bin_map_random(fh, g, nb, ch):
    for i, (H, W) in enumerate(SHAPES):
        img = rand_img(H, W, ch, 100 * nb + 10 * ch + i)
        assert np.array_equal(g.gpu_bins(img, nb), oracle.bin_map(img, nb)), (H, W)


@pytest.mark.parametrize("table", [1, 2])
@pytest.mark.parametrize("nb", [8, 16, 4])
@pytest.mark.parametrize("ch", [1, 3])
def test_bin_map_table_placements(fh, g, nb, ch, table):
    """The bin map with the table quadrant staged in shared memory (1) and
    with the whole table read through the cache (2) equals the oracle's."""
    fh.hog_tune_set(fh.HOG_TUNE_TABLE, table)
    try:
        for i, (H, W) in enumerate(SHAPES):
            img = rand_img(H, W, ch, 700 * nb + 10 * ch + i)
            assert np.array_equal(g.gpu_bins(img, nb), oracle.bin_map(img, nb)), (H, W)
    finally:
        fh.hog_tune_set(fh.HOG_TUNE_TABLE, 0)


SCHEDULE_SHAPES = SHAPES + [(16, 128), (18, 130), (31, 255), (600, 800), (17, 1023), (2, 5000), (300, 4),
                            (1100, 200)]


@pytest.mark.parametrize("schedule", [0, 1, 2])
@pytest.mark.parametrize("nb", [8, 9])
@pytest.mark.parametrize("ch", [1, 3])
def test_bin_map_schedules(fh, g, nb, ch, schedule):
    """Both bin-map schedules (1: grid-stride over quads, loads from global
    memory; 2: 128 x 16 tiles staged in shared memory) and the library's
    choice (0) equal the oracle's bin map.  Rows padded to a multiple of 16
    bytes let schedule 2 apply (every tile edge: ragged widths and heights,
    images narrower than a tile, one row, one column); unpadded rows and an
    unaligned base fall back to schedule 1."""
    fh.hog_tune_set(fh.HOG_TUNE_BINMAP_SCHEDULE, schedule)
    try:
        for i, (H, W) in enumerate(SCHEDULE_SHAPES):
            img = rand_img(H, W, ch, 900 * nb + 10 * ch + i)
            ref = oracle.bin_map(img, nb)
            pad = (-W * ch) % 16
            assert np.array_equal(g.gpu_bins(img, nb, pitch_pad=pad), ref), (H, W, "padded")
            assert np.array_equal(g.gpu_bins(img, nb, pitch_pad=pad + 16, offset=3), ref), (H, W, "offset")
    finally:
        fh.hog_tune_set(fh.HOG_TUNE_BINMAP_SCHEDULE, 0)


@pytest.mark.parametrize("ch", [1, 3])
def test_bin_map_pitch_and_alignment(fh, g, ch):
    img = rand_img(45, 203, ch, 5)
    ref = oracle.bin_map(img, 8)
    for pad, off in [(0, 1), (1, 0), (5, 3), (16, 0), (13, 2)]:
        assert np.array_equal(g.gpu_bins(img, 8, pitch_pad=pad, offset=off), ref), (pad, off)


def test_bin_map_closed_form_ramps(fh, g):
    yy, xx = np.mgrid[0:50, 0:60]  # every ramp stays within 0..255
    for img, b in [(3 * xx, 0), (5 * yy, 2), (250 - 5 * yy, 6), (250 - 2 * xx, 4), (2 * xx + 2 * yy, 1)]:
        bins = g.gpu_bins(img.astype(np.uint8), 8)
        assert np.all(bins[1:-1, 1:-1] == b)
        assert np.all(bins[0] == 255) and np.all(bins[:, -1] == 255)


def test_bin_map_workloads(fh, g):
    for cfg in (wl.config0(), wl.config1()):
        img = cfg["images"][0]
        assert np.array_equal(g.gpu_bins(img, cfg["n_bins"]), oracle.bin_map(img, cfg["n_bins"]))


# ---------------------------------------------------------------- integral images
II_SHAPES = [(1, 1), (5, 5), (2, 3), (8, 513), (33, 1025), (37, 2000), (600, 800), (240, 320), (19, 511),
             (3, 4097), (301, 6)]


def oracle_bins(H, W, nb, seed, p_none=0.3):
    rng = np.random.default_rng(seed)
    b = rng.integers(0, nb, size=(H, W)).astype(np.uint8)
    b[rng.random((H, W)) < p_none] = 255
    return b


@pytest.mark.parametrize("nb", [8, 3, 16, 20])
def test_integral_int32(fh, g, nb):
    for i, (H, W) in enumerate(II_SHAPES):
        bins = oracle_bins(H, W, nb, 7 * nb + i)
        assert np.array_equal(g.gpu_integral(bins, nb), oracle.integral(bins, nb)), (H, W)


@pytest.mark.parametrize("nb", [8, 16])
def test_integral_uint16_modular(fh, g, nb):
    for i, (H, W) in enumerate([(600, 800), (37, 2000), (300, 700)]):
        bins = oracle_bins(H, W, nb, 31 * nb + i, p_none=0.05)
        bins[np.random.default_rng(i).random((H, W)) < 0.5] = 1  # one dominant bin: planes pass 2^16
        ref = oracle.integral(bins, nb)
        assert ref.max() > 65535 or (H, W) != (600, 800)
        assert np.array_equal(g.gpu_integral(bins, nb, fh.HOG_U16), (ref & 0xFFFF).astype(np.uint16)), (H, W)


@pytest.mark.parametrize("path,h", [(1, 4), (1, 8), (1, 16), (1, 32), (2, 16), (2, 32), (3, 0)])
def test_integral_band_heights(fh, g, path, h):
    """Every schedule (HOG_TUNE_INTEGRAL_PATH: three launches, single pass,
    cluster pass) at every tile height (HOG_TUNE_INTEGRAL_BAND_ROWS), int32 and
    uint16, one window of bins and several (N_b = 20, 64): the tiles, the
    carries between bands and groups, and partial bands at the bottom."""
    fh.hog_tune_set(fh.HOG_TUNE_INTEGRAL_BAND_ROWS, h)
    fh.hog_tune_set(fh.HOG_TUNE_INTEGRAL_PATH, path)
    try:
        for i, (H, W, nb) in enumerate([(600, 800, 8), (301, 6, 8), (70, 300, 20), (33, 1025, 64), (97, 130, 3),
                                        (1000, 257, 16)]):
            bins = oracle_bins(H, W, nb, 1000 * h + i)
            ref = oracle.integral(bins, nb)
            assert np.array_equal(g.gpu_integral(bins, nb), ref), (h, H, W, nb)
            assert np.array_equal(g.gpu_integral(bins, nb, fh.HOG_U16), (ref & 0xFFFF).astype(np.uint16)), (h, H, W, nb)
    finally:
        fh.hog_tune_set(fh.HOG_TUNE_INTEGRAL_BAND_ROWS, 0)
        fh.hog_tune_set(fh.HOG_TUNE_INTEGRAL_PATH, 0)


@pytest.mark.parametrize("ii_dtype", ["i32", "u16"])
def test_integral_three_launches_large(fh, g, ii_dtype):
    """Three launches (the library's choice above 640 rows) at 1920x1080 and
    3840x2160, 8 bins: 2160 rows of tiles with every group whole, and
    1000x1000 with a partial last group; int32 and uint16 planes, against
    the oracle."""
    fh.hog_tune_set(fh.HOG_TUNE_INTEGRAL_PATH, 1)
    try:
        for i, (H, W) in enumerate([(1080, 1920), (2160, 3840), (1000, 1000)]):
            bins = oracle_bins(H, W, 8, 700 + i, p_none=0.2)
            ref = oracle.integral(bins, 8)
            if ii_dtype == "i32":
                assert np.array_equal(g.gpu_integral(bins, 8), ref), (H, W)
            else:
                out = g.gpu_integral(bins, 8, fh.HOG_U16)
                assert np.array_equal(out, (ref & 0xFFFF).astype(np.uint16)), (H, W)
    finally:
        fh.hog_tune_set(fh.HOG_TUNE_INTEGRAL_PATH, 0)


def test_integral_single_pass_many_tiles(fh, g):
    """The single pass forced onto large maps, where a tile sums the
    aggregates of up to 134 tiles above it and 29 to its left: 1920x1080 and
    3840x2160 (8 bins), against the oracle."""
    fh.hog_tune_set(fh.HOG_TUNE_INTEGRAL_PATH, 2)
    try:
        for i, (H, W) in enumerate([(1080, 1920), (2160, 3840)]):
            bins = oracle_bins(H, W, 8, 500 + i, p_none=0.2)
            assert np.array_equal(g.gpu_integral(bins, 8), oracle.integral(bins, 8)), (H, W)
    finally:
        fh.hog_tune_set(fh.HOG_TUNE_INTEGRAL_PATH, 0)


@pytest.mark.parametrize("nb,warp_rows", [(8, 0), (8, 2), (8, 4), (8, 8), (3, 0), (16, 0), (20, 0), (20, 8)])
def test_integral_cluster_pass(fh, g, nb, warp_rows):
    """The cluster pass (one cluster of CTAs per 128-column group, carries
    through distributed shared memory, the row carries counted from the bins
    to the left) at every row count per warp (HOG_TUNE_INTEGRAL_WARP_ROWS: 2
    and 4 take images up to 640 rows, 8 up to 1280): cluster sizes from 1 to
    16 CTAs, the tallest image each takes, ragged right and bottom edges, an
    unaligned width (scalar loads and stores), and the widest image (63 groups
    to the left of the last one).  The pass uses no workspace: a zero-filled
    one stays zero, which also shows that the pass ran.  Images it does not
    take fall back to another schedule."""
    shapes = [(600, 800), (1, 1), (5, 129), (64, 128), (65, 130), (130, 333), (480, 640), (640, 300),
              (641, 300), (1080, 1920), (1280, 260), (17, 8192), (9, 8191), (301, 6), (1281, 100)]
    fh.hog_tune_set(fh.HOG_TUNE_INTEGRAL_PATH, 3)
    fh.hog_tune_set(fh.HOG_TUNE_INTEGRAL_WARP_ROWS, warp_rows)
    tallest = 640 if warp_rows in (2, 4) else 1280
    try:
        for i, (H, W) in enumerate(shapes):
            bins = oracle_bins(H, W, nb, 4000 + 37 * nb + i, p_none=0.25)
            ref = oracle.integral(bins, nb)
            ws = torch.zeros(fh.hog_integral_workspace_bytes(W, H, nb), dtype=torch.uint8, device="cuda")
            assert np.array_equal(g.gpu_integral(bins, nb, ws=ws), ref), (H, W, nb)
            assert np.array_equal(g.gpu_integral(bins, nb, fh.HOG_U16, ws=ws), (ref & 0xFFFF).astype(np.uint16)), \
                (H, W, nb)
            assert (int(ws.count_nonzero()) == 0) == (H <= tallest), (H, W, "cluster pass taken or not")
    finally:
        fh.hog_tune_set(fh.HOG_TUNE_INTEGRAL_PATH, 0)
        fh.hog_tune_set(fh.HOG_TUNE_INTEGRAL_WARP_ROWS, 0)


def test_integral_one_workspace_many_calls(fh, g):
    """One workspace, zero-filled once per image size, serves calls of that
    size with different bin counts, dtypes and schedules in a row (each
    single-pass launch accepts only the flags of its own launch and leaves
    the tag for the next)."""
    ws = torch.zeros(fh.hog_integral_workspace_bytes(1100, 600, 64), dtype=torch.uint8, device="cuda")
    sizes = {(600, 1100): [(8, 0), (8, 0), (20, 1), (20, 2), (64, 2), (8, 2), (3, 1), (16, 2)],
             (37, 259): [(16, 2), (8, 0), (8, 1), (8, 3), (8, 2), (20, 3), (8, 1)],
             (1, 5): [(8, 2), (8, 2)]}
    try:
        for (H, W), calls in sizes.items():
            ws.zero_()  # a new image size
            for i, (nb, path) in enumerate(calls):
                fh.hog_tune_set(fh.HOG_TUNE_INTEGRAL_PATH, path)
                bins = oracle_bins(H, W, nb, 900 + i)
                ref = oracle.integral(bins, nb)
                dt = fh.HOG_U16 if i % 3 == 2 else fh.HOG_I32
                got = g.gpu_integral(bins, nb, dt, ws=ws)
                want = (ref & 0xFFFF).astype(np.uint16) if dt == fh.HOG_U16 else ref
                assert np.array_equal(got, want), (H, W, i, nb, path)
    finally:
        fh.hog_tune_set(fh.HOG_TUNE_INTEGRAL_PATH, 0)
    assert fh.hog_device_status() == 0


def test_integral_workload_bins(fh, g):
    img = wl.config1()["images"][0]
    bins = oracle.bin_map(img, 8)
    assert np.array_equal(g.gpu_integral(bins, 8), oracle.integral(bins, 8))


# ---------------------------------------------------------------- cell histograms
@pytest.mark.parametrize("stride", [1, 2, 4, 8])
@pytest.mark.parametrize("cell_dtype", ["i32", "bf16", "f32"])
def test_cell_hist(fh, g, stride, cell_dtype):
    cd = {"i32": fh.HOG_I32, "bf16": fh.HOG_BF16, "f32": fh.HOG_F32}[cell_dtype]
    for i, (H, W) in enumerate([(8, 8), (40, 77), (130, 259), (7, 30)]):
        bins = oracle_bins(H, W, 8, 3 * stride + i)
        ii = oracle.integral(bins, 8)
        ref = oracle.cell_hist_ii(ii, 8, 8, stride)
        assert np.array_equal(g.gpu_cells(ii, 8, 8, stride, cell_dtype=cd), ref), (H, W)


@pytest.mark.parametrize("rows", [1, 4, 8, 16])
@pytest.mark.parametrize("nb,cell,stride", [(8, 8, 4), (16, 8, 4), (8, 16, 8), (8, 8, 2), (16, 32, 4)])
def test_cell_hist_launch_shapes(fh, g, rows, nb, cell, stride):
    """Every cell-histogram launch shape (HOG_TUNE_CELL_ROWS: 1 = per-cell
    corner reads, 4/8/16 = staged sample grid) gives the oracle's cells from
    int32 and uint16 integral images, on maps spanning several tiles."""
    fh.hog_tune_set(fh.HOG_TUNE_CELL_ROWS, rows)
    try:
        for i, (H, W) in enumerate([(150, 700), (301, 233)]):
            bins = oracle_bins(H, W, nb, 50 * nb + rows + i)
            ii = oracle.integral(bins, nb)
            ref = oracle.cell_hist_ii(ii, nb, cell, stride)
            assert np.array_equal(g.gpu_cells(ii, nb, cell, stride), ref), (H, W)
            got16 = g.gpu_cells((ii & 0xFFFF).astype(np.uint16), nb, cell, stride, ii_dtype=fh.HOG_U16)
            assert np.array_equal(got16, ref), (H, W)
    finally:
        fh.hog_tune_set(fh.HOG_TUNE_CELL_ROWS, 0)


def test_cell_hist_from_uint16(fh, g):
    bins = oracle_bins(600, 800, 8, 99, p_none=0.02)
    ii = oracle.integral(bins, 8)
    ref = oracle.cell_hist_ii(ii, 8, 8, 4)
    got = g.gpu_cells((ii & 0xFFFF).astype(np.uint16), 8, 8, 4, ii_dtype=fh.HOG_U16)
    assert np.array_equal(got, ref)


def test_cell_hist_other_cells(fh, g):
    bins = oracle_bins(70, 90, 9, 4)
    ii = oracle.integral(bins, 9)
    for cell, stride in [(16, 4), (6, 3), (5, 5), (1, 1)]:
        assert np.array_equal(g.gpu_cells(ii, 9, cell, stride), oracle.cell_hist_ii(ii, 9, cell, stride))


# ---------------------------------------------------------------- window scores
def cells_of(img, nb, stride):
    return oracle.cell_hist_direct(oracle.bin_map(img, nb), nb, 8, stride)


@pytest.mark.parametrize("stride", [8, 4, 2, 1])
@pytest.mark.parametrize("cell_dtype", ["i32", "f32"])
def test_score_f32(fh, g, stride, cell_dtype):
    cd = fh.HOG_I32 if cell_dtype == "i32" else fh.HOG_F32
    rng = np.random.default_rng(stride)
    img = rand_img(300, 260, 3, stride)
    cells = cells_of(img, 8, stride)
    w = rng.normal(0, 0.01, 1024).astype(np.float32)
    for bias in (0.0, 0.37):
        ref = oracle.window_score(cells, w, bias, stride=stride)
        got = g.gpu_scores(cells, w, fh.HOG_F32, bias, stride=stride, cell_dtype=cd)
        tol = g.score_tolerance(cells, w, bias, stride=stride)
        assert got.shape == ref.shape
        assert np.all(np.abs(got - ref) <= tol)


def test_score_i8_exact(fh, g):
    rng = np.random.default_rng(8)
    img = rand_img(280, 200, 3, 8)
    cells = cells_of(img, 8, 4)
    w = rng.integers(-127, 128, 1024).astype(np.int8)
    ref = oracle.window_score(cells, w, 3.0, stride=4)
    got = g.gpu_scores(cells, w, fh.HOG_I8, 3.0, stride=4)
    assert got.dtype == np.int32 and np.array_equal(got, ref.astype(np.int64))


def test_score_bf16_weights_and_cells(fh, g):
    rng = np.random.default_rng(9)
    img = rand_img(290, 230, 3, 9)
    cells = cells_of(img, 8, 4)
    w = rng.normal(0, 0.01, 1024).astype(np.float32)
    w_bf = torch.from_numpy(w).to(torch.bfloat16).float().numpy()  # the weights the kernel sees
    ref = oracle.window_score(cells, w_bf, 0.0, stride=4)
    for cd in (fh.HOG_I32, fh.HOG_BF16, fh.HOG_F32):
        got = g.gpu_scores(cells, w, fh.HOG_BF16, 0.0, stride=4, cell_dtype=cd)
        assert np.all(np.abs(got - ref) <= g.score_tolerance(cells, w_bf, 0.0, stride=4))


def test_score_shapes(fh, g):
    rng = np.random.default_rng(10)
    for (H, W, nb, cx, cy, stride) in [(128, 64, 8, 8, 16, 8), (127, 64, 8, 8, 16, 8), (140, 80, 9, 8, 16, 4),
                                       (96, 96, 4, 4, 4, 2), (64, 64, 16, 3, 5, 1)]:
        img = rand_img(H, W, 1, H + W)
        cells = oracle.cell_hist_direct(oracle.bin_map(img, nb), nb, 8, stride)
        w = rng.normal(0, 0.1, cx * cy * nb).astype(np.float32)
        ref = oracle.window_score(cells, w, 0.0, cx, cy, 8, stride)
        got = g.gpu_scores(cells, w, fh.HOG_F32, 0.0, stride=stride, cells_x=cx, cells_y=cy)
        assert got.shape == ref.shape
        if ref.size:
            assert np.all(np.abs(got - ref) <= g.score_tolerance(cells, w, 0.0, 8, stride, cx, cy))


# ---------------------------------------------------------------- detection list
def test_detect_int_exact(fh, g):
    rng = np.random.default_rng(11)
    for ny, nx in [(1, 1), (7, 9), (119, 185), (300, 401), (0, 5)]:
        S = rng.integers(-50, 50, size=(ny, nx)).astype(np.int32)
        xs, ys, sc = oracle.detect(S.astype(np.float64), 4, 10.0)
        det, n = g.gpu_detect(S, 4, 10.0, image=3, level=2)
        assert n == len(xs)
        assert np.array_equal(det["x"], xs) and np.array_equal(det["y"], ys)
        assert np.array_equal(det["score"], sc.astype(np.float32))
        assert np.all(det["image"] == 3) and np.all(det["level"] == 2)


def test_detect_float_and_overflow(fh, g):
    rng = np.random.default_rng(12)
    S = rng.normal(0, 1, size=(211, 333)).astype(np.float32)
    S[5, 7] = 0.5  # exactly on the threshold: kept
    xs, ys, sc = oracle.detect(S.astype(np.float64), 4, 0.5)
    det, n = g.gpu_detect(S, 4, 0.5)
    assert n == len(xs) and np.array_equal(det["x"], xs) and np.array_equal(det["y"], ys)
    det, n2 = g.gpu_detect(S, 4, 0.5, max_out=100)
    assert n2 == len(xs) and len(det) == 100 and np.array_equal(det["x"], xs[:100])


def test_detect_many_tiles(fh, g):
    """A map of 2154 tiles (look-back over many windows of 32 predecessors):
    the list equals the oracle's, in order, also truncated mid-list, call
    after call on the same workspace; a workspace below
    hog_detect_workspace_bytes is refused."""
    rng = np.random.default_rng(14)
    ny, nx = 2100, 2100  # 4.41M scores, 2154 tiles
    S = rng.normal(0, 1, size=(ny, nx)).astype(np.float32)
    xs, ys, sc = oracle.detect(S.astype(np.float64), 4, 1.5)
    det, n = g.gpu_detect(S, 4, 1.5)
    assert n == len(xs) and np.array_equal(det["x"], xs) and np.array_equal(det["y"], ys)
    assert np.array_equal(det["score"], sc.astype(np.float32))
    det, n2 = g.gpu_detect(S, 4, 1.5, max_out=len(xs) // 2 + 3)
    k = len(xs) // 2 + 3
    assert n2 == len(xs) and len(det) == k and np.array_equal(det["x"], xs[:k]) and np.array_equal(det["y"], ys[:k])
    ws_b = fh.hog_detect_workspace_bytes(nx, ny)
    assert ws_b >= 8 * 2154
    s_d = torch.from_numpy(S.reshape(-1)).cuda()
    out = torch.empty(16 * fh.DET_BYTES, dtype=torch.uint8, device="cuda")
    cnt = torch.zeros(1, dtype=torch.int32, device="cuda")
    ws = torch.zeros(ws_b, dtype=torch.uint8, device="cuda")
    with pytest.raises(fh.HogError):
        fh.hog_detect(s_d, fh.HOG_F32, nx, ny, 4, 1.5, 0, 0, out, 16, cnt, ws, ws_b - 256)


def test_detect_truncation_and_offsets(fh, g):
    """The list stops at max_out exactly (at tile boundaries and inside a
    tile), nothing past it is written, and any 4-byte-aligned start works."""
    rng = np.random.default_rng(13)
    S = rng.normal(0, 1, size=(97, 211)).astype(np.float32)  # ~20.5k scores: 11 tiles of 2048
    xs, ys, sc = oracle.detect(S.astype(np.float64), 4, 0.0)
    n_ref = len(xs)
    s = torch.from_numpy(S.reshape(-1)).cuda()
    ws_b = fh.hog_detect_workspace_bytes(211, 97)
    ws = torch.zeros(ws_b, dtype=torch.uint8, device="cuda")  # one workspace for every call below
    for max_out in (0, 1, 1023, 1024, 1025, 5000, n_ref - 1, n_ref, n_ref + 7):
        for shift in (0, 4, 8, 12):
            total = (n_ref + 16) * fh.DET_BYTES + 64
            buf = torch.full((total,), 0x5A, dtype=torch.uint8, device="cuda")
            cnt = torch.full((1,), -7, dtype=torch.int32, device="cuda")
            fh.hog_detect(s, fh.HOG_F32, 211, 97, 4, 0.0, 1, 0, buf.data_ptr() + shift, max_out, cnt, ws, ws_b)
            host = buf.cpu().numpy()
            assert int(cnt.item()) == n_ref
            k = min(max_out, n_ref)
            det = host[shift: shift + k * fh.DET_BYTES].copy().view(fh.dets_to_numpy(b"", 0).dtype)
            assert np.array_equal(det["x"], xs[:k]) and np.array_equal(det["y"], ys[:k])
            assert np.array_equal(det["score"], sc[:k].astype(np.float32))
            assert np.all(host[:shift] == 0x5A) and np.all(host[shift + k * fh.DET_BYTES:] == 0x5A)


# ---------------------------------------------------------------- whole path
def compare_pipeline(fh, g, img, nb, stride, w, bias, thr, ii_dtype, cell_dtype):
    H, W = img.shape[:2]
    ch = 1 if img.ndim == 2 else 3
    pipe = fh.HogPipeline(W, H, ch, nb, stride, ii_dtype=ii_dtype, cell_dtype=cell_dtype)
    pipe.set_weights(w, bias, thr if thr is not None else -1e30)
    pipe.set_image(img)
    pipe.run()
    got = pipe.results()
    ref = oracle.pipeline(img, nb, w, bias, stride, thr if thr is not None else -1e30)
    assert np.array_equal(got["bins"], ref["bins"])
    if ii_dtype == fh.HOG_I32:
        assert np.array_equal(got["ii"], ref["ii"])
    else:
        assert np.array_equal(got["ii"], (ref["ii"] & 0xFFFF).astype(np.uint16))
    assert np.array_equal(got["cells"], ref["cells"])
    tol = g.score_tolerance(ref["cells"], w, bias, stride=stride)
    assert np.all(np.abs(got["scores"] - ref["scores"]) <= tol)
    t = thr if thr is not None else -1e30
    g.check_detections(got["detections"], got["count"], got["scores"], ref["scores"], tol, t, stride)
    return got


def test_pipeline_config0(fh, g):
    c = wl.config0()
    compare_pipeline(fh, g, c["images"][0], 8, 8, c["w"], 0.0, 0.0, fh.HOG_I32, fh.HOG_I32)


@pytest.mark.parametrize("ii_dtype", ["i32", "u16"])
def test_pipeline_config1(fh, g, ii_dtype):
    c = wl.config1()
    it = fh.HOG_I32 if ii_dtype == "i32" else fh.HOG_U16
    got = compare_pipeline(fh, g, c["images"][0], 8, 4, c["w"], 0.0, c["thr"], it, fh.HOG_I32)
    assert got["count"] > 0


def test_pipeline_end_to_end_host(fh, g):
    c = wl.config1()
    img = c["images"][0]
    pipe = fh.HogPipeline(800, 600, 3, 8, 4)
    pipe.set_weights(c["w"], 0.0, c["thr"])
    pipe.img_host.copy_(torch.from_numpy(img.reshape(-1)))
    det, n = pipe.detect_host()
    ref = oracle.pipeline(img, 8, c["w"], 0.0, 4)
    S_gpu = pipe.scores[: pipe.nx * pipe.ny].cpu().numpy().reshape(pipe.ny, pipe.nx)
    tol = g.score_tolerance(ref["cells"], c["w"], 0.0, stride=4)
    g.check_detections(det, n, S_gpu, ref["scores"], tol, c["thr"], 4)
    # the same from one captured graph, on a second image and then the first again; with the
    # image copied in, and with the bin map reading the page-locked image in place (zero copy)
    img2 = wl.rgb_smooth_shapes(800, 600, wl.rng_for(1, 99))
    for zero_copy in (False, True):
        pipe.capture_host(zero_copy)
        for im in (img2, img):
            det, n = pipe.detect_host(torch.from_numpy(im.reshape(-1)))
            ref = oracle.pipeline(im, 8, c["w"], 0.0, 4)
            assert np.array_equal(pipe.bins.cpu().numpy().reshape(600, 800), ref["bins"])
            S_gpu = pipe.scores[: pipe.nx * pipe.ny].cpu().numpy().reshape(pipe.ny, pipe.nx)
            g.check_detections(det, n, S_gpu, ref["scores"],
                               g.score_tolerance(ref["cells"], c["w"], 0.0, stride=4), c["thr"], 4)


# ---------------------------------------------------------------- tensor-core scores
@pytest.mark.parametrize("nb", [8, 16])
@pytest.mark.parametrize("stride", [8, 4, 2])
def test_score_tensor_cores(fh, g, stride, nb):
    """bf16 cell map -> the tcgen05 implicit-GEMM kernel (N_b = 16: two cell
    halves per window).  bf16 weights: within the FP32-path bound of the
    oracle run on the same bf16-rounded weights; int8 weights: bit-exact.  The
    image spans several window tiles and row bands, with ragged ends in both
    directions."""
    rng = np.random.default_rng(20 + stride + nb)
    img = rand_img(520, 700, 3, 40 + stride)
    cells = cells_of(img, nb, stride)
    w = rng.normal(0, 0.01, 128 * nb).astype(np.float32)
    w_bf = torch.from_numpy(w).to(torch.bfloat16).float().numpy()
    ref = oracle.window_score(cells, w_bf, 0.25, stride=stride)
    with score_engine(fh, 2):
        got = g.gpu_scores(cells, w, fh.HOG_BF16, 0.25, stride=stride, cell_dtype=fh.HOG_BF16)
    assert got.shape == ref.shape
    assert np.all(np.abs(got - ref) <= g.score_tolerance(cells, w_bf, 0.25, stride=stride))
    wi = rng.integers(-127, 128, 128 * nb).astype(np.int8)
    ref_i = oracle.window_score(cells, wi, 3.0, stride=stride)
    for engine in (2, 1):  # tensor cores, then CUDA cores where they apply
        with score_engine(fh, engine):
            got_i = g.gpu_scores(cells, wi, fh.HOG_I8, 3.0, stride=stride, cell_dtype=fh.HOG_BF16)
        assert got_i.dtype == np.int32 and np.array_equal(got_i, ref_i.astype(np.int64)), engine


@pytest.mark.parametrize("nb,stride,F", [(8, 4, 1), (8, 4, 5), (8, 8, 17), (16, 4, 3), (8, 2, 9)])
def test_score_multi_filter(fh, g, nb, stride, F):
    """Several filters in one call: each filter's map equals the oracle's
    (bf16 weights: within the FP32-path bound on the bf16-rounded weights;
    int8: exact) and is bit-identical to scoring that filter alone.  17
    filters exceed one launch group, so the call splits them."""
    rng = np.random.default_rng(200 + 10 * nb + F)
    img = rand_img(330, 420, 3, 60 + stride)
    cells = cells_of(img, nb, stride)
    ncy, ncx, _ = cells.shape
    K = 128 * nb
    r = 8 // stride
    nx, ny = ncx - 7 * r, ncy - 15 * r
    c = torch.from_numpy(cells.astype(np.float32).reshape(-1)).to(torch.bfloat16).cuda()
    W = rng.normal(0, 0.01, (F, K)).astype(np.float32)
    B = rng.normal(0, 0.5, F).astype(np.float32)
    W_bf = torch.from_numpy(W).to(torch.bfloat16)
    ref = oracle.window_score_multi(cells, W_bf.double().numpy(), B, stride=stride)
    out = torch.zeros(F * nx * ny, dtype=torch.float32, device="cuda")
    fh.hog_window_score_multi(c, fh.HOG_BF16, ncx, ncy, nb, 8, 16, 8, stride, W_bf.cuda(), fh.HOG_BF16, F, B, out)
    got = out.cpu().numpy().reshape(F, ny, nx)
    for f in range(F):
        tol = g.score_tolerance(cells, W_bf[f].double().numpy(), float(B[f]), stride=stride)
        assert np.all(np.abs(got[f] - ref[f]) <= tol), f
        one = g.gpu_scores(cells, W[f], fh.HOG_BF16, float(B[f]), stride=stride, cell_dtype=fh.HOG_BF16)
        assert np.array_equal(one, got[f]), f  # the same engine scores a filter alone and with others
    Wi = rng.integers(-127, 128, (F, K)).astype(np.int8)
    Bi = np.round(rng.normal(0, 20, F)).astype(np.float32)
    out_i = torch.zeros(F * nx * ny, dtype=torch.int32, device="cuda")
    fh.hog_window_score_multi(c, fh.HOG_BF16, ncx, ncy, nb, 8, 16, 8, stride, torch.from_numpy(Wi).cuda(),
                              fh.HOG_I8, F, Bi, out_i)
    ref_i = oracle.window_score_multi(cells, Wi.astype(np.float64), Bi, stride=stride)
    assert np.array_equal(out_i.cpu().numpy().reshape(F, ny, nx), ref_i.astype(np.int64))


def test_score_multi_filter_f32(fh, g):
    """f32 weights: the CUDA-core kernel per filter, within the FP32 bound."""
    rng = np.random.default_rng(301)
    img = rand_img(300, 260, 3, 9)
    cells = cells_of(img, 8, 4)
    ncy, ncx, _ = cells.shape
    nx, ny = ncx - 14, ncy - 30
    F = 4
    W = rng.normal(0, 0.01, (F, 1024)).astype(np.float32)
    B = [0.0, 0.5, -0.25, 2.0]
    out = torch.zeros(F * nx * ny, dtype=torch.float32, device="cuda")
    fh.hog_window_score_multi(g.dev(cells.astype(np.float32).reshape(-1)), fh.HOG_F32, ncx, ncy, 8, 8, 16, 8, 4,
                              g.dev(W.reshape(-1)), fh.HOG_F32, F, B, out)
    got = out.cpu().numpy().reshape(F, ny, nx)
    ref = oracle.window_score_multi(cells, W, B, stride=4)
    for f in range(F):
        assert np.all(np.abs(got[f] - ref[f]) <= g.score_tolerance(cells, W[f], B[f], stride=4))


@pytest.mark.parametrize("nb,stride,eps", [(8, 4, 1.0), (16, 4, 0.0), (8, 8, 0.5), (9, 2, 2.0)])
def test_block_norm_and_block_score(fh, g, nb, stride, eps):
    """Overlapping L2-normalised blocks: the block map within 2 ulp-scale of
    the FP64 oracle for every cell dtype, and the 7 x 15-block window score
    (hog_window_score on the block map) within the FP32-path bound."""
    rng = np.random.default_rng(400 + nb + stride)
    img = rand_img(300, 230, 3, 70 + nb)
    cells = cells_of(img, nb, stride)
    ncy, ncx, _ = cells.shape
    r = 8 // stride
    ref = oracle.block_norm(cells, r, eps)
    nby, nbx, k = ref.shape
    for cd in (fh.HOG_I32, fh.HOG_F32, fh.HOG_BF16):
        if cd == fh.HOG_BF16:
            c = torch.from_numpy(cells.astype(np.float32).reshape(-1)).to(torch.bfloat16).cuda()
        else:
            c = g.dev(cells.astype(np.int32 if cd == fh.HOG_I32 else np.float32).reshape(-1))
        out = torch.full((nby * nbx * k + 8,), -3.0, dtype=torch.float32, device="cuda")
        fh.hog_block_norm(c, cd, ncx, ncy, nb, r, eps, out)
        got = out.cpu().numpy()
        assert np.all(got[nby * nbx * k:] == -3.0)
        got = got[: nby * nbx * k].reshape(nby, nbx, k)
        assert np.all(np.abs(got - ref) <= 4e-7 * np.maximum(np.abs(ref), 1e-30) + 1e-12), cd
    w = rng.normal(0, 0.01, 15 * 7 * k).astype(np.float32)
    bl = torch.from_numpy(got.reshape(-1).copy()).cuda()
    ny, nx = nby - 14 * r, nbx - 6 * r
    sc = torch.zeros(max(nx * ny, 1), dtype=torch.float32, device="cuda")
    fh.hog_window_score(bl, fh.HOG_F32, nbx, nby, k, 7, 15, 8, stride, g.dev(w), fh.HOG_F32, 0.3, sc)
    S = sc.cpu().numpy()[: nx * ny].reshape(ny, nx)
    S64 = oracle.block_window_score(ref, w, 0.3, r=r)
    mass = oracle.block_window_score(np.abs(ref), np.abs(w.astype(np.float64)), 0.3, r=r)
    assert np.all(np.abs(S - S64) <= 1e-5 * mass + 1e-6)


# ---------------------------------------------------------------- soft votes
@pytest.mark.parametrize("nb", [4, 8, 9, 16, 64])
def test_soft_lut_exhaustive(fh, g, nb):
    buf = torch.empty(fh.HOG_SOFT_LUT_BYTES // 2, dtype=torch.int16, device="cuda")
    fh.hog_build_soft_lut(nb, buf)
    tab = buf.cpu().numpy().view(np.uint16).reshape(511, 512)
    ref, margin = oracle.soft_lut(nb)
    assert margin > 1e-9
    assert np.all(tab[:, 511] == 0xFFFF)
    assert np.array_equal(tab[:, :511], ref)


@pytest.mark.parametrize("tile_rows", [0, 8, 16])
@pytest.mark.parametrize("ch", [1, 3])
@pytest.mark.parametrize("nb,cell,stride", [(8, 8, 4), (8, 8, 8), (16, 8, 4), (9, 16, 4), (8, 32, 8)])
def test_cells_soft(fh, g, ch, nb, cell, stride, tile_rows):
    """Soft-vote cells from the image in one kernel equal the oracle's direct
    sums of per-pixel votes, on images spanning several tiles with ragged
    edges, in tiles of 8 or 16 cell rows (HOG_TUNE_FUSED_TILE_ROWS; 0: the
    library's choice); the window score over them is within the FP32 bound."""
    buf = torch.empty(fh.HOG_SOFT_LUT_BYTES // 2, dtype=torch.int16, device="cuda")
    fh.hog_build_soft_lut(nb, buf)
    fh.hog_tune_set(fh.HOG_TUNE_FUSED_TILE_ROWS, tile_rows)
    for i, (H, W) in enumerate([(77, 300), (240, 330), (131, 517)]):
        img = rand_img(H, W, ch, 3000 + 10 * nb + i)
        ref = oracle.soft_cells(img, nb, cell, stride)
        ncy, ncx = ref.shape[:2]
        d = g.dev(img.reshape(-1))
        for cd in (fh.HOG_I32, fh.HOG_F32):
            out = torch.full((max(ncx * ncy * nb, 1) + 4,), -1, dtype=fh.TORCH_DTYPE[cd], device="cuda")
            fh.hog_cell_hist_soft(d, W, H, ch, W * ch, buf, nb, cell, stride, cd, out)
            host = out.cpu().numpy()
            assert np.all(host[ncx * ncy * nb:] == -1)
            got = host[: ncx * ncy * nb].astype(np.int64).reshape(ncy, ncx, nb)
            assert np.array_equal(got, ref), (H, W, cd)
    fh.hog_tune_set(fh.HOG_TUNE_FUSED_TILE_ROWS, 0)
    if cell == 8 and stride == 4:
        rng = np.random.default_rng(nb)
        w = rng.normal(0, 0.001, 128 * nb).astype(np.float32)
        S64 = oracle.window_score(ref, w, 0.1, stride=4)
        S = g.gpu_scores(ref, w, fh.HOG_F32, 0.1, stride=4, cell_dtype=fh.HOG_F32)
        assert np.all(np.abs(S - S64) <= g.score_tolerance(ref, w, 0.1, stride=4))


@pytest.mark.parametrize("nb", [8, 16])
@pytest.mark.parametrize("stride", [8, 4, 2])
def test_score_f32_weights_on_tensor_cores(fh, g, stride, nb):
    """f32 weights with bf16 cells run on the tensor cores as three exact
    bf16 parts per weight: within the FP32-path bound of the FP64 oracle run
    on the original f32 weights (no weight rounding), with a large bias too."""
    rng = np.random.default_rng(500 + stride + nb)
    img = rand_img(330, 420, 3, 90 + stride)
    cells = cells_of(img, nb, stride)
    w = rng.normal(0, 0.01, 128 * nb).astype(np.float32)
    w[::7] *= 1e3  # mixed magnitudes: the low parts matter
    for bias in (0.0, -123.25):
        ref = oracle.window_score(cells, w, bias, stride=stride)
        with score_engine(fh, 1):
            cc = g.gpu_scores(cells, w, fh.HOG_F32, bias, stride=stride, cell_dtype=fh.HOG_BF16)
        assert np.all(np.abs(cc - ref) <= g.score_tolerance(cells, w, bias, stride=stride))
        with score_engine(fh, 2):
            got = g.gpu_scores(cells, w, fh.HOG_F32, bias, stride=stride, cell_dtype=fh.HOG_BF16)
        assert got.shape == ref.shape
        tol = g.score_tolerance(cells, w, bias, stride=stride)
        assert np.all(np.abs(got - ref) <= tol)
        # the same weights rounded to bf16 would be far off: the parts are what make it f32-accurate
        w_bf = torch.from_numpy(w).to(torch.bfloat16).float().numpy()
        coarse = oracle.window_score(cells, w_bf, bias, stride=stride)
        assert np.max(np.abs(coarse - ref) / tol) > 10 * np.max(np.abs(got - ref) / tol)


def test_score_bf16_error_against_f32_weights(fh, g):
    """The bf16 path against the FP64 oracle with the original f32 weights:
    the error is the weight rounding (bf16 keeps 8 significant bits, so at
    most 2^-8 sum |w| h) plus the FP32 accumulation; the measured maximum is
    printed."""
    rng = np.random.default_rng(77)
    img = wl.config1()["images"][0]
    cells = cells_of(img, 8, 4)
    w = rng.normal(0, 0.01, 1024).astype(np.float32)
    ref = oracle.window_score(cells, w, 0.0, stride=4)
    got = g.gpu_scores(cells, w, fh.HOG_BF16, 0.0, stride=4, cell_dtype=fh.HOG_BF16)
    mass = oracle.window_score(cells, np.abs(w.astype(np.float64)), 0.0, stride=4)
    err = np.abs(got - ref)
    assert np.all(err <= (2.0 ** -8 + 1e-5) * mass)
    print(f"bf16 scores: max abs error {err.max():.3g}, max relative to sum|w|h {(err[mass > 0] / mass[mass > 0]).max():.3g}")


# ---------------------------------------------------------------- fused image -> cells
@pytest.mark.parametrize("tile_rows", [0, 4, 8, 16])
@pytest.mark.parametrize("table", [1, 2])
@pytest.mark.parametrize("ch", [1, 3])
@pytest.mark.parametrize("nb,cell,stride", [(8, 8, 4), (8, 8, 8), (16, 8, 4), (8, 16, 4), (8, 16, 8)])
def test_cells_fused(fh, g, ch, nb, cell, stride, table, tile_rows):
    """hog_cell_hist_fused equals the oracle's Eq. 6 cell map of the oracle's
    bins, bit for bit, on images spanning several tiles with ragged edges,
    with the table staged in shared memory (1) or read through the cache (2),
    in tiles of 4, 8 or 16 cell rows (HOG_TUNE_FUSED_TILE_ROWS; 0: the
    library's choice)."""
    fh.hog_tune_set(fh.HOG_TUNE_TABLE, table)
    fh.hog_tune_set(fh.HOG_TUNE_FUSED_TILE_ROWS, tile_rows)
    for i, (H, W) in enumerate([(77, 300), (240, 320), (131, 517), (16, 16), (600, 800)]):
        img = rand_img(H, W, ch, 1000 + 10 * nb + i)
        ref = oracle.cell_hist_ii(oracle.integral(oracle.bin_map(img, nb), nb), nb, cell, stride)
        ncy, ncx = ref.shape[:2]
        lut = g.gpu_lut(nb)
        d = g.dev(img.reshape(-1))
        for cd in (fh.HOG_I32, fh.HOG_F32, fh.HOG_BF16):
            out = torch.full((max(ncx * ncy * nb, 1),), -1, dtype=fh.TORCH_DTYPE[cd], device="cuda")
            fh.hog_cell_hist_fused(d, W, H, ch, W * ch, lut, nb, cell, stride, cd, out)
            got = out.float().cpu().numpy()[: ncx * ncy * nb].reshape(ncy, ncx, nb)
            assert np.array_equal(got, ref), (H, W, cd)
    fh.hog_tune_set(fh.HOG_TUNE_TABLE, 0)
    fh.hog_tune_set(fh.HOG_TUNE_FUSED_TILE_ROWS, 0)


@pytest.mark.parametrize("tile_rows", [4, 8, 16])
@pytest.mark.parametrize("cell,stride", [(16, 4), (32, 8)])
def test_cells_fused_single_bin_extremes(fh, g, cell, stride, tile_rows):
    """A diagonal ramp puts every interior pixel in one bin, so the tile-local
    corner sums reach their largest values (r = 4, tiles of 16 rows the
    largest); the counts must still be exact, written at 2-, 4- and 16-byte
    aligned addresses."""
    fh.hog_tune_set(fh.HOG_TUNE_FUSED_TILE_ROWS, tile_rows)
    H, W = 300, 700
    yy, xx = np.mgrid[0:H, 0:W]
    img = ((xx + 2 * yy) % 256).astype(np.uint8)  # (dx, dy) = (2, 4) except at the wrap
    ref = oracle.cell_hist_ii(oracle.integral(oracle.bin_map(img, 8), 8), 8, cell, stride)
    ncy, ncx = ref.shape[:2]
    lut = g.gpu_lut(8)
    d = g.dev(img.reshape(-1))
    n = ncx * ncy * 8
    for cd, shifts in ((fh.HOG_BF16, (0, 1, 2)), (fh.HOG_F32, (0, 1)), (fh.HOG_I32, (0, 3))):
        if cd == fh.HOG_BF16 and cell > 16:
            continue  # counts above 256 are not exact in bf16: the call refuses that combination
        esz = torch.empty(0, dtype=fh.TORCH_DTYPE[cd]).element_size()
        for sh in shifts:  # offsets in elements: 16-byte, 4-byte and 2-byte aligned starts
            buf = torch.full((n + 16,), -1, dtype=fh.TORCH_DTYPE[cd], device="cuda")
            fh.hog_cell_hist_fused(d, W, H, 1, W, lut, 8, cell, stride, cd, buf.data_ptr() + sh * esz)
            host = buf.float().cpu().numpy()
            assert np.array_equal(host[sh: sh + n].reshape(ncy, ncx, 8), ref), (cd, sh)
            assert np.all(host[:sh] == -1) and np.all(host[sh + n:] == -1)
    fh.hog_tune_set(fh.HOG_TUNE_FUSED_TILE_ROWS, 0)


def test_pipeline_fused_config1(fh, g):
    c = wl.config1()
    img = c["images"][0]
    pipe = fh.HogPipeline(800, 600, 3, 8, 4)
    pipe.fused = True
    pipe.set_weights(c["w"], 0.0, c["thr"])
    pipe.set_image(img)
    pipe.run()
    got = pipe.results()
    ref = oracle.pipeline(img, 8, c["w"], 0.0, 4, c["thr"])
    assert np.array_equal(got["cells"], ref["cells"])
    tol = g.score_tolerance(ref["cells"], c["w"], 0.0, stride=4)
    assert np.all(np.abs(got["scores"] - ref["scores"]) <= tol)
    g.check_detections(got["detections"], got["count"], got["scores"], ref["scores"], tol, c["thr"], 4)
