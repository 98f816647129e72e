"""The C-ABI library loads and exports every entry point that include/*.h
declares; host-side argument checks reject bad calls before touching CUDA.
No compute call is made here (this runs without a GPU)."""

import ctypes
import glob
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADERS = sorted(glob.glob(os.path.join(ROOT, "include", "*.h")))


def declared_functions():
    src = "".join(open(h).read() for h in HEADERS)
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"^\s*(?:const\s+)?[a-z_0-9]+\*?\s+\*?(hog_[a-z_0-9]+)\s*\(", src, flags=re.M)))


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


def test_header_declares_the_six_stage_calls():
    names = declared_functions()
    for n in ["hog_build_lut", "hog_bin_map", "hog_integral", "hog_cell_hist", "hog_window_score", "hog_detect"]:
        assert n in names


def test_library_exports_every_declared_symbol(fh):
    lib = ctypes.CDLL(fh.LIB_PATH)
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, missing
    assert set(fh.EXPORTED) == set(declared_functions())


def test_version_and_strings(fh):
    assert fh.hog_version() >= 100
    assert fh.lib().hog_status_string(fh.HOG_ERR_ARG) == b"HOG_ERR_ARG"


def test_workspace_sizes(fh):
    assert fh.hog_integral_workspace_bytes(800, 600, 8) > 0
    assert fh.hog_integral_workspace_bytes(0, 600, 8) == 0
    assert fh.hog_integral_workspace_bytes(800, 600, 0) == 0
    assert fh.hog_detect_workspace_bytes(185, 119) >= 4 * 11
    assert fh.hog_detect_workspace_bytes(-1, 5) == 0


def test_argument_errors_need_no_gpu(fh):
    L = fh.lib()
    ARG = fh.HOG_ERR_ARG
    assert L.hog_build_lut(8, None, None) == ARG
    assert L.hog_build_lut(0, 4096, None) == ARG
    assert L.hog_build_lut(65, 4096, None) == ARG
    assert L.hog_build_lut(8, 4097, None) == ARG  # table must be 16-byte aligned
    assert L.hog_bin_map(None, 8, 8, 1, 8, 4096, 8, 4096, None) == ARG
    assert L.hog_bin_map(4096, 8, 8, 2, 16, 4096, 8, 4096, None) == ARG      # channels
    assert L.hog_bin_map(4096, 8, 8, 3, 23, 4096, 8, 4096, None) == ARG      # pitch < 3W
    assert L.hog_bin_map(4096, 0, 8, 1, 8, 4096, 8, 4096, None) == ARG       # W
    assert L.hog_integral(4096, 8, 8, 8, fh.HOG_F32, 4096, 4096, 1 << 20, None) == ARG  # dtype
    assert L.hog_integral(4096, 8, 8, 8, fh.HOG_I32, 4096, 4096, 0, None) == ARG        # workspace
    assert L.hog_integral(4096, 8, 8, 8, fh.HOG_I32, 4096, 4097, 1 << 20, None) == ARG  # alignment
    assert L.hog_cell_hist(4096, 64, 64, 8, fh.HOG_I32, 8, 9, fh.HOG_I32, 4096, None) == ARG  # stride > cell
    assert L.hog_cell_hist(4096, 64, 64, 8, fh.HOG_I32, 32, 8, fh.HOG_BF16, 4096, None) == ARG  # bf16, cell 32
    assert L.hog_window_score(4096, fh.HOG_I32, 10, 10, 8, 8, 16, 8, 3, 4096, fh.HOG_F32, 0.0, 4096, None) == ARG
    assert L.hog_window_score(4096, fh.HOG_I32, 10, 10, 8, 8, 16, 8, 4, 4096, fh.HOG_U8, 0.0, 4096, None) == ARG
    assert L.hog_window_score(4096, fh.HOG_I32, 10, 10, 8, 8, 16, 8, 4, 4096, fh.HOG_F32, float("nan"), 4096,
                              None) == ARG
    assert L.hog_detect(4096, fh.HOG_F32, 10, 10, 4, 0.5, 0, 0, 4096, 10, 4096, 4096, 0, None) == ARG
    assert L.hog_detect(4096, fh.HOG_BF16, 10, 10, 4, 0.5, 0, 0, 4096, 10, 4096, 4096, 256, None) == ARG
    assert L.hog_detect(None, fh.HOG_F32, 10, 10, 4, 0.5, 0, 0, 4096, 10, 4096, 4096, 256, None) == ARG
    assert L.hog_device_status(None, 0) == ARG
    assert L.hog_selftest_wait_timeout(2, 1000, None) == ARG
    assert L.hog_selftest_wait_timeout(0, 0, None) == ARG


def test_int8_scores_outside_the_exact_range_are_refused(fh):
    # int8 weights promise exact int32 scores; f32 accumulation keeps that only
    # while 127 * cells_x * cells_y * cell^2 + |round(bias)| < 2^24
    L = fh.lib()
    UNS = fh.HOG_ERR_UNSUPPORTED
    # cell 64, 8 x 16 cells: 127 * 128 * 4096 = 66,584,576 >= 2^24
    assert L.hog_window_score(4096, fh.HOG_I32, 200, 200, 8, 8, 16, 64, 64, 4096, fh.HOG_I8, 0.0, 4096,
                              None) == UNS
    # cell 32: 127 * 128 * 1024 = 16,646,144 < 2^24, but a bias of 2^17 pushes it over
    assert L.hog_window_score(4096, fh.HOG_I32, 200, 200, 8, 8, 16, 32, 32, 4096, fh.HOG_I8, 131072.0, 4096,
                              None) == UNS
    biases = (ctypes.c_float * 2)(0.0, 131072.0)
    assert L.hog_window_score_multi(4096, fh.HOG_I32, 200, 200, 8, 8, 16, 32, 32, 4096, fh.HOG_I8, 2, biases,
                                    4096, None) == UNS


def test_server_argument_errors_need_no_gpu(fh):
    L = fh.lib()
    ARG = fh.HOG_ERR_ARG
    good = dict(n_bins=8, cell=8, stride=4, cells_x=8, cells_y=16, w_dtype=fh.HOG_BF16, bias=0.0, thr=0.5,
                fused=-1, ii_dtype=fh.HOG_I32, n_slots=4, budget_bytes=1 << 20, max_W=640, max_H=480)
    h = ctypes.c_void_p(1)
    w = (ctypes.c_uint16 * (8 * 16 * 8))()
    assert L.hog_server_create(None, w, ctypes.byref(h)) == ARG and h.value is None
    assert L.hog_server_create(ctypes.byref(fh.HogServerConfig(**good)), None, ctypes.byref(h)) == ARG
    for bad in (dict(n_bins=0), dict(stride=3), dict(cells_x=0), dict(w_dtype=fh.HOG_U8), dict(fused=2),
                dict(ii_dtype=fh.HOG_F32), dict(n_slots=0), dict(n_slots=65), dict(budget_bytes=0),
                dict(max_W=0), dict(thr=float("nan")), dict(bias=float("inf")), dict(image_in_place=2),
                dict(image_in_place=-1)):
        cfg = fh.HogServerConfig(**{**good, **bad})
        assert L.hog_server_create(ctypes.byref(cfg), w, ctypes.byref(h)) == ARG, bad
    cfg = fh.HogServerConfig(**{**good, "fused": 1, "n_bins": 9})  # the fused call takes N_b 8 or 16
    assert L.hog_server_create(ctypes.byref(cfg), w, ctypes.byref(h)) == fh.HOG_ERR_UNSUPPORTED
    ok = ctypes.c_int(7)
    assert L.hog_server_submit(None, 0, 4096, 64, 128, 3, ctypes.byref(ok)) == ARG
    n = ctypes.c_int(0)
    assert L.hog_server_poll(None, None, 0, ctypes.byref(n)) == ARG
    assert L.hog_server_release(None, 0) == ARG
    assert L.hog_server_stats(None, None, None, None) == ARG
    assert L.hog_server_pauses(None, None, None, 0, ctypes.byref(n)) == ARG
    assert L.hog_server_request_bytes(None, 64, 128, 3) == 0
    assert L.hog_server_destroy(None) == fh.HOG_OK


def test_batch_plan_on_the_host(fh):
    """hog_batch_plan is host arithmetic; bad plans and arguments are refused
    before anything is enqueued."""
    item = fh.HogBatchItem(4096, 640 * 3, 640, 480, 4096, 8192, 0, 0)
    small = fh.HogBatchItem(4096, 60 * 3, 60, 100, 4096, 0, 1, 0)  # smaller than a window: no scores needed
    plan = fh.hog_batch_plan([item, small], 3, 8, 8, 4, 8, 16)
    assert len(bytes(plan)) == fh.hog_batch_plan_bytes(2) == 64 + 2 * 96
    with pytest.raises(fh.HogError):
        fh.hog_batch_plan([item], 3, 9, 8, 4, 8, 16)  # N_b 9: no fused kernel
    with pytest.raises(fh.HogError):
        fh.hog_batch_plan([fh.HogBatchItem(4096, 100, 640, 480, 4096, 8192, 0, 0)], 3, 8, 8, 4, 8, 16)  # pitch
    with pytest.raises(fh.HogError):
        fh.hog_batch_plan([fh.HogBatchItem(4096, 640 * 3, 640, 480, 4096, 0, 0, 0)], 3, 8, 8, 4, 8, 16)  # scores
    assert fh.hog_batch_plan_bytes(0) == 0
    junk = (ctypes.c_uint64 * 32)()
    L = fh.lib()
    ARG = fh.HOG_ERR_ARG
    assert L.hog_cell_hist_fused_batch(junk, 4096, 4096, fh.HOG_BF16, None) == ARG  # not a plan
    assert L.hog_cell_hist_fused_batch(plan, 4100, 4096, fh.HOG_BF16, None) == ARG  # device copy misaligned
    assert L.hog_cell_hist_fused_batch(plan, 4096, 4100, fh.HOG_BF16, None) == ARG  # table misaligned
    assert L.hog_window_score_batch(plan, 4096, fh.HOG_BF16, None, fh.HOG_BF16, 0.0, None) == ARG
    assert fh.hog_detect_batch_workspace_bytes(plan) > 0
    assert L.hog_detect_batch(plan, 4096, fh.HOG_F32, 0.5, 4096, 10, 4096, None, 4096, 0, None) == ARG  # workspace
    assert fh.hog_pyramid_bytes(640, 480, 3, 3) == 320 * 240 * 3 + 160 * 120 * 3
    assert fh.hog_pyramid_bytes(640, 480, 3, 1) == 0
    assert L.hog_pyramid(None, 640, 480, 3, 1920, 3, 4096, None) == ARG
    assert L.hog_pyramid(4096, 640, 480, 3, 100, 3, 4096, None) == ARG  # pitch


def header_enum(name):
    """name -> value of the enumerators of the typedef'd enum `name` in include/*.h."""
    src = "".join(open(h).read() for h in HEADERS)
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    end = re.search(r"\}\s*" + name + r"\s*;", src)
    assert end, name
    body = src[src.rindex("typedef enum", 0, end.start()):end.start()]  # the last enum opened before it
    out = {}
    for k, v in re.findall(r"(HOG_[A-Z0-9_]+)\s*=\s*(-?\d+)", body):
        out[k] = int(v)
    return out


def test_binding_constants_match_the_header(fh):
    """The binding's knob numbers and the header's enum are one list: every
    knob the header declares has the same number in Python, and the autotuner
    only names knobs below HOG_TUNE_KNOBS, each once."""
    knobs = header_enum("hog_tune_knob")
    assert knobs, "no knobs parsed"
    for k, v in knobs.items():
        assert getattr(fh, k) == v, k
    n = knobs["HOG_TUNE_KNOBS"]
    assert sorted(v for k, v in knobs.items() if k != "HOG_TUNE_KNOBS") == list(range(n))
    from paper_1703_06256_gb300 import autotune

    ids = [knob for knob, _ in autotune.KNOBS.values()]
    assert len(ids) == len(set(ids)) and all(0 <= i < n for i in ids)
    for names in autotune.PATH_KNOBS.values():
        assert set(names) <= set(autotune.KNOBS)
