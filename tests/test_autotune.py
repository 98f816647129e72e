"""Host logic of the autotuner: the coordinate-descent search, the cache,
and the knob calls of the library (no GPU needed)."""

import json
import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def at():
    import importlib.util

    spec = importlib.util.spec_from_file_location("_fasthog_build", os.path.join(ROOT, "paper_1703_06256_gb300",
                                                                                  "build.py"))
    b = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(b)
    b.build()
    sys.path.insert(0, ROOT)
    from paper_1703_06256_gb300 import autotune

    yield autotune
    autotune.reset()


def test_search_finds_the_separable_optimum(at):
    cand = {"a": (0, 4, 8, 16, 32), "b": (0, 1, 2, 4), "c": (0, 16, 32)}
    opt = {"a": 16, "b": 2, "c": 32}
    calls = []

    def cost(cfg):
        calls.append(json.dumps(cfg, sort_keys=True))
        return 1.0 + sum((cand[k].index(v) - cand[k].index(opt[k])) ** 2 for k, v in cfg.items())

    best, t, seen = at.search(cand, cost)
    assert best == opt and t == 1.0
    assert len(calls) == len(set(calls)) == len(seen)  # no configuration measured twice
    assert json.dumps({"a": 0, "b": 0, "c": 0}, sort_keys=True) in seen  # the defaults are always measured


def test_search_keeps_the_default_when_nothing_is_faster(at):
    best, t, seen = at.search({"a": (0, 4, 8)}, lambda cfg: 1.0 + cfg["a"])
    assert best == {"a": 0} and t == 1.0 and len(seen) == 3


def test_cache_roundtrip(at, tmp_path):
    path = str(tmp_path / "tune.json")
    n = []

    def measure(cfg):
        n.append(cfg)
        return 2.0 - 0.5 * (cfg["score_tc_rows"] == 32) - 0.25 * (cfg["fused_ctas_per_sm"] == 1)

    t1 = at.Autotuner(path, device_name="GB300-test")
    e = t1.tune({"W": 800, "H": 600, "path": "fused"}, measure, at.PATH_KNOBS["fused"])
    assert e["config"] == {"fused_ctas_per_sm": 1, "fused_tile_rows": 0, "score_path": 0, "score_tc_rows": 32,
                           "slide_windows": 0, "table": 0}
    assert e["default_ms"] == 2.0 and e["ms"] == 1.25
    k = len(n)
    t2 = at.Autotuner(path, device_name="GB300-test")
    assert t2.tune({"H": 600, "W": 800, "path": "fused"}, measure, at.PATH_KNOBS["fused"]) == e
    assert len(n) == k  # served from the cache
    t3 = at.Autotuner(path, device_name="other-gpu")
    t3.tune({"W": 800, "H": 600, "path": "fused"}, measure, at.PATH_KNOBS["fused"])
    assert len(n) > k  # another device is another key


def test_knob_calls(at):
    import paper_1703_06256_gb300 as fh

    at.apply({"integral_band_rows": 8, "score_tc_rows": 32})
    assert at.current()["integral_band_rows"] == 8 and at.current()["score_tc_rows"] == 32
    for name, (_, vals) in at.KNOBS.items():
        for v in vals:
            at.apply({name: v})
            assert at.current()[name] == v
    with pytest.raises(fh.HogError):
        fh.hog_tune_set(fh.HOG_TUNE_INTEGRAL_BAND_ROWS, 12)
    with pytest.raises(fh.HogError):
        fh.hog_tune_set(fh.HOG_TUNE_FUSED_CTAS_PER_SM, 3)
    with pytest.raises(fh.HogError):
        fh.hog_tune_set(fh.HOG_TUNE_BINMAP_SCHEDULE, 3)
    with pytest.raises(fh.HogError):
        fh.hog_tune_set(fh.HOG_TUNE_FUSED_TILE_ROWS, 12)
    with pytest.raises(fh.HogError):
        fh.hog_tune_set(17, 1)
    assert fh.hog_tune_get(17) == -1
    at.reset()
    assert all(v == 0 for v in at.current().values())
