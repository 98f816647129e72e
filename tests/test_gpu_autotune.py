"""The launch-shape knobs change no result: the whole path gives the same
bins, integral images, cells, scores and detections under every knob value
(the score engine knob: the same integers, and float scores within the FP32
bound); and the tuner returns a valid configuration."""

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

import oracle  # noqa: E402
import workloads as wl  # noqa: E402


def run(fh, img, w, fused, w_dtype, cell_dtype):
    H, W = img.shape[:2]
    p = fh.HogPipeline(W, H, 3, 8, 4, cell_dtype=cell_dtype, w_dtype=w_dtype)
    p.fused = fused
    p.set_weights(w, 0.0, 0.5)
    p.set_image(img)
    p.run()
    return p.results()


@pytest.mark.parametrize("fused", [False, True])
def test_knobs_change_no_result(fused):
    import paper_1703_06256_gb300 as fh
    from paper_1703_06256_gb300 import autotune

    rng = wl.rng_for(12)
    img = wl.rgb_smooth_shapes(1000, 700, rng, n_shapes=6)
    w = wl.weights_f32(8, rng)
    autotune.reset()
    ref = run(fh, img, w, fused, fh.HOG_BF16, fh.HOG_BF16)
    try:
        for name in autotune.PATH_KNOBS["fused" if fused else "separate"]:
            for v in autotune.KNOBS[name][1]:
                autotune.apply({name: v})
                got = run(fh, img, w, fused, fh.HOG_BF16, fh.HOG_BF16)
                keys = ("cells",) if fused else ("bins", "ii", "cells")
                for k in keys:
                    assert np.array_equal(np.asarray(got[k]), np.asarray(ref[k])), (name, v, k)
                autotune.apply({name: 0})
                if name == "score_path":  # another engine: another f32 summation order
                    mass = oracle.window_score(np.abs(ref["cells"]), np.abs(w.astype(np.float64)), 0.0, stride=4)
                    assert np.all(np.abs(got["scores"] - ref["scores"]) <= 2e-5 * mass), (name, v)
                    continue
                assert np.array_equal(got["scores"], ref["scores"]) and got["count"] == ref["count"], (name, v)
                assert np.array_equal(got["detections"], ref["detections"]), (name, v)
    finally:
        autotune.reset()


def test_tune_pipeline(tmp_path):
    import paper_1703_06256_gb300 as fh
    from paper_1703_06256_gb300 import autotune

    rng = wl.rng_for(13)
    img = wl.rgb_smooth_shapes(800, 600, rng, n_shapes=6)
    p = fh.HogPipeline(800, 600, 3, 8, 4, cell_dtype=fh.HOG_BF16, w_dtype=fh.HOG_BF16)
    p.set_weights(wl.weights_f32(8, rng), 0.0, 0.5)
    p.set_image(img)
    try:
        tuner = autotune.Autotuner(str(tmp_path / "t.json"))
        e = autotune.tune_pipeline(p, tuner, reps=3)
        assert set(e["config"]) == set(autotune.PATH_KNOBS["separate"])
        assert e["ms"] <= e["default_ms"] and e["measured"] >= 1
        assert autotune.current()["integral_band_rows"] == e["config"]["integral_band_rows"]
        assert (tmp_path / "t.json").exists()
    finally:
        autotune.reset()
