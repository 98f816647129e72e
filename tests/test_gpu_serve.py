"""Continuous batching: every request's detections are the same whether it is
served alone or in a mix of overlapping requests of other sizes, and equal
to the oracle's decision (within the float tolerance band)."""

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

import oracle  # noqa: E402
import workloads as wl  # noqa: E402


@pytest.mark.parametrize("fused", [True, False])
def test_same_alone_and_in_the_mix(fused):
    import paper_1703_06256_gb300 as fh
    from paper_1703_06256_gb300.serve import HogServer, Request

    rng = wl.rng_for(4)
    w = wl.weights_f32(8, rng)
    sizes = [(320, 240), (800, 600), (1000, 704), (512, 512), (1280, 720), (640, 480), (400, 1000), (96, 160)]
    images = [wl.rgb_smooth_shapes(W, H, rng, n_shapes=6) for (W, H) in sizes]
    srv = HogServer(w, 0.0, 0.5, w_dtype=fh.HOG_F32, budget_bytes=256 << 20, n_streams=4, fused=fused)
    alone = {i: srv.run_one(img, i) for i, img in enumerate(images)}
    mix = srv.serve([Request(i, img, 0.0) for i, img in enumerate(images)])
    assert sorted(r.rid for r in mix) == list(range(len(images)))
    assert srv.idle() and srv.used == 0
    for r in mix:
        a = alone[r.rid]
        assert r.count == a.count
        assert np.array_equal(r.detections, a.detections)
        assert np.all(r.detections["image"] == r.rid)
    # and against the oracle: same windows except within the tolerance band of the threshold
    for i, img in enumerate(images):
        ref = oracle.pipeline(img, 8, w, 0.0, 4)
        S = ref["scores"]
        if S.size == 0:
            assert alone[i].count == 0
            continue
        tol = 1e-5 * oracle.window_score(np.abs(ref["cells"]), np.abs(w.astype(np.float64)), 0.0, stride=4)
        got = np.zeros(S.shape, bool)
        d = alone[i].detections
        got[d["y"] // 4, d["x"] // 4] = True
        far = np.abs(S - 0.5) > tol
        assert np.array_equal(got[far], (S >= 0.5)[far])
