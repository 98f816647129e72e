"""Continuous batching (the library's request server): every request's
detections are the same whether it is served alone or in a mix of
overlapping requests of other sizes, and match the oracle's decision outside
the float tolerance band of the threshold."""

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

import oracle  # noqa: E402
import workloads as wl  # noqa: E402

SIZES = [(320, 240), (800, 600), (1000, 704), (512, 512), (1280, 720), (640, 480), (400, 1000), (96, 160),
         (48, 200), (64, 128)]


def _images(rng):
    imgs = [wl.rgb_smooth_shapes(W, H, rng, n_shapes=6) for (W, H) in SIZES]
    imgs[5] = imgs[5].max(axis=2).copy()  # one gray request
    return imgs


def _check_vs_oracle(img, w, bias, thr, res):
    ref = oracle.pipeline(img, 8, w, bias, 4)
    S = ref["scores"]
    if S.size == 0:
        assert res.count == 0
        return
    tol = 1e-5 * (oracle.window_score(np.abs(ref["cells"]), np.abs(w.astype(np.float64)), 0.0, stride=4) + abs(bias))
    got = np.zeros(S.shape, bool)
    d = res.detections
    got[d["y"] // 4, d["x"] // 4] = True
    far = np.abs(S - thr) > tol
    assert np.array_equal(got[far], (S >= thr)[far])
    assert np.all(d["score"] >= thr)


@pytest.mark.parametrize("fused,budget,streams", [(True, 8 << 20, 4), (False, 96 << 20, 3)])
def test_same_alone_and_in_the_mix(fused, budget, streams):
    import paper_1703_06256_gb300 as fh
    from paper_1703_06256_gb300.serve import HogServer, Request

    rng = wl.rng_for(4)
    w = wl.weights_f32(8, rng)
    images = _images(rng)
    srv = HogServer(w, 0.0, 0.5, w_dtype=fh.HOG_F32, budget_bytes=budget, n_streams=streams, fused=fused,
                    max_wh=(1280, 1000))
    need = [srv.working_set(im.shape[1], im.shape[0], 1 if im.ndim == 2 else 3) for im in images]
    assert max(need) <= budget < sum(need)  # the budget, not only the slots, limits admission
    alone = {i: srv.run_one(img, i) for i, img in enumerate(images)}
    mix = srv.serve([Request(i, img, 0.0) for i, img in enumerate(images)])
    assert sorted(r.rid for r in mix) == list(range(len(images)))
    assert srv.idle() and srv.used == 0
    for r in mix:
        a = alone[r.rid]
        assert r.count == a.count == len(r.detections)
        assert np.array_equal(r.detections, a.detections)
        assert np.all(r.detections["image"] == r.rid)
        assert r.shape == images[r.rid].shape[:2]
    for i, img in enumerate(images):
        _check_vs_oracle(img, w, 0.0, 0.5, alone[i])
    srv.close()


@pytest.mark.parametrize("fused", [True, False])
def test_native_dispatcher_same_as_alone(fused):
    """The server's own dispatcher thread (hog_server_start / enqueue /
    collect): requests queued at staggered arrival times, under a budget that
    holds only some of them at once, give the same lists as each alone; the
    native stamps are ordered (enqueue <= admit <= done); the synchronous
    calls are refused while the thread runs."""
    import paper_1703_06256_gb300 as fh
    from paper_1703_06256_gb300.serve import HogServer, Request

    rng = wl.rng_for(4)
    w = wl.weights_f32(8, rng)
    images = _images(rng)
    budget = 8 << 20 if fused else 96 << 20
    srv = HogServer(w, 0.0, 0.5, w_dtype=fh.HOG_F32, budget_bytes=budget, n_streams=4, fused=fused,
                    max_wh=(1280, 1000))
    alone = {i: srv.run_one(img, i) for i, img in enumerate(images)}
    reqs = [Request(i, img, 0.0005 * (i % 4)) for i, img in enumerate(images * 3)]
    mix, replay = srv.serve_native(reqs)
    assert sorted(r.rid for r in mix) == list(range(len(reqs)))
    assert replay["replay_late_p99_ms"] >= 0
    # the dispatcher's pause record: stamps in order, within the run
    n_pauses, pauses = fh.hog_server_pauses(srv._h)
    assert n_pauses == replay["dispatcher_pauses"] >= len(pauses)
    first, last = min(r.t_enqueue_ns for r in mix), max(r.t_done_ns for r in mix)
    assert all(first - 10**9 < a < b <= last + 10**9 and b - a > 10**6 for a, b in pauses)
    assert all(r.t_enqueue_ns <= r.t_done_ns for r in mix)
    for r in mix:
        a = alone[r.rid % len(images)]
        assert r.count == a.count == len(r.detections)
        assert np.array_equal(r.detections["x"], a.detections["x"])
        assert np.array_equal(r.detections["score"], a.detections["score"])
        assert np.all(r.detections["image"] == r.rid)
        assert r.latency > 0
    assert srv.idle() and srv.used == 0
    # while the dispatcher runs, the caller-driven calls are refused
    fh.hog_server_start(srv._h)
    try:
        with pytest.raises(fh.HogError):
            srv.try_submit(Request(0, images[0]))
    finally:
        fh.hog_server_stop(srv._h)
    srv.close()


def test_int8_weights_exact_in_the_mix():
    """Integer weights: scores are exact, so the lists equal the oracle's exactly."""
    import paper_1703_06256_gb300 as fh
    from paper_1703_06256_gb300.serve import HogServer, Request

    rng = wl.rng_for(6)
    w = wl.weights_i8(8, rng)
    images = _images(rng)
    thr = 40.0
    srv = HogServer(w, 3.0, thr, w_dtype=fh.HOG_I8, budget_bytes=512 << 20, n_streams=6, max_wh=(1280, 1000))
    mix = srv.serve([Request(i, img, 0.0) for i, img in enumerate(images)])
    for r in mix:
        ref = oracle.pipeline(images[r.rid], 8, w.astype(np.float64), 3.0, 4)
        S = ref["scores"]
        ys, xs = np.nonzero(S >= thr) if S.size else (np.zeros(0, int), np.zeros(0, int))
        assert r.count == len(ys)
        assert np.array_equal(r.detections["x"], xs * 4) and np.array_equal(r.detections["y"], ys * 4)
        assert np.array_equal(r.detections["score"], S[ys, xs].astype(np.float32))
    srv.close()


def test_oversize_request_is_refused():
    import paper_1703_06256_gb300 as fh
    from paper_1703_06256_gb300.serve import HogServer, Request

    w = wl.weights_f32(8, wl.rng_for(4))
    srv = HogServer(w, 0.0, 0.5, w_dtype=fh.HOG_F32, budget_bytes=1 << 20, n_streams=2, max_wh=(640, 480))
    img = np.zeros((480, 641, 3), np.uint8)  # wider than max_W
    with pytest.raises(fh.HogError):
        srv.try_submit(Request(0, img))
    img = np.zeros((480, 640, 3), np.uint8)  # fits the size limit, not the 1 MiB budget
    assert srv.working_set(640, 480, 3) > 1 << 20
    with pytest.raises(fh.HogError):
        srv.try_submit(Request(1, img))
    assert srv.idle()
    srv.close()


@pytest.mark.parametrize("fused", [True, False])
def test_images_read_in_place(fused):
    """image_in_place: page-locked request images are read in place by the
    first kernel (no copy is enqueued), pageable ones are still copied in;
    every request's list equals the copying server's, with the dispatcher
    thread and without it."""
    import paper_1703_06256_gb300 as fh
    from paper_1703_06256_gb300.serve import HogServer, Request

    rng = wl.rng_for(4)
    w = wl.weights_f32(8, rng)
    images = _images(rng)
    mixed = [torch.from_numpy(np.ascontiguousarray(im)).pin_memory() if i % 2 == 0 else im
             for i, im in enumerate(images)]
    kw = dict(w_dtype=fh.HOG_F32, budget_bytes=96 << 20, n_streams=4, fused=fused, max_wh=(1280, 1000))
    ref = HogServer(w, 0.0, 0.5, **kw)
    want = {r.rid: r for r in ref.serve([Request(i, im, 0.0) for i, im in enumerate(images)])}
    ref.close()
    srv = HogServer(w, 0.0, 0.5, image_in_place=True, **kw)
    got_sync = srv.serve([Request(i, im, 0.0) for i, im in enumerate(mixed)])
    got_native, _ = srv.serve_native([Request(i, im, 0.0005 * i) for i, im in enumerate(mixed)])
    for got in (got_sync, got_native):
        assert sorted(r.rid for r in got) == list(range(len(images)))
        for r in got:
            a = want[r.rid]
            assert r.count == a.count
            assert np.array_equal(r.detections, a.detections)
    srv.close()
