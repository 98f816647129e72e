"""The batch calls (include/fasthog_batch.h) against the oracle: pyramid
levels bit-exact against repeated 2:1 decimation; per item, cells bit-exact,
scores within the stated tolerance (exact for int8 weights), and one
detection list in (item, row-major) order with the item's tags and counts;
and identical to the per-image calls on each item."""

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

import oracle  # noqa: E402
import workloads as wl  # noqa: E402

SIZES = [(320, 240), (200, 150), (640, 480), (64, 128), (48, 300), (513, 271), (1000, 130), (130, 1000)]


@pytest.fixture(scope="module")
def fh():
    import paper_1703_06256_gb300 as m

    assert torch.cuda.is_available()
    m.hog_device_status(clear=True)
    yield m
    assert m.hog_device_status() == 0, "a kernel reported a timed-out wait"


def images(ch, seed):
    rng = wl.rng_for(7, seed)
    out = []
    for (W, H) in SIZES:
        img = wl.rgb_smooth_shapes(W, H, rng, n_shapes=5)
        out.append(img if ch == 3 else img.max(axis=2).copy())
    return out


def levels_of(img, levels):
    out = [img]
    for _ in range(1, levels):
        if min(out[-1].shape[:2]) < 2:
            break
        out.append(oracle.decimate(out[-1]))
    return out


@pytest.mark.parametrize("ch", [1, 3])
def test_pyramid_matches_decimation(fh, ch):
    rng = np.random.default_rng(5)
    for (H, W) in [(480, 640), (271, 513), (7, 9), (1, 5), (130, 1000)]:
        img = rng.integers(0, 256, size=(H, W) if ch == 1 else (H, W, 3), dtype=np.uint8)
        for levels in (1, 2, 4):
            nbytes = fh.hog_pyramid_bytes(W, H, ch, levels)
            out = torch.full((max(nbytes, 1) + 64,), 0x5A, dtype=torch.uint8, device="cuda")
            d = torch.from_numpy(img.reshape(-1)).cuda()
            fh.hog_pyramid(d, W, H, ch, W * ch, levels, out)
            host = out.cpu().numpy()
            off = 0
            for lv, ref in enumerate(levels_of(img, levels)):
                if lv == 0:
                    continue
                n = ref.size
                assert ref.shape[:2] == (H >> lv, W >> lv)
                assert np.array_equal(host[off: off + n], ref.reshape(-1)), (H, W, levels, lv)
                off += n
            assert off == nbytes and np.all(host[off:] == 0x5A)


def check_batch(fh, b, imgs, w_eff, bias, thr, exact):
    """Items against the oracle on the pyramid levels of `imgs`."""
    got = b.results()
    dets = got["detections"]
    lists = []
    for m, it in zip(b.item_meta, got["items"]):
        lvl = levels_of(imgs[m["image"]], b.levels)[m["level"]]
        ref = oracle.pipeline(lvl, b.n_bins, w_eff, bias, b.stride)
        assert np.array_equal(it["cells"], ref["cells"]), (m["image"], m["level"])
        S, S64 = it["scores"], ref["scores"]
        assert S.shape == S64.shape
        if S.size:
            if exact:
                assert np.array_equal(S.astype(np.int64), S64.astype(np.int64))
            else:
                tol = 1e-5 * (oracle.window_score(np.abs(ref["cells"]), np.abs(w_eff), 0.0, stride=b.stride)
                              + abs(bias))
                assert np.all(np.abs(S - S64) <= tol)
        ys, xs = np.nonzero(S >= thr) if S.size else (np.zeros(0, int), np.zeros(0, int))
        lists.append((xs * b.stride, ys * b.stride, S[ys, xs] if S.size else np.zeros(0), m["image"], m["level"]))
    # one list: items in plan order, each item's windows row-major (decided on the GPU's own scores)
    assert got["count"] == sum(len(x[0]) for x in lists) == len(dets)
    assert np.array_equal(got["item_counts"], [len(x[0]) for x in lists])
    k = 0
    for xs, ys, sc, img_i, lv in lists:
        part = dets[k: k + len(xs)]
        assert np.array_equal(part["x"], xs) and np.array_equal(part["y"], ys)
        assert np.array_equal(part["score"], np.asarray(sc, np.float32))
        assert np.all(part["image"] == img_i) and np.all(part["level"] == lv)
        k += len(xs)


@pytest.mark.parametrize("ch", [3, 1])
def test_batch_pyramid_bf16(fh, ch):
    from paper_1703_06256_gb300.batch import HogPlanBatch

    imgs = images(ch, 1)
    rng = wl.rng_for(8)
    w = wl.weights_f32(8, rng)
    w_bf = torch.from_numpy(w).to(torch.bfloat16).double().numpy()  # the weights the tensor cores see
    b = HogPlanBatch([(W, H) for (W, H) in SIZES], channels=ch, levels=3, n_bins=8, stride=4)
    b.set_images(imgs)
    b.set_weights(w, 0.0, 0.5)
    b.capture()
    b.run()
    b.run()  # a second replay gives the same results
    check_batch(fh, b, imgs, w_bf, 0.0, 0.5, exact=False)


def test_batch_int8_exact(fh):
    from paper_1703_06256_gb300.batch import HogPlanBatch

    imgs = images(3, 2)
    rng = wl.rng_for(9)
    w = wl.weights_i8(8, rng)
    b = HogPlanBatch(SIZES, channels=3, levels=2, n_bins=8, stride=4, w_dtype=fh.HOG_I8)
    b.set_images(imgs)
    b.set_weights(w, 3.0, 40.0)
    b.run()
    check_batch(fh, b, imgs, w.astype(np.float64), 3.0, 40.0, exact=True)


def test_batch_nb16_tensor_cores_bf16(fh):
    """N_b = 16 with bf16 weights: the batched tensor-core score with two
    16-byte halves per cell (the kernel the pyramid benchmark times at
    N_b = 16), three pyramid levels, against the oracle on the bf16 weights."""
    from paper_1703_06256_gb300.batch import HogPlanBatch

    imgs = images(3, 12)
    w = wl.weights_f32(16, wl.rng_for(12))
    w_bf = torch.from_numpy(w).to(torch.bfloat16).double().numpy()  # the weights the tensor cores see
    b = HogPlanBatch(SIZES, channels=3, levels=3, n_bins=16, stride=4, w_dtype=fh.HOG_BF16)
    assert b.cell_dtype == fh.HOG_BF16
    b.set_images(imgs)
    b.set_weights(w, 0.125, 0.5)
    b.capture()
    b.run()
    check_batch(fh, b, imgs, w_bf, 0.125, 0.5, exact=False)


def test_batch_nb16_tensor_cores_int8_exact(fh):
    """N_b = 16 with int8 weights on the batched tensor-core score: int32
    scores bit-exact against the oracle, and the list exact."""
    from paper_1703_06256_gb300.batch import HogPlanBatch

    imgs = images(3, 13)
    w = wl.weights_i8(16, wl.rng_for(13))
    b = HogPlanBatch(SIZES, channels=3, levels=3, n_bins=16, stride=4, w_dtype=fh.HOG_I8)
    b.set_images(imgs)
    b.set_weights(w, -2.0, 25.0)
    b.run()
    check_batch(fh, b, imgs, w.astype(np.float64), -2.0, 25.0, exact=True)


@pytest.mark.parametrize("nb,stride", [(16, 4), (8, 8)])
def test_batch_f32_weights(fh, nb, stride):
    """f32 weights (three exact bf16 parts on the tensor cores, bf16 cells);
    N_b 16 and stride 8."""
    from paper_1703_06256_gb300.batch import HogPlanBatch

    imgs = images(3, 3)
    rng = wl.rng_for(10)
    w = wl.weights_f32(nb, rng)
    b = HogPlanBatch(SIZES, channels=3, levels=2, n_bins=nb, stride=stride, w_dtype=fh.HOG_F32)
    b.set_images(imgs)
    b.set_weights(w, 0.0, 0.5)
    b.run()
    check_batch(fh, b, imgs, w.astype(np.float64), 0.0, 0.5, exact=False)


def test_batch_equals_per_image_calls(fh):
    """Batch results are bit-identical to hog_cell_hist_fused +
    hog_window_score on each item alone."""
    from paper_1703_06256_gb300.batch import HogPlanBatch

    imgs = images(3, 4)
    w = wl.weights_f32(8, wl.rng_for(11))
    b = HogPlanBatch(SIZES, channels=3, levels=2, n_bins=8, stride=4)
    b.set_images(imgs)
    b.set_weights(w, 0.25, 0.5)
    b.run()
    got = b.results()
    fh.hog_tune_set(fh.HOG_TUNE_SCORE_PATH, 2)  # the batch scores on the tensor cores; so does each item here
    for m, it in zip(b.item_meta, got["items"]):
        lvl = levels_of(imgs[m["image"]], 2)[m["level"]]
        H, W = lvl.shape[:2]
        p = fh.HogPipeline(W, H, 3, 8, 4, cell_dtype=fh.HOG_BF16, w_dtype=fh.HOG_BF16)
        p.fused = True
        p.set_weights(w, 0.25, 0.5)
        p.set_image(lvl)
        p.run()
        one = p.results()
        assert np.array_equal(one["cells"], it["cells"])
        assert np.array_equal(one["scores"], it["scores"])
    fh.hog_tune_set(fh.HOG_TUNE_SCORE_PATH, 0)
