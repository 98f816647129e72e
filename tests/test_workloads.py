"""The seeded input recipe (workloads/): the same seed gives the same inputs,
and the shapes, types, value ranges and stream statistics are the ones the
recipe states (images of the stated sizes and channels, weights of 16 x 8
cells x N_b, integer weights in [-127, 127], request sizes on the multiple-of-8
grid within 320x240 .. 3840x2160, Poisson arrivals at the given rate)."""

import numpy as np

import workloads as wl


def test_seeded_and_repeatable():
    a, b = wl.config1(), wl.config1()
    assert np.array_equal(a["images"][0], b["images"][0]) and np.array_equal(a["w"], b["w"])
    c = wl.config1(seed=5)
    assert not np.array_equal(a["images"][0], c["images"][0])
    assert wl.rng_for(1).integers(0, 1 << 30) == np.random.Generator(np.random.PCG64(wl.BASE_SEED + 1)).integers(
        0, 1 << 30)


def test_config_shapes_and_types():
    c0 = wl.config0()
    img0 = c0["images"][0]
    assert img0.shape == (240, 320) and img0.dtype == np.uint8
    assert (c0["n_bins"], c0["stride"]) == (8, 8)
    c1 = wl.config1()
    img1 = c1["images"][0]
    assert img1.shape == (600, 800, 3) and img1.dtype == np.uint8
    assert (c1["n_bins"], c1["stride"], c1["thr"]) == (8, 4, 0.5)
    assert c1["w"].shape == (16 * 8 * 8,) and c1["w"].dtype == np.float32
    assert 0.005 < float(c1["w"].std()) < 0.015  # N(0, 0.01)
    c3 = wl.config3(n_images=2, W=96, H=64)
    assert len(c3["images"]) == 2 and all(im.shape == (64, 96, 3) for im in c3["images"])
    wi = c3["w_i8"]
    assert wi.dtype == np.int8 and wi.shape == (1024,) and wi.min() >= -127 and wi.max() <= 127


def test_images_cover_the_value_range_and_have_smooth_regions():
    img = wl.config1()["images"][0].astype(np.int32)
    assert img.min() <= 16 and img.max() >= 239
    dx = np.abs(img[:, 2:] - img[:, :-2]).max(axis=2)
    # mostly small gradients (smooth noise and flat shapes), some large ones (shape edges)
    assert np.mean(dx <= 8) > 0.8 and dx.max() >= 128


def test_request_stream():
    reqs = wl.request_stream(4000, rate_per_s=1000.0)
    ws = np.array([r["W"] for r in reqs])
    hs = np.array([r["H"] for r in reqs])
    assert np.all(ws % 8 == 0) and np.all(hs % 8 == 0)
    assert ws.min() >= 320 and ws.max() <= 3840 and hs.min() >= 240 and hs.max() <= 2160
    t = np.array([r["t"] for r in reqs])
    gaps = np.diff(t)
    assert np.all(gaps >= 0) and abs(gaps.mean() - 1e-3) < 1e-4  # Poisson arrivals at 1000/s
    assert reqs == wl.request_stream(4000, rate_per_s=1000.0)  # seeded
    img = wl.request_image(dict(W=64, H=48, seed=reqs[0]["seed"]))
    assert img.shape == (48, 64, 3) and img.dtype == np.uint8


def test_batch_sizes():
    c2 = wl.config2(n_images=6)
    assert len(c2["images"]) == 6
    for im in c2["images"]:
        assert (im.shape[1], im.shape[0]) in wl.BATCH_SIZES and im.shape[2] == 3
