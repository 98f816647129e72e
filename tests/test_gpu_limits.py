"""Sizes at the limits of the API: images 65535 pixels wide or tall (the
whole path against the oracle), and an image of 2^30 pixels whose integral
planes lie up to 7.5 GB into their buffer, checked by properties that hold
at any size (bin-map crops against the oracle, the total of the integral
images, cells against direct counts of the bin map, scores against the FP64
score of the GPU's own cells, the detection count, and the fused path
against the five calls)."""

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


@pytest.mark.parametrize("W,H", [(65535, 140), (72, 65535)])
def test_extreme_aspect_against_the_oracle(fh, W, H):
    rng = np.random.default_rng(W + H)
    img = rng.integers(0, 256, size=(H, W, 3), dtype=np.uint8)
    w = wl.weights_f32(8, rng)
    p = fh.HogPipeline(W, H, 3, 8, 4)
    p.set_weights(w, 0.0, 0.5)
    p.set_image(img)
    p.run()
    got = p.results()
    ref = oracle.pipeline(img, 8, w, 0.0, 4)
    assert np.array_equal(got["bins"], ref["bins"])
    assert np.array_equal(got["ii"], ref["ii"])
    assert np.array_equal(got["cells"], ref["cells"])
    S64 = ref["scores"]
    assert got["scores"].shape == S64.shape
    if S64.size:
        tol = 1e-5 * oracle.window_score(np.abs(ref["cells"]), np.abs(w.astype(np.float64)), 0.0, stride=4)
        assert np.all(np.abs(got["scores"] - S64) <= tol)
    assert got["count"] == int(np.count_nonzero(got["scores"] >= 0.5))


def test_a_billion_pixels(fh):
    W = H = 32768
    gen = torch.Generator(device="cuda").manual_seed(1703)
    # smooth-ish content: a coarse random field upsampled, plus fine noise
    coarse = torch.randint(0, 256, (H // 64, W // 64), device="cuda", generator=gen, dtype=torch.uint8)
    img = coarse.repeat_interleave(64, 0).repeat_interleave(64, 1)
    img = (img.int() + torch.randint(0, 24, (H, W), device="cuda", generator=gen, dtype=torch.int32)).clamp_(0, 255)
    img = img.to(torch.uint8).contiguous()
    w = wl.weights_f32(8, wl.rng_for(15))
    p = fh.HogPipeline(W, H, 1, 8, 4, max_out=1 << 20)
    p.set_weights(w, 0.0, 2.0)
    p.img.copy_(img.reshape(-1))
    del img
    p.run()
    torch.cuda.synchronize()
    bins = p.bins.view(H, W)
    # the image border has no bin (Eq. 1 needs both neighbours)
    for edge in (bins[0], bins[H - 1], bins[:, 0], bins[:, W - 1]):
        assert bool((edge == 255).all())
    # bin-map crops (with one pixel of context) at the corners and the middle, against the oracle
    for (y0, x0) in [(1, 1), (H - 41, W - 41), (H // 2, W // 2), (1, W - 41), (H - 41, 1)]:
        crop = p.img.view(H, W)[y0 - 1: y0 + 41, x0 - 1: x0 + 41].cpu().numpy()
        ref = oracle.bin_map(crop, 8)[1:-1, 1:-1]
        assert np.array_equal(bins[y0: y0 + 40, x0: x0 + 40].cpu().numpy(), ref), (y0, x0)
    # the integral images: their last entries sum to the number of binned pixels
    plane = W * H
    last = [int(p.ii[b * plane + plane - 1].item()) for b in range(8)]
    assert sum(last) == int((bins != 255).sum().item())
    for b in (0, 7):
        assert last[b] == int((bins == b).sum().item())
    # cells (Eq. 6 on the integral images) against direct counts of the bin map
    ncx, ncy = p.ncx, p.ncy
    cells = p.cells.view(ncy, ncx, 8)
    rng = np.random.default_rng(16)
    picks = [(0, 0), (ncy - 1, ncx - 1), (ncy - 1, 0), (0, ncx - 1)] + [tuple(v) for v in
                                                                    rng.integers(0, [ncy, ncx], size=(12, 2))]
    for (j, i) in picks:
        blk = bins[4 * j: 4 * j + 8, 4 * i: 4 * i + 8].reshape(-1).long()
        cnt = torch.bincount(blk[blk < 8], minlength=8).cpu().numpy()
        assert np.array_equal(cells[j, i].cpu().numpy().astype(np.int64), cnt), (j, i)
    # scores at sampled windows against the FP64 score of the GPU's own cells
    nx, ny = p.nx, p.ny
    S = p.scores[: nx * ny].view(ny, nx)
    for (py, px) in [(0, 0), (ny - 1, nx - 1), (ny // 3, nx // 2)]:
        c = cells[py: py + 31, px: px + 15].cpu().numpy().astype(np.int64)
        s64 = oracle.window_score(c, w, 0.0, stride=4)[0, 0]
        mass = oracle.window_score(np.abs(c), np.abs(w.astype(np.float64)), 0.0, stride=4)[0, 0]
        assert abs(float(S[py, px].item()) - s64) <= 1e-5 * mass, (py, px)
    # the detection count is the number of scores at or above the threshold
    assert int(p.count.item()) == int((S >= 2.0).sum().item())
    # the fused path gives the same cells
    fused = torch.empty_like(p.cells)
    fh.hog_cell_hist_fused(p.img, W, H, 1, W, p.lut, 8, 8, 4, fh.HOG_F32, fused)
    torch.cuda.synchronize()
    assert torch.equal(fused, p.cells)
