"""The precision workload: 32 RGB 1920x1080 images, N_b = 8, 8x8 cells,
64x128 window, stride 4 (the paper's inner product, Section 4, on the tensor
cores).

- bf16 cells x bf16 weights with FP32 accumulation (tcgen05), against the
  FP64 oracle on the ORIGINAL f32 weights: the error splits into the weight
  rounding (bf16 keeps 8 significant bits, unit roundoff 2^-8 of each
  weight) and the FP32 accumulation (within 1e-5 of the scale).  Both are
  measured and bounded per window relative to sum_k |w_k| h_k + |bias|; the
  largest values are printed (run with -s to see them).
- int8 weights (uniform integers in [-127, 127]): int32 scores and the list
  bit-exact against the oracle.
- cells bit-exact against the oracle on every image.
"""

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
def cfg3():
    return wl.config3()


@pytest.fixture(scope="module")
def oracle_cells(cfg3):
    return [oracle.cell_hist_ii(oracle.integral(oracle.bin_map(img, 8), 8), 8, 8, 4) for img in cfg3["images"]]


def run_images(fh, cfg3, w, w_dtype, bias, thr):
    """The five calls on each image (bf16 cells), as the library runs them."""
    H, W = cfg3["images"][0].shape[:2]
    p = fh.HogPipeline(W, H, 3, 8, 4, cell_dtype=fh.HOG_BF16, w_dtype=w_dtype)
    p.set_weights(w, bias, thr)
    out = []
    for img in cfg3["images"]:
        p.set_image(img)
        p.run()
        out.append(p.results())
    return out


def test_precision_bf16_error_1080p(fh, cfg3, oracle_cells):
    w = cfg3["w"].astype(np.float64)
    w_bf = torch.from_numpy(cfg3["w"]).to(torch.bfloat16).double().numpy()  # the weights the tensor cores see
    bias = 0.0
    got = run_images(fh, cfg3, cfg3["w"], fh.HOG_BF16, bias, 0.5)
    worst_abs = worst_rel = worst_acc = worst_round = 0.0
    for res, cells in zip(got, oracle_cells):
        assert np.array_equal(res["cells"], cells)
        S = res["scores"].astype(np.float64)
        S64 = oracle.window_score(cells, w, bias, stride=4)
        S64_bf = oracle.window_score(cells, w_bf, bias, stride=4)
        scale = oracle.window_score(np.abs(cells), np.abs(w), abs(bias), stride=4)
        scale_bf = oracle.window_score(np.abs(cells), np.abs(w_bf), abs(bias), stride=4)
        err = np.abs(S - S64)
        worst_abs = max(worst_abs, float(err.max()))
        empty = scale == 0  # no binned pixel in the window: the score is the bias, exactly
        assert np.all(S[empty] == np.float32(bias))
        live = ~empty
        worst_rel = max(worst_rel, float((err[live] / scale[live]).max()))
        worst_acc = max(worst_acc, float((np.abs(S - S64_bf)[live] / scale_bf[live]).max()))
        worst_round = max(worst_round, float((np.abs(S64_bf - S64)[live] / scale[live]).max()))
    print(f"\n1080p x32 bf16 tensor-core score vs FP64 on the f32 weights: max |err| = {worst_abs:.3e}, "
          f"max |err| / (sum|w|h + |b|) = {worst_rel:.3e} (weight rounding alone {worst_round:.3e}); "
          f"FP32 accumulation vs FP64 on the bf16 weights: {worst_acc:.3e} of the scale")
    assert worst_acc <= 1e-5
    assert worst_round <= 2.0 ** -8
    assert worst_rel <= 2.0 ** -8 + 1e-5


def test_precision_int8_exact_1080p(fh, cfg3, oracle_cells):
    w8 = cfg3["w_i8"]
    bias, thr = 7.0, 2000.0
    got = run_images(fh, cfg3, w8, fh.HOG_I8, bias, thr)
    total = 0
    for res, cells in zip(got, oracle_cells):
        assert np.array_equal(res["cells"], cells)
        S64 = oracle.window_score(cells, w8.astype(np.float64), bias, stride=4)
        assert res["scores"].dtype == np.int32
        assert np.array_equal(res["scores"].astype(np.int64), S64.astype(np.int64))
        xs, ys, sc = oracle.detect(S64, 4, thr)
        det = res["detections"]
        assert res["count"] == len(xs)
        assert np.array_equal(det["x"], xs) and np.array_equal(det["y"], ys)
        assert np.array_equal(det["score"], sc.astype(np.float32))
        total += len(xs)
    assert total > 0
