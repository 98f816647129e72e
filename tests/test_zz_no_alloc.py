"""hog_detect_noalloc: the detect entry point for callers that cannot allocate
device scratch (it uses a fixed array inside the library instead of a
caller-provided workspace).  Its lists must equal hog_detect's on the same
scores, call after call, since every call reuses the same array.

This file is collected last on purpose, so that a run stopping at its first
failure has already run every other test."""

import ctypes

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def fh():
    import paper_1703_06256_gb300 as m

    assert torch.cuda.is_available()
    return m


def run_both(fh, S, stride, thr, max_out):
    """One call of each entry point through the C ABI on the same scores."""
    L = fh.lib()
    ny, nx = S.shape
    dtype = fh.HOG_I32 if S.dtype == np.int32 else fh.HOG_F32
    s = torch.from_numpy(np.ascontiguousarray(S).reshape(-1)).cuda()
    outs, counts = [], []
    for use_noalloc in (False, True):
        out = torch.full((max(max_out, 1) * fh.DET_BYTES,), 0x5A, dtype=torch.uint8, device="cuda")
        cnt = torch.full((1,), -1, dtype=torch.int32, device="cuda")
        stream = torch.cuda.current_stream().cuda_stream
        if use_noalloc:
            rc = L.hog_detect_noalloc(s.data_ptr(), dtype, nx, ny, stride, ctypes.c_float(thr), 5, 1,
                                      out.data_ptr(), max_out, cnt.data_ptr(), stream)
        else:
            ws_b = L.hog_detect_workspace_bytes(nx, ny)
            ws = torch.zeros(max(ws_b, 256), dtype=torch.uint8, device="cuda")
            rc = L.hog_detect(s.data_ptr(), dtype, nx, ny, stride, ctypes.c_float(thr), 5, 1, out.data_ptr(),
                              max_out, cnt.data_ptr(), ws.data_ptr(), ws_b, stream)
        assert rc == fh.HOG_OK
        torch.cuda.synchronize()
        n = int(cnt.item())
        counts.append(n)
        outs.append(fh.dets_to_numpy(out.cpu(), min(n, max_out)))
    return outs, counts


def test_noalloc_matches_workspace_entry_point_twice(fh):
    rng = np.random.default_rng(2024)
    # two different score maps in a row (the second call reuses the scratch
    # the first one left behind); both span many 2048-score tiles
    for call, (ny, nx) in enumerate([(211, 333), (119, 185)]):
        S = rng.normal(0.0, 1.0, size=(ny, nx)).astype(np.float32)
        (ref, got), (n_ref, n_got) = run_both(fh, S, 4, 0.5, ny * nx)
        assert n_ref == n_got and n_got > 2048, call
        assert np.array_equal(ref, got), call
    # integer scores with a capped list
    S = rng.integers(-50, 50, size=(300, 401)).astype(np.int32)
    for _ in range(2):
        (ref, got), (n_ref, n_got) = run_both(fh, S, 8, 10.0, 500)
        assert n_ref == n_got and len(got) == 500 and np.array_equal(ref, got)


def test_noalloc_many_tiles_and_at_its_limit(fh):
    import oracle

    rng = np.random.default_rng(2025)
    # 2100 x 2100 scores: 2154 tiles, against hog_detect and the oracle's list
    S = rng.normal(0.0, 1.0, size=(2100, 2100)).astype(np.float32)
    (ref, got), (n_ref, n_got) = run_both(fh, S, 4, 2.5, 2100 * 2100)
    xs, ys, sc = oracle.detect(S.astype(np.float64), 4, 2.5)
    assert n_ref == n_got == len(xs)
    assert np.array_equal(ref, got)
    assert np.array_equal(got["x"], xs) and np.array_equal(got["y"], ys)
    assert np.array_equal(got["score"], sc.astype(np.float32))
    # exactly HOG_DETECT_NOALLOC_MAX_SCORES scores (every status word of the
    # scratch in use), twice in a row, with a list capped mid-way
    ny, nx = 8192, fh.HOG_DETECT_NOALLOC_MAX_SCORES // 8192
    S = torch.randn(ny * nx, generator=torch.Generator().manual_seed(7)).numpy().reshape(ny, nx)
    for _ in range(2):
        (ref, got), (n_ref, n_got) = run_both(fh, S, 4, 3.5, 5000)
        ys, xs = np.nonzero(S >= np.float32(3.5))
        assert n_ref == n_got == len(xs) and len(got) == 5000
        assert np.array_equal(ref, got)
        assert np.array_equal(got["x"], xs[:5000] * 4) and np.array_equal(got["y"], ys[:5000] * 4)


def test_noalloc_rejects_sizes_beyond_its_scratch(fh):
    L = fh.lib()
    big = fh.HOG_DETECT_NOALLOC_MAX_SCORES // 4096 + 1  # ny * 4096 > the limit
    cnt = torch.zeros(1, dtype=torch.int32, device="cuda")
    s = torch.zeros(1, dtype=torch.float32, device="cuda")
    rc = L.hog_detect_noalloc(s.data_ptr(), fh.HOG_F32, 4096, big, 4, ctypes.c_float(0.5), 0, 0, None, 0,
                              cnt.data_ptr(), torch.cuda.current_stream().cuda_stream)
    assert rc == fh.HOG_ERR_ARG  # refused on the host: nothing was launched
