"""The bounded device-side waits run out cleanly: a wait on something that
nothing provides (an mbarrier no thread arrives at; a device flag no CTA
raises) gives up after its limit, the kernel sets HOG_STATUS_TIMEOUT and
returns, the status clears, and the context stays usable for the detection
path afterwards.  No fault, trap or hang is involved: the waits are bounded
(1 ms here), and nothing else is in flight in the waiting kernel."""

import time

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
    return m


@pytest.mark.parametrize("mode", [0, 1])
def test_wait_runs_out_and_sets_the_status(fh, mode):
    assert fh.hog_device_status(clear=True) in (0, fh.HOG_STATUS_TIMEOUT)
    assert fh.hog_device_status() == 0
    t0 = time.perf_counter()
    fh.hog_selftest_wait_timeout(mode, 1000)  # 1 ms
    torch.cuda.synchronize()
    el = time.perf_counter() - t0
    assert fh.hog_device_status() == fh.HOG_STATUS_TIMEOUT
    assert el >= 1e-3  # the kernel waited its limit before giving up
    assert fh.hog_device_status(clear=True) == fh.HOG_STATUS_TIMEOUT
    assert fh.hog_device_status() == 0


def test_context_usable_after_a_timeout(fh):
    fh.hog_selftest_wait_timeout(0, 1000)
    fh.hog_selftest_wait_timeout(1, 1000)
    torch.cuda.synchronize()
    assert fh.hog_device_status(clear=True) == fh.HOG_STATUS_TIMEOUT
    c = wl.config0()
    img = c["images"][0]
    H, W = img.shape
    pipe = fh.HogPipeline(W, H, 1, c["n_bins"], c["stride"])
    pipe.set_weights(c["w"], c["bias"], 0.0)
    pipe.set_image(img)
    pipe.run()
    got = pipe.results()
    ref = oracle.pipeline(img, c["n_bins"], c["w"], c["bias"], c["stride"], 0.0)
    assert np.array_equal(got["ii"], ref["ii"]) and np.array_equal(got["cells"], ref["cells"])
    assert fh.hog_device_status() == 0


def test_selftest_argument_errors(fh):
    with pytest.raises(fh.HogError):
        fh.hog_selftest_wait_timeout(2, 1000)
    with pytest.raises(fh.HogError):
        fh.hog_selftest_wait_timeout(0, 0)
    with pytest.raises(fh.HogError):
        fh.hog_selftest_wait_timeout(0, 1000001)
