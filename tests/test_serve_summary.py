"""The serving figures (serve.latency_summary) from hand-made results: the
percentiles, the rates, which requests a long dispatcher pause touched, p99
without them, and the wait / GPU split of the slowest requests."""

import os

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def serve():
    import importlib.util

    spec = importlib.util.spec_from_file_location("_fasthog_build", os.path.join(ROOT, "paper_1703_06256_gb300",
                                                                                  "build.py"))
    b = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(b)
    b.build()
    from paper_1703_06256_gb300 import serve as m

    return m


def results(serve, n=100):
    out = []
    for k in range(n):
        lat_ms = k + 1  # 1 .. n ms
        t0 = 1_000_000_000 + k * 2_000_000  # queued every 2 ms
        out.append(serve.Result(rid=k, detections=None, count=0, latency=lat_ms * 1e-3, shape=(100, 200, 3),
                                t_enqueue_ns=t0, t_admit_ns=t0 + 250_000, t_done_ns=t0 + lat_ms * 1_000_000))
    return out


def test_percentiles_and_rates(serve):
    res = results(serve)
    s = serve.latency_summary(res, wall=0.5)
    lat = np.arange(1, 101, dtype=float)
    assert s["requests"] == 100
    assert s["p50_ms"] == round(float(np.percentile(lat, 50)), 3) == 50.5
    assert s["p99_ms"] == round(float(np.percentile(lat, 99)), 3)
    assert s["images_per_s"] == 200.0 and s["mpixel_per_s"] == round(100 * 200 * 100 / 0.5 / 1e6, 1)
    assert "long_pauses" not in s and "slowest" not in s


def test_pauses_and_slowest(serve):
    res = results(serve)
    t_first = res[0].t_enqueue_ns
    # one long pause of 10 ms starting 50 ms in, one short one of 2 ms
    long_ = (t_first + 50_000_000, t_first + 60_000_000)
    short = (t_first + 150_000_000, t_first + 152_000_000)
    s = serve.latency_summary(res, wall=0.5, pauses_ns=[long_, short], long_pause_ms=5.0)
    assert s["long_pauses"] == 1 and s["longest_pause_ms"] == 10.0
    hit = [r for r in res if long_[0] < r.t_done_ns and long_[1] > r.t_enqueue_ns]
    assert s["requests_in_long_pauses"] == len(hit) > 0
    clear = np.array([r.latency * 1e3 for r in res if r not in hit])
    assert s["p99_ms_outside_long_pauses"] == round(float(np.percentile(clear, 99)), 3)
    slow = s["slowest"]
    assert [e["gpu_ms"] + e["wait_ms"] for e in slow] == pytest.approx([100.0, 99.0, 98.0, 97.0, 96.0])
    assert all(e["wait_ms"] == 0.25 and (e["W"], e["H"]) == (200, 100) for e in slow)
    assert slow[0]["at_ms"] == 198.0  # the last request, queued 99 x 2 ms after the first
