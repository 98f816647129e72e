"""Host-side pieces of bench.py that the reported figures rest on: the
algorithmic bytes each stage's roofline divides by (per-unit figures times the
units of one launch), and the committed ncu DRAM traffic, which the bench
reports only while the profiled kernel's source is unchanged."""

import hashlib
import os

import pytest

import bench


def n_pos(extent, box, stride):
    return (extent - box) // stride + 1


@pytest.mark.parametrize("W,H", [(800, 600), (3840, 2160), (641, 333)])
def test_algorithmic_bytes_per_unit(W, H):
    nb, cell, stride, r = 8, 8, 4, 2
    ncx, ncy = n_pos(W, cell, stride), n_pos(H, cell, stride)
    windows = (ncx - 7 * r) * (ncy - 15 * r)
    b = bench.algorithmic_bytes(W, H, nb, ncx, ncy, windows)
    px = W * H
    assert b["bin_map"] == px * 4                       # 3 RGB bytes in, one bin out per pixel
    assert b["integral"] == px * (1 + 4 * nb)           # one bin in, N_b int32 entries out
    assert b["cell_hist"] == ncx * ncy * nb * (4 + 2)   # one sample in, one bf16 count out per cell and bin
    assert b["score"] == ncx * ncy * nb * 2 + windows * 4
    assert b["detect"] == windows * 4
    b16 = bench.algorithmic_bytes(W, H, nb, ncx, ncy, windows, ii_bytes=2)
    assert b16["integral"] == px * (1 + 2 * nb) and b16["cell_hist"] == ncx * ncy * nb * (2 + 2)


def test_algorithmic_bytes_quoted_figures():
    # the figures the bench line and the profiles quote
    b = bench.algorithmic_bytes(800, 600, 8, 199, 149, 185 * 119)
    assert b["integral"] == 15_840_000
    b4 = bench.algorithmic_bytes(3840, 2160, 8, 959, 539, 945 * 509)
    assert (b4["bin_map"], b4["integral"], b4["cell_hist"], b4["score"], b4["detect"]) == (
        33_177_600, 273_715_200, 24_811_248, 10_194_436, 1_924_020)


def test_profiled_traffic_follows_the_source(tmp_path, monkeypatch):
    src = tmp_path / "kern.cu"
    src.write_text("// a kernel\n")
    sha = hashlib.sha256(src.read_bytes()).hexdigest()[:16]
    (tmp_path / "profiles").mkdir()
    (tmp_path / "profiles" / "traffic.txt").write_text(
        "# stage workload bytes source_file sha256_16\n"
        f"integral 800x600 519424 kern.cu {sha}\n")
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    assert bench.profiled_traffic("integral", "800x600") == 519424
    assert bench.profiled_traffic("integral", "3840x2160") is None  # no capture for that workload
    assert bench.profiled_traffic("score", "800x600") is None
    src.write_text("// a kernel, changed\n")
    assert bench.profiled_traffic("integral", "800x600") is None  # the capture no longer describes it
    os.remove(src)
    assert bench.profiled_traffic("integral", "800x600") is None


def test_committed_traffic_matches_the_sources():
    # every line of the committed file names an existing source; the stages of
    # the benchmark workload are all recorded
    path = os.path.join(bench.ROOT, "profiles", "traffic.txt")
    stages = set()
    for ln in open(path).read().splitlines():
        if ln.startswith("#") or not ln.strip():
            continue
        stage, workload, nbytes, src, sha = ln.split()
        assert os.path.exists(os.path.join(bench.ROOT, src)), src
        assert int(nbytes) > 0 and len(sha) == 16
        stages.add((stage, workload))
    for st in ("bin_map", "integral", "cell_hist", "score", "detect"):
        assert (st, "800x600") in stages and (st, "3840x2160") in stages
