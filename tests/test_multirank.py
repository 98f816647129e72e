"""The N > 1 path on the host: two gloo ranks shard a batch of images, time
their (simulated) replicas and agree on the whole-job throughput with the
max over ranks, exactly as bench.py does with NCCL on GPUs."""

import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402


def free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, n_images, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        from paper_1703_06256_gb300 import replicas

        mine = replicas.shard(list(range(n_images)), rank, world)
        # every rank learns every share (host-side check only; the data path has no collective)
        gathered = [None] * world
        dist.all_gather_object(gathered, mine)
        seconds = 0.5 + rank  # rank 1 is the slow replica
        t_max = replicas.max_over_ranks(seconds)
        rate = replicas.aggregate_rate(len(mine), t_max, world)
        out[rank] = (gathered, t_max, rate)
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_shard_and_agree_on_time():
    world, n_images = 2, 11
    port = free_port()
    ctx = mp.get_context("spawn")
    with ctx.Manager() as mgr:
        out = mgr.dict()
        procs = [ctx.Process(target=_rank_main, args=(r, world, port, n_images, out)) for r in range(world)]
        for p in procs:
            p.start()
        for p in procs:
            p.join(timeout=120)
            assert p.exitcode == 0
        res = dict(out)
    for rank in range(world):
        gathered, t_max, rate = res[rank]
        flat = sorted(i for share in gathered for i in share)
        assert flat == list(range(n_images))  # every image exactly once
        assert t_max == 1.5  # the slowest replica's time on every rank
        assert rate == pytest.approx(len(gathered[rank]) * world / 1.5)


def test_shard_edges():
    from paper_1703_06256_gb300 import replicas

    assert replicas.shard([1, 2, 3], 0, 1) == [1, 2, 3]
    assert replicas.shard([1, 2, 3], 2, 4) == [3]
    assert replicas.shard([1, 2, 3], 3, 4) == []
    with pytest.raises(ValueError):
        replicas.shard([1], 2, 2)
    assert replicas.max_over_ranks(3.5) == 3.5  # no process group: the value itself


def _bench_rank_main(rank, world, port, out):
    import sys
    import time

    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    sys.path.insert(0, root)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        import bench
        from paper_1703_06256_gb300 import replicas

        last = {}

        def run_step(k):
            t0 = time.perf_counter()
            time.sleep(0.01 * (rank + 1))  # rank 1 is the slow replica
            last["ms"] = (time.perf_counter() - t0) * 1e3

        mine = bench.timed_region(run_step, lambda: last["ms"], 3, dist.barrier, lambda: None)
        slowest = replicas.max_over_ranks(mine)
        out[rank] = (mine, slowest, replicas.aggregate_rate(1, slowest * 1e-3, world))
    finally:
        dist.destroy_process_group()


def test_bench_timed_region_two_gloo_ranks():
    """bench.py's own timed region (barrier and synchronise on both sides,
    per-rank mean) under two gloo ranks, then the max over ranks and the
    whole-job rate, as its N > 1 path runs them with NCCL."""
    world = 2
    port = free_port()
    ctx = mp.get_context("spawn")
    with ctx.Manager() as mgr:
        out = mgr.dict()
        procs = [ctx.Process(target=_bench_rank_main, args=(r, world, port, out)) for r in range(world)]
        for p in procs:
            p.start()
        for p in procs:
            p.join(timeout=120)
            assert p.exitcode == 0
        res = dict(out)
    assert res[0][0] < res[1][0]
    for rank in range(world):
        mine, slowest, rate = res[rank]
        assert slowest == res[1][0]  # every rank agrees on the slowest replica's time
        assert rate == pytest.approx(world / (slowest * 1e-3))


def test_bench_gpus_flag_launches_one_rank_per_gpu():
    """`bench.py --gpus 2` outside torchrun starts two ranks (here the
    reference arm, which needs no GPU: rank 0 times the oracle and prints,
    rank 1 exits without work)."""
    import json
    import subprocess
    import sys

    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    env = {k: v for k, v in os.environ.items() if k not in ("RANK", "WORLD_SIZE", "LOCAL_RANK")}
    r = subprocess.run([sys.executable, os.path.join(root, "bench.py"), "--impl", "reference", "--gpus", "2",
                        "--steps", "1", "--warmup", "0"], capture_output=True, text=True, timeout=600, env=env)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [ln for ln in r.stdout.splitlines() if ln.startswith("{")]
    assert len(lines) == 1  # rank 0 alone prints
    line = json.loads(lines[0])
    assert line["impl"] == "reference" and line["n_gpus"] == 2 and line["value"] > 0
