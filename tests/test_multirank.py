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
