"""The host side of running on several GPUs, with world_size-2 gloo process
groups on the CPU (no GPU needed).

The single-cloud barcode does not shard (one filtration order, one pivot table),
so ``bench.py --gpus N`` runs N replicas: the job's time is the slowest rank's,
its work the sum over ranks.  The batched workload shards by cloud: clouds are
independent, so each rank takes a longest-processing-time-first share and no
device collective is involved.
"""
import math
import os
import socket
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)


def _free_port() -> int:
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, weights, q):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    import bench
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        slow = bench.max_over_ranks(10.0 + 7.0 * rank)  # rank 1 is the slow one
        work = bench.sum_over_ranks(100.0 + rank)
        shard = bench.lpt_shards(weights, world)[rank]
        everyone = [None] * world
        dist.all_gather_object(everyone, shard)
        q.put((rank, slow, work, everyone))
    finally:
        dist.destroy_process_group()


def _run(world, weights):
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, world, port, weights, q)) for r in range(world)]
    for p in procs:
        p.start()
    out = [q.get(timeout=120) for _ in range(world)]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    return sorted(out)


def test_two_ranks_agree_on_time_work_and_shards():
    weights = [math.comb(n, 3) for n in (64, 512, 300, 128, 400, 77, 250, 511)]
    out = _run(2, weights)
    for rank, slow, work, everyone in out:
        assert slow == 17.0          # the slowest rank's time, on every rank
        assert work == 201.0         # both ranks' work
        flat = sorted(i for shard in everyone for i in shard)
        assert flat == list(range(len(weights)))  # every cloud once
    import bench
    assert out[0][3] == bench.lpt_shards(weights, 2)  # the same split everywhere


def test_whole_job_rate_uses_the_slowest_rank():
    import bench
    assert bench.whole_job_rate(2 * 1000.0, 500.0) == pytest.approx(4000.0)


@pytest.mark.parametrize("world", [1, 2, 3, 8])
def test_lpt_shards_cover_and_balance(world):
    import bench
    weights = [math.comb(64 + (37 * i) % 449, 3) for i in range(256)]
    shards = bench.lpt_shards(weights, world)
    assert sorted(i for s in shards for i in s) == list(range(256))
    loads = [sum(weights[i] for i in s) for s in shards]
    # LPT: no rank exceeds the average by more than the heaviest item
    assert max(loads) <= sum(weights) / world + max(weights)


def test_single_process_helpers_are_identities():
    import bench
    assert bench.max_over_ranks(3.5) == 3.5
    assert bench.sum_over_ranks(2.0) == 2.0
