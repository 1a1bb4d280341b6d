"""The multi-process path on CPUs: two gloo ranks join the group from the
launcher's environment, agree on the slowest rank's time, partition the
beams with no overlap, draw distinct input seeds, and compute the whole-job
weak-scaling throughput; only rank 0 runs the CPU reference arm."""
import os
import socket

import pytest
import torch.multiprocessing as mp

from paper_2605_03531_b300 import shard


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port),
                      WORLD_SIZE=str(world), RANK=str(rank), LOCAL_RANK=str(rank))
    import torch.distributed as dist
    w, r, _ = shard.init("gloo")
    assert (w, r) == (world, rank)
    shard.barrier(w)
    slowest = shard.max_over_ranks(1.5 + rank, w)
    total = shard.sum_over_ranks(10 + rank, w)
    mine = shard.shard(range(11), w, r)
    every = [None] * w
    dist.all_gather_object(every, mine)
    seeds = [None] * w
    dist.all_gather_object(seeds, shard.rank_seed(5, r))
    out.put((rank, slowest, total, every, seeds,
             shard.weak_value(100.0, slowest, w), shard.runs_reference(w, r)))
    shard.finish(w)


def test_two_gloo_ranks():
    world, port = 2, _free_port()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_worker, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in range(world))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, slowest, total, every, seeds, value, ref in res:
        assert slowest == pytest.approx(2.5)           # max over ranks
        assert total == pytest.approx(21.0)
        flat = sorted(b for part in every for b in part)
        assert flat == list(range(11))                 # disjoint and complete
        assert len(set(seeds)) == world
        assert value == pytest.approx(2 * 100.0 / 2.5)
        assert ref == (rank == 0)


def test_single_rank_needs_no_group():
    for k in ("WORLD_SIZE", "RANK", "LOCAL_RANK"):
        os.environ.pop(k, None)
    w, r, _ = shard.init("gloo")
    assert (w, r) == (1, 0)
    assert shard.max_over_ranks(3.0, w) == 3.0
    assert shard.shard([4, 5, 6], 1, 0) == [4, 5, 6]
    assert shard.runs_reference(1, 0)
