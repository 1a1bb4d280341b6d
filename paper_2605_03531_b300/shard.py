"""One process per GPU, beams partitioned across ranks with no exchange on
the data path: beams are independent, so a rank only needs its own share of
them, and the processes meet only for a barrier and the maximum of their
timings.  The same calls run over NCCL on GPUs and over gloo on CPUs."""
from __future__ import annotations

import os


def world_from_env():
    """(world size, rank, local rank) from the launcher's environment."""
    return (int(os.environ.get("WORLD_SIZE", "1")), int(os.environ.get("RANK", "0")),
            int(os.environ.get("LOCAL_RANK", "0")))


def init(backend=None):
    """Join the process group when launched with more than one rank
    (nccl when CUDA is available, else gloo); returns (world, rank, local)."""
    import torch
    world, rank, local = world_from_env()
    if world > 1:
        import torch.distributed as dist
        if backend is None:
            backend = "nccl" if torch.cuda.is_available() else "gloo"
        if backend == "nccl":
            torch.cuda.set_device(local)
            dist.init_process_group("nccl", device_id=torch.device("cuda", local))
        else:
            dist.init_process_group(backend)
    elif torch.cuda.is_available():
        torch.cuda.set_device(0)
    return world, rank, local


def _device():
    import torch
    import torch.distributed as dist
    if dist.get_backend() == "nccl":
        return torch.device("cuda", torch.cuda.current_device())
    return torch.device("cpu")


def barrier(world):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


def max_over_ranks(v, world):
    """The largest of every rank's value (e.g. a timed region's length)."""
    if world == 1:
        return v
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(v)], dtype=torch.float64, device=_device())
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def sum_over_ranks(v, world):
    if world == 1:
        return v
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(v)], dtype=torch.float64, device=_device())
    dist.all_reduce(t, op=dist.ReduceOp.SUM)
    return float(t.item())


def shard(items, world, rank):
    """This rank's share of a list of independent beams (round robin, so
    every rank gets a similar mix)."""
    return list(items)[rank::world]


def rank_seed(base, rank):
    """Distinct input seeds per rank for the synthetic beams."""
    return int(base) + 1000 * int(rank)


def weak_value(units_per_rank, seconds_max, world):
    """Whole-job throughput when every rank processes the same amount of
    work: all ranks' units over the slowest rank's time."""
    return world * float(units_per_rank) / float(seconds_max)


def runs_reference(world, rank):
    """The CPU reference arm runs once per job: on rank 0."""
    return world == 1 or rank == 0


def finish(world):
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()
