"""Weak-scaling shards over processes (one per GPU).

MICKEY instances are independent, so the data path has no exchange: rank r
of `world` takes instances r*n .. (r+1)*n - 1 of the workload's draw
sequence and generates them on its own GPU.  The only collectives are the
barrier around the timed region and the maximum of the ranks' times, which
work on whichever backend the process group uses (NCCL on GPUs, gloo on
CPU).
"""
from __future__ import annotations

import torch
import torch.distributed as dist

from . import workloads


def bounds(rank: int, world: int, n_per_rank: int) -> tuple[int, int]:
    """Instance range [start, stop) of `rank`."""
    if not 0 <= rank < world:
        raise ValueError("rank %d outside a world of %d" % (rank, world))
    return rank * n_per_rank, (rank + 1) * n_per_rank


def plain_shard(rank: int, world: int, n_per_rank: int, n_bits: int,
                name: str = workloads.PLAIN_SCALE["name"],
                seed: int = workloads.PLAIN_SCALE["seed"]) -> workloads.StreamSet:
    """This rank's instances of the plain workload (drawn directly, without
    generating the other ranks' draws)."""
    start, _ = bounds(rank, world, n_per_rank)
    return workloads.fixed_streams(name, seed, n_per_rank, n_bits, first=start)


def _device() -> torch.device:
    if dist.get_backend() == "nccl":
        return torch.device("cuda", torch.cuda.current_device())
    return torch.device("cpu")


def max_over_ranks(x: float) -> float:
    """Largest x over the ranks (x itself without a process group)."""
    if not dist.is_initialized() or dist.get_world_size() == 1:
        return float(x)
    t = torch.tensor([float(x)], dtype=torch.float64, device=_device())
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def barrier() -> None:
    if dist.is_initialized() and dist.get_world_size() > 1:
        dist.barrier()
