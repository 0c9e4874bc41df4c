"""Replicas over several GPUs, one process per GPU.

Slices (and detectors) are independent once each carries its halos, as the
paper sends successive slices to different trigger CPUs ("DAQ system of
NEMO Phase II"), so N GPUs run N replicas of the whole path on their own
shares: no collective touches the data.  Only the measurement is combined:
the step time is the maximum over ranks and the hits are summed.  The
reductions go through torch.distributed, with NCCL on GPU tensors or gloo on
CPU tensors.
"""
from __future__ import annotations

import torch
import torch.distributed as dist


def world() -> tuple[int, int]:
    """(rank, world size) of the initialised process group, else (0, 1)."""
    if dist.is_available() and dist.is_initialized():
        return dist.get_rank(), dist.get_world_size()
    return 0, 1


def shard(n: int, rank: int, world_size: int) -> range:
    """Contiguous share of n independent units for a rank: the first n mod
    world_size ranks take one extra unit; together the shares cover 0..n-1
    once."""
    if world_size < 1 or not 0 <= rank < world_size:
        raise ValueError("rank must lie in [0, world_size)")
    q, r = divmod(n, world_size)
    lo = rank * q + min(rank, r)
    return range(lo, lo + q + (1 if rank < r else 0))


def _reduce(x: float, op, device) -> float:
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=op)
    return float(t.item())


def max_over_ranks(x: float, device="cpu") -> float:
    rank, ws = world()
    return x if ws == 1 else _reduce(x, dist.ReduceOp.MAX, device)


def sum_over_ranks(x: float, device="cpu") -> float:
    rank, ws = world()
    return x if ws == 1 else _reduce(x, dist.ReduceOp.SUM, device)


def barrier() -> None:
    if world()[1] > 1:
        dist.barrier()
