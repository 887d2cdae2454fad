"""Walker sharding across GPUs (one process per GPU).

Walkers are independent, so the forward MO vgl needs no collective: each rank
evaluates a contiguous range of walkers.  The adjoint of a loss summed over
all walkers has one exchange step: dL/dC and dL/dR_nuc are sums over walkers,
so the per-rank gradients are all-reduced (summed).
"""
from __future__ import annotations

from typing import Tuple


def shard_range(walk_num: int, rank: int, world: int) -> Tuple[int, int]:
    """[begin, end) of the walkers owned by `rank` (contiguous, sizes differ
    by at most one)."""
    if world < 1 or not 0 <= rank < world:
        raise ValueError(f"bad rank {rank} for world size {world}")
    base, extra = divmod(walk_num, world)
    begin = rank * base + min(rank, extra)
    return begin, begin + base + (1 if rank < extra else 0)


def allreduce_gradients(dC, dR, group=None):
    """Sum the per-shard dL/dC and dL/dR_nuc over all ranks, in place."""
    import torch.distributed as dist
    if not dist.is_available() or not dist.is_initialized():
        return dC, dR
    for t in (dC, dR):
        if t is not None:
            dist.all_reduce(t, op=dist.ReduceOp.SUM, group=group)
    return dC, dR
