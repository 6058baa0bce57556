"""Multi-GPU host logic: one process per GPU, queries sharded across ranks.

Matching problems are independent (each query is its own Algorithm 1 run),
so the data path needs no collective: rank r runs its own contiguous share
of the queries on its GPU. Collectives appear only around it: a barrier and
a max-over-ranks reduction of the timed region, and (for users who want all
results on one rank) a gather of the result records.
"""
from __future__ import annotations

import os
from typing import List, Sequence, Tuple


def rank_env() -> Tuple[int, int, int]:
    """(rank, world_size, local_rank) from the torchrun environment."""
    return (int(os.environ.get("RANK", "0")), int(os.environ.get("WORLD_SIZE", "1")),
            int(os.environ.get("LOCAL_RANK", "0")))


def shard_range(n: int, world: int, rank: int) -> Tuple[int, int]:
    """Contiguous share [start, end) of n items for `rank` of `world`; shares
    differ in size by at most one and cover 0..n-1 exactly once."""
    if world < 1 or not 0 <= rank < world:
        raise ValueError("bad rank/world")
    base, extra = divmod(n, world)
    start = rank * base + min(rank, extra)
    return start, start + base + (1 if rank < extra else 0)


def max_over_ranks(value: float) -> float:
    """Largest value over all ranks (the job time is the slowest rank's)."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(value)
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([float(value)], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def gather_results(local: Sequence, n: int) -> List:
    """All ranks' shares of a length-n result list, in query order, on every
    rank (shares as shard_range assigns them)."""
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return list(local)
    world = dist.get_world_size()
    parts: List = [None] * world
    dist.all_gather_object(parts, list(local))
    out: List = []
    for r in range(world):
        s, e = shard_range(n, world, r)
        assert len(parts[r]) == e - s, "shard sizes disagree"
        out.extend(parts[r])
    return out
