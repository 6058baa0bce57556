"""Multi-GPU host logic: one process per GPU, queries sharded across ranks.

Matching problems are independent (each query is its own Algorithm 1 run),
so the data path needs no collective: rank r runs its own contiguous share
of the queries on its GPU. Collectives appear only around it: a barrier and
a max-over-ranks reduction of the timed region, and (for users who want all
results on one rank) a gather of the result records.
"""
from __future__ import annotations

import os
from typing import List, Optional, Sequence, Tuple


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


# ---------------------------------------------------------------- one signal in slices
def slice_bounds(N: int, world: int, rank: int, align: int = 16) -> Tuple[int, int]:
    """Contiguous slice [n0, n1) of N entries for `rank`; every start is a
    multiple of `align` entries (the fold's 16-byte boundary), the last slice
    takes the remainder."""
    if world < 1 or not 0 <= rank < world:
        raise ValueError("bad rank/world")
    step = -(-N // world)
    step = -(-step // align) * align
    n0 = min(N, rank * step)
    return n0, min(N, n0 + step)


class LibSliceOps:
    """The library's slice entry points for match_sliced, on this rank's GPU."""

    def __init__(self, plan, t_dev):
        self.plan, self.t = plan, t_dev
        self.P = plan.info["P"]

    def fold_slice(self, x_slice, n0: int, length: int):
        import torch
        dt = torch.float32 if x_slice.dtype in (torch.float32, torch.float16) else torch.int32
        y = torch.empty(2 * self.P, dtype=dt, device=self.t.device)
        self.plan.fold_slice(x_slice, n0, length, y)
        return y

    def correlate_folds(self, y) -> dict:
        import torch
        from . import decode_results, result_buffer
        out = result_buffer(1, device=self.t.device)
        self.plan.correlate_folds(y, self.t, out)
        torch.cuda.synchronize(self.t.device)
        return decode_results(out)[0]

    def candidates(self, res: dict) -> List[int]:
        from . import tm_crt_candidates
        i = self.plan.info
        return tm_crt_candidates(i["N"], i["M1"], i["M2"], res["m1"], res["m2"])

    def score_slice(self, x_slice, n0: int, length: int, members):
        import torch
        m = members.to(device=self.t.device, dtype=torch.int64)
        out = torch.zeros(m.numel(), dtype=torch.float64, device=self.t.device)
        self.plan.score_slice(x_slice, n0, length, self.t, m, out)
        return out


def match_sliced(ops, x_slice, n0: int, length: int, owner: int = 0, device=None) -> Optional[dict]:
    """Algorithm 1 for one signal cut into contiguous slices, one per rank
    (x_slice holds entries [n0, n0+length) of the signal).

    Folds are sums over the signal's entries (Eq. (2)), so each rank folds
    its slice and one SUM reduction brings the folds to `owner`, which runs
    steps 4-8 (argmax, closed-form S1 ∩ S2). The members go out by broadcast;
    each rank adds its slice's part of their exact scores (Eq. (1) restricted
    to the slice) and a second SUM reduction gives step 9 on the owner: the
    largest score, ties to the smallest shift. Returns the result on the
    owner, None on the other ranks."""
    import torch
    import torch.distributed as dist
    rank = dist.get_rank() if dist.is_initialized() else 0
    y = ops.fold_slice(x_slice, n0, length)
    dev = device if device is not None else y.device   # the collectives' device (CUDA for NCCL)
    if dist.is_initialized():
        dist.reduce(y, dst=owner, op=dist.ReduceOp.SUM)
    res, members = None, []
    if rank == owner:
        res = ops.correlate_folds(y)
        members = ops.candidates(res)
    cnt = torch.tensor([len(members)], dtype=torch.int64, device=dev)
    if dist.is_initialized():
        dist.broadcast(cnt, src=owner)
    m = torch.tensor(members if rank == owner else [0] * int(cnt.item()), dtype=torch.int64, device=dev)
    if dist.is_initialized() and m.numel() > 0:
        dist.broadcast(m, src=owner)
    sc = ops.score_slice(x_slice, n0, length, m) if m.numel() > 0 else torch.zeros(0, dtype=torch.float64,
                                                                                  device=dev)
    if dist.is_initialized() and sc.numel() > 0:
        sc = sc.to(dev)
        dist.reduce(sc, dst=owner, op=dist.ReduceOp.SUM)
    if rank != owner:
        return None
    out = dict(res)
    flags = int(res["status"]) & ~0xFF & ~0x400            # keep all flags but "score pending"
    if not members:
        out.update(shift=-1, score=0.0, status=1 | flags)  # EMPTY
        return out
    scores = sc.cpu().tolist()
    best = max(range(len(members)), key=lambda c: (scores[c], -members[c]))
    out.update(shift=int(members[best]), score=float(scores[best]),
               status=(0 if len(members) == 1 else 2) | flags)   # FOUND / RESOLVED
    return out
