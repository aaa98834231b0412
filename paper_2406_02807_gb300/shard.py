"""Work partition across processes (one GPU each).

Queries are independent and the tree is a read-only replica, so the path shards with
no data exchange: each rank builds and uploads its own copy of the tree and answers
its own slice of the queries.  The only collectives are for measurement (a barrier and
the maximum of the ranks' times).
"""
from __future__ import annotations


def shard_range(total: int, rank: int, world: int) -> tuple[int, int]:
    """Contiguous [begin, end) slice of `total` items for `rank` of `world` (strong
    scaling: the slices cover every item once, sizes differ by at most one)."""
    if world < 1 or not 0 <= rank < world or total < 0:
        raise ValueError("need world >= 1, 0 <= rank < world and total >= 0")
    base, extra = divmod(total, world)
    begin = rank * base + min(rank, extra)
    return begin, begin + base + (1 if rank < extra else 0)


def weak_slice(per_rank: int, rank: int) -> tuple[int, int]:
    """[begin, end) of a rank's own `per_rank` items in one global sequence (weak
    scaling: every rank gets the same amount of work, disjoint from the others)."""
    if per_rank < 0 or rank < 0:
        raise ValueError("need per_rank >= 0 and rank >= 0")
    return rank * per_rank, (rank + 1) * per_rank


def max_over_ranks(value: float, dist=None, device=None) -> float:
    """The maximum of `value` over the ranks of the default process group (the value
    itself without one)."""
    if dist is None or not dist.is_available() or not dist.is_initialized():
        return float(value)
    import torch
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())
