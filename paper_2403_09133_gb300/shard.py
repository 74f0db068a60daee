"""Several GPUs, one process each, on independent problems: which rank solves which problem
of a batch, and the max-over-ranks reduction of timings.

Problems of a batch are independent SDPs, so ranks exchange nothing on the data path: each
rank solves its own share in one persistent launch, and only the timings and counts meet at
the end (one small all-reduce, never inside a timed region).  The partition is the
longest-processing-time rule: problems in decreasing order of estimated work, each to the
rank with the least work so far (ties to the lower rank), which every rank computes alike.
"""
from __future__ import annotations

from typing import List, Sequence


def work_estimate(n: int, nnz: int) -> float:
    """Work of one solve, proportional to rows plus stored entries (a CG iteration touches
    each once); the same estimate orders problems inside a batch launch."""
    return float(n) + float(nnz)


def assign(works: Sequence[float], world: int) -> List[int]:
    """Rank of every problem under the longest-processing-time rule."""
    if world < 1:
        raise ValueError("world must be >= 1")
    order = sorted(range(len(works)), key=lambda i: (-float(works[i]), i))
    load = [0.0] * world
    owner = [0] * len(works)
    for i in order:
        r = min(range(world), key=lambda k: (load[k], k))
        owner[i] = r
        load[r] += float(works[i])
    return owner


def shard(works: Sequence[float], rank: int, world: int) -> List[int]:
    """Indices of the problems `rank` solves, in increasing order."""
    if not 0 <= rank < world:
        raise ValueError("rank out of range")
    owner = assign(works, world)
    return [i for i, r in enumerate(owner) if r == rank]


def _reduce(values: Sequence[float], op_name: str, device=None) -> List[float]:
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return [float(v) for v in values]
    t = torch.tensor([float(v) for v in values], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=getattr(dist.ReduceOp, op_name))
    return t.tolist()


def max_over_ranks(values: Sequence[float], device=None) -> List[float]:
    """Element-wise maximum over the ranks of the default process group (the values
    themselves without one); `device` is where the backend reduces (cuda for NCCL)."""
    return _reduce(values, "MAX", device)


def sum_over_ranks(values: Sequence[float], device=None) -> List[float]:
    return _reduce(values, "SUM", device)
