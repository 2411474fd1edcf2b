"""Multi-GPU host logic: the path shards by session (and eye), with the scene
replicated on every rank and no data-path collective.  The only collectives
are the timing barrier and the max-over-ranks reduction of elapsed times.
"""

from __future__ import annotations

from typing import List, Sequence, TypeVar

T = TypeVar("T")


def shard(items: Sequence[T], rank: int, world: int) -> List[T]:
    """Round-robin share of independent units (sessions) for one rank."""
    if world < 1 or not 0 <= rank < world:
        raise ValueError(f"bad rank {rank} of {world}")
    return [it for i, it in enumerate(items) if i % world == rank]


def max_over_ranks(values: Sequence[float], device: str = "cpu") -> List[float]:
    """Element-wise maximum of per-rank values (all ranks get the result)."""
    import torch
    import torch.distributed as dist
    t = torch.tensor(list(values), dtype=torch.float64, device=device)
    if dist.is_available() and dist.is_initialized() and dist.get_world_size() > 1:
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return [float(x) for x in t.cpu()]
