"""Sample sharding across ranks (one process per GPU).

Samples are independent and the sampler is counter-based, so rank g of G takes
the contiguous Philox index range [offset + g*N_rank, offset + (g+1)*N_rank)
and needs no data exchange; per-rank integer counts add up exactly, in any
order, to the counts of one process over the whole range.
"""
from __future__ import annotations


def shard_range(n_per_rank: int, rank: int, world: int, offset: int = 0):
    """(offset, N) of this rank's samples under weak scaling (n_per_rank each)."""
    if not (0 <= rank < world):
        raise ValueError("rank out of range")
    return offset + rank * n_per_rank, n_per_rank


def combine_counts(t, group=None):
    """Sum int64 counts (counts3 or grad counts) over ranks; exact."""
    import torch.distributed as dist
    if dist.is_available() and dist.is_initialized() and dist.get_world_size(group) > 1:
        dist.all_reduce(t, op=dist.ReduceOp.SUM, group=group)
    return t
