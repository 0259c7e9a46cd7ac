"""Band sharding across ranks (one process per GPU).

Bands are independent transforms (Sec. 2.2: the same transform on every
column of Psi), so a batch splits across ranks with no exchange on the data
path; the only collectives are the timing barrier and a max over ranks of
the step time. Each rank creates its own plan for its shard.
"""
from __future__ import annotations


def band_shard(total_bands: int, world: int, rank: int):
    """Contiguous [start, start + count) of a batch of total_bands; shard
    sizes differ by at most one band."""
    if world < 1 or not (0 <= rank < world) or total_bands < 0:
        raise ValueError("need world >= 1, 0 <= rank < world, total_bands >= 0")
    base, extra = divmod(total_bands, world)
    start = rank * base + min(rank, extra)
    return start, base + (1 if rank < extra else 0)


def max_over_ranks(value: float, device=None) -> float:
    """Largest value over all ranks of the default process group (the value
    itself when torch.distributed is not initialised)."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()):
        return float(value)
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())
