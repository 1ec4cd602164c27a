"""Voxel sharding across ranks (one process per GPU).

Voxels and chains are independent and nothing is exchanged during a run, so a
volume splits into contiguous voxel ranges with no collective on the data
path.  The RNG counter uses the global voxel index (voxel_base + local
index), so the pieces reproduce the unsplit run exactly; gathering results is
a host-side concatenation along the voxel axis.
"""
from __future__ import annotations


def strong_range(n_vox: int, rank: int, world: int) -> tuple:
    """(first, count) of rank's share of a fixed volume of n_vox voxels."""
    if world < 1 or not 0 <= rank < world:
        raise ValueError("bad rank/world")
    base, extra = divmod(n_vox, world)
    first = rank * base + min(rank, extra)
    return first, base + (1 if rank < extra else 0)


def weak_range(n_per_rank: int, rank: int) -> tuple:
    """(first, count) of rank's volume when every rank samples n_per_rank
    voxels of one larger volume (weak scaling)."""
    if rank < 0 or n_per_rank < 0:
        raise ValueError("bad rank/size")
    return rank * n_per_rank, n_per_rank
