"""Sharding of the path's units over ranks.

Histories (and RNG streams) are independent units: a unit's seed depends
only on its id (Eqs. 2-4), so ranks split the ids into contiguous ranges and
exchange nothing on the data path.  The int64 fixed-point tallies and the
integer counters of the ranks then sum, in any order, to the bits one rank
running every unit produces.  bench.py and the multi-rank tests take their
ranges from here.
"""
from __future__ import annotations


def rank_range(rank: int, world: int, total: int) -> tuple[int, int]:
    """Strong scaling: rank `rank` of `world` owns ids [lo, hi) of [0, total)
    (contiguous, sizes differing by at most one)."""
    if not 0 <= rank < world:
        raise ValueError(f"rank {rank} outside a world of {world}")
    return rank * total // world, (rank + 1) * total // world


def weak_range(rank: int, per_rank: int) -> tuple[int, int]:
    """Weak scaling: every rank owns `per_rank` ids, rank r the r-th block."""
    if rank < 0:
        raise ValueError(f"rank {rank} is negative")
    return rank * per_rank, (rank + 1) * per_rank
