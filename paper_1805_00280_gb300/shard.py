"""Walk-id sharding over ranks (one GPU per rank, no collective on the data path).

Walks are independent units (FN-Multi's observation, Section 3.4 of the
paper), so N ranks split a job by walk id.  With weak scaling every rank runs
the per-GPU workload -- r walks from each start vertex -- as its own rounds of
one N*r-round job: rank k owns walk ids [k*S*r, (k+1)*S*r) of the job
"r*N walks from each of the S starts".  The union over ranks is exactly that
job, so gathering the rows in rank order reproduces one device running it.
"""
from __future__ import annotations


def weak_shard(world: int, rank: int, n_starts: int, r: int) -> tuple[int, int, int]:
    """(r_total, walk_begin, walk_count) of this rank's share under weak scaling."""
    if world < 1 or not 0 <= rank < world or n_starts < 1 or r < 1:
        raise ValueError("bad shard arguments")
    per = n_starts * r
    return r * world, rank * per, per


def strong_shard(world: int, rank: int, total_walks: int) -> tuple[int, int]:
    """(walk_begin, walk_count) of this rank's share of a fixed job (strong scaling):
    contiguous, sizes differing by at most one."""
    if world < 1 or not 0 <= rank < world or total_walks < 0:
        raise ValueError("bad shard arguments")
    base, extra = divmod(total_walks, world)
    begin = rank * base + min(rank, extra)
    return begin, base + (1 if rank < extra else 0)
