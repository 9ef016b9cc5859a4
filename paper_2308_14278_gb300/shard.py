"""Work partition across GPUs (one process per GPU).

Rays are independent (§3.2 Level 3), so a map shards without any exchange
during shooting:

  * one map over N ranks: each rank shoots a contiguous range of the ray
    lattice made of whole level-1 row bands (32-row groups when there are
    fewer bands than ranks), and the integer count maps are summed once at
    the end.  Integer addition is exact and order-independent, so the summed
    map is bit-identical to the map shot on one GPU;
  * many maps (a batch) over N ranks: each rank takes whole maps, balanced by
    ray count, and nothing is exchanged.

This module holds the partition and the reduction only; the shooting is the
library's (ml_shoot_rays with the rank's range).
"""
from __future__ import annotations


def ray_ranges(n3x: int, n3y: int, n1y: int, world: int):
    """[begin, end) lattice ray ranges of the ranks: contiguous, disjoint,
    covering all n3x * n3y rays, cut at level-1 row-band boundaries (n1y rows)
    or, with fewer bands than ranks, at 32-row boundaries; the row units are
    spread so that rank loads differ by at most one unit."""
    if world < 1:
        raise ValueError("world must be >= 1")
    unit = n1y if (n3y + n1y - 1) // n1y >= world else 32
    n_units = (n3y + unit - 1) // unit
    out = []
    for r in range(world):
        u0 = (r * n_units) // world
        u1 = ((r + 1) * n_units) // world
        j0 = min(n3y, u0 * unit)
        j1 = min(n3y, u1 * unit)
        out.append((j0 * n3x, j1 * n3x))
    return out


def maps_for_rank(ray_counts, rank: int, world: int):
    """Indices of the maps that rank `rank` shoots: greedy longest-first
    assignment of whole maps to the least-loaded rank (ties to the lower
    rank), deterministic on every rank."""
    order = sorted(range(len(ray_counts)), key=lambda i: (-ray_counts[i], i))
    load = [0] * world
    mine = []
    for i in order:
        r = min(range(world), key=lambda q: (load[q], q))
        load[r] += ray_counts[i]
        if r == rank:
            mine.append(i)
    return sorted(mine)


def reduce_counts(counts, dst=None, group=None):
    """Sum the ranks' integer count maps in place: onto rank `dst` only
    (torch.distributed.reduce; the other ranks' buffers are then undefined),
    or onto every rank when dst is None (all_reduce).  Integer addition is
    exact, so the result is the one-GPU map.

    The library's counts are uint32; they travel as int32 because that is the
    32-bit integer type the collectives reduce.  Two's-complement int32
    addition wraps modulo 2^32 exactly as uint32 addition does, so the sum's
    bits are the uint32 sum's; a pixel that wraps is then caught by the map
    sum check of ml_field_stats, as on one GPU."""
    import torch.distributed as dist
    if dst is None:
        dist.all_reduce(counts, op=dist.ReduceOp.SUM, group=group)
    else:
        dist.reduce(counts, dst=dst, op=dist.ReduceOp.SUM, group=group)
    return counts
