"""Batch sharding over GPUs: host logic only.

One KKT system does not shard (its factor is one elimination tree), but a
batch of systems on one pattern does: rank r of W takes a contiguous block
of system indices, analyses the pattern itself (or reuses a loaded
analysis), factors and solves its block on its own GPU, and the solutions
and statistics are gathered on the host. No collective touches the data
path; the gather moves host arrays over a CPU process group.
"""
from __future__ import annotations

import numpy as np

__all__ = ["partition", "gather_blocks", "solve_sharded"]


def partition(nsys: int, world: int) -> list[tuple[int, int]]:
    """Contiguous, balanced blocks [lo, hi) of nsys system indices over world
    ranks: the first nsys % world ranks take one system more. Ranks beyond
    nsys get empty blocks."""
    if nsys < 0 or world < 1:
        raise ValueError("nsys >= 0 and world >= 1 required")
    q, r = divmod(nsys, world)
    out, lo = [], 0
    for k in range(world):
        hi = lo + q + (1 if k < r else 0)
        out.append((lo, hi))
        lo = hi
    return out


def gather_blocks(block: dict, rank: int, world: int, group=None, dst: int = 0):
    """Gather each rank's result dict {name: array with the block's systems
    along axis 0} on rank dst and concatenate the blocks in rank order
    (= system order). Returns the merged dict on dst, None elsewhere. With
    world == 1 the block is returned as is."""
    if world == 1:
        return block
    import torch.distributed as D
    objs = [None] * world if rank == dst else None
    D.gather_object(block, objs, dst=dst, group=group)
    if rank != dst:
        return None
    keys = objs[0].keys()
    return {k: np.concatenate([np.asarray(o[k]) for o in objs if len(o[k])], axis=0)
            if any(len(o[k]) for o in objs) else np.asarray(objs[0][k]) for k in keys}


def solve_sharded(solve_block, nsys: int, rank: int, world: int, group=None, dst: int = 0):
    """Runs solve_block(lo, hi) -> dict of per-system arrays on this rank's
    block of the batch and gathers the blocks on rank dst (see partition and
    gather_blocks)."""
    lo, hi = partition(nsys, world)[rank]
    return gather_blocks(solve_block(lo, hi), rank, world, group=group, dst=dst)
