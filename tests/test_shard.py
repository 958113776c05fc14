"""Batch sharding over ranks (the multi-GPU form of the batched workload):
contiguous blocks of system indices per rank and a host gather in system
order. Two gloo ranks on the CPU each solve their block of small systems on
one pattern (through the oracle here: no GPU); the gathered solutions must
equal a single-process solve of the whole batch, bit for bit."""
import os
import socket

import numpy as np
import pytest
import torch.multiprocessing as mp

from paper_2110_03636_b300 import shard


@pytest.mark.parametrize("nsys,world", [(5, 2), (256, 8), (3, 4), (0, 2), (7, 1)])
def test_partition_is_contiguous_and_balanced(nsys, world):
    blocks = shard.partition(nsys, world)
    assert len(blocks) == world
    assert blocks[0][0] == 0 and blocks[-1][1] == nsys
    for (a, b), (c, d) in zip(blocks, blocks[1:]):
        assert b == c
    sizes = [b - a for a, b in blocks]
    assert max(sizes) - min(sizes) <= 1 and sizes == sorted(sizes, reverse=True)


def _batch():
    import workloads as W
    base = W.make_config("grid2d_n2000")
    return base, [W.reweight(base, seed=(1, b)) for b in range(5)]


def _solve_block(lo, hi):
    import oracle as O
    base, systems = _batch()
    sym = O.Symbolic(base.n, base.m, base.H_colptr, base.H_rowidx, base.J_rowptr, base.J_colidx)
    dx, dy, rr = [], [], []
    for x in systems[lo:hi]:
        f = O.Factor(sym, x.H_vals, x.J_vals, x.delta, x.gamma)
        a, b, info = f.solve(x.r_x, x.r_y)
        dx.append(a)
        dy.append(b)
        rr.append(info["rr"])
    n, m = base.n, base.m
    return {"dx": np.array(dx).reshape(-1, n), "dy": np.array(dy).reshape(-1, m), "rr": np.array(rr),
            "index": np.arange(lo, hi)}


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out):
    import torch.distributed as D
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    D.init_process_group("gloo", rank=rank, world_size=world)
    try:
        res = shard.solve_sharded(_solve_block, 5, rank, world)
        out.put((rank, res))
    finally:
        D.destroy_process_group()


def test_two_gloo_ranks_solve_their_blocks_and_gather():
    world = 2
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    got = {}
    for _ in range(world):
        r, res = q.get(timeout=300)
        got[r] = res
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert got[1] is None
    merged = got[0]
    ref = _solve_block(0, 5)
    np.testing.assert_array_equal(merged["index"], np.arange(5))
    np.testing.assert_array_equal(merged["dx"], ref["dx"])
    np.testing.assert_array_equal(merged["dy"], ref["dy"])
    assert (merged["rr"] <= 1e-8).all()
