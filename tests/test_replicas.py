"""Multi-GPU form of the benchmark, host side: N independent replicas
(one KKT system does not shard), each rank taking the value sets from its
own offset, and the max over ranks of the timed region. Runs as two gloo
ranks on the CPU."""
import os
import socket

import pytest
import torch.multiprocessing as mp

import bench


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out):
    import torch
    import torch.distributed as D
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    D.init_process_group("gloo", rank=rank, world_size=world)
    try:
        sets = [bench.value_set(t, rank) for t in range(bench.N_VALUE_SETS)]
        mx = bench.max_over_ranks(10.0 * (rank + 1), torch.device("cpu"))
        out.put((rank, sets, mx))
    finally:
        D.destroy_process_group()


def test_two_gloo_replicas():
    world = 2
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    res = dict()
    for _ in range(world):
        r, sets, mx = q.get(timeout=120)
        res[r] = (sets, mx)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    # every rank cycles through all value sets, from its own offset
    for r in range(world):
        assert sorted(res[r][0]) == list(range(bench.N_VALUE_SETS))
        assert res[r][0][0] == r
    # the timed region is the slowest rank's
    assert res[0][1] == res[1][1] == 20.0


def test_single_process_max_is_identity():
    import torch
    assert bench.max_over_ranks(3.5, torch.device("cpu")) == 3.5
