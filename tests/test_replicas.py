"""Replica bookkeeping of bench.py on CPU: two gloo ranks (one process each).

The solve itself does not shard (replicas only): each rank runs its own sequence with
seeds shifted by 1000 * rank, and the whole-job rate divides every rank's solves by the
slowest rank's time.
"""
import os
import socket

import numpy as np
import pytest
import torch.multiprocessing as mp

import bench


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out):
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        src = bench.sources(8, 2, rank)
        ms_local = 100.0 + 50.0 * rank          # rank 1 is the slow one
        ms_total, value = bench.aggregate(world, 2, 3, ms_local)
        out[rank] = (float(src[0][0, 0, 0]), float(src[1][1, 2, 3]), ms_total, value)
    finally:
        dist.destroy_process_group()


def test_two_replicas_aggregate_over_ranks():
    world = 2
    port = _free_port()
    ctx = mp.get_context("spawn")
    with ctx.Manager() as mgr:
        out = mgr.dict()
        procs = [ctx.Process(target=_rank, args=(r, world, port, out)) for r in range(world)]
        for p in procs:
            p.start()
        for p in procs:
            p.join(120)
            assert p.exitcode == 0
        res = dict(out)
    # distinct inputs per replica
    assert res[0][0] != res[1][0] and res[0][1] != res[1][1]
    # both ranks see the max time and the whole-job rate: 2 ranks x 2 sources x 3 steps / 0.15 s
    for r in range(world):
        assert res[r][2] == pytest.approx(150.0)
        assert res[r][3] == pytest.approx(2 * 2 * 3 / 0.150)


def test_single_rank_needs_no_process_group():
    ms_total, value = bench.aggregate(1, 10, 3, 600.0)
    assert ms_total == 600.0 and value == pytest.approx(50.0)
    a, b = bench.sources(8, 3, 0), bench.sources(8, 3, 1)
    assert not np.array_equal(a[0], b[0])
    np.testing.assert_allclose(a[2] - a[0], 2 * (a[1] - a[0]), atol=1e-12)
