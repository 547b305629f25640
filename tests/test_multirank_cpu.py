"""Multi-rank host logic on CPU (gloo, world size 2): every rank runs its own
replica of the workload (no data-path collective); the job time is the max
over ranks and the whole-job rate counts every rank's work."""
import os
import socket

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    # rank r "took" (1 + r) seconds for compression and (2 - r) for queries
    tc, tq = bench.reduce_max([1.0 + rank, 2.0 - rank], "cpu")
    ws, rk, _ = bench._dist()
    rate = bench.aggregate_rate(ws, 3, 1e9, tc)
    out[rank] = (tc, tq, ws, rk, rate)
    dist.barrier()
    dist.destroy_process_group()


def test_replicas_reduce_max_over_two_gloo_ranks():
    ctx = mp.get_context("spawn")
    mgr = ctx.Manager()
    out = mgr.dict()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, out)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    for r in range(2):
        tc, tq, ws, rk, rate = out[r]
        assert (tc, tq) == (2.0, 2.0)          # max over ranks
        assert ws == 2 and rk == r
        assert rate == pytest.approx(2 * 3 * 1e9 / 2.0)


def test_single_process_is_identity():
    import bench
    assert bench.reduce_max([1.5, 2.5], "cpu") == [1.5, 2.5]
    assert bench.aggregate_rate(1, 4, 10.0, 2.0) == 20.0
