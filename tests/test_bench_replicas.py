"""bench.py's replica aggregation on two gloo ranks (CPU): the slowest rank's time and the sum of the
ranks' units give the whole-job throughput; barriers pair up across ranks."""
import os
import socket

import pytest


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    import bench
    import torch.distributed as td
    bench.dist_init("gloo")
    assert bench.dist_info() == (world, rank, rank)
    bench.barrier()
    t = bench.reduce_over_ranks(10.0 + rank, "max")      # per-rank step times
    u = bench.reduce_over_ranks(100.0 * (rank + 1), "sum")  # per-rank units
    bench.barrier()
    out.put((rank, t, u))
    td.destroy_process_group()


def test_replica_aggregation_two_gloo_ranks():
    mp = pytest.importorskip("torch.multiprocessing")
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert res == [(0, 11.0, 300.0), (1, 11.0, 300.0)]


def test_single_process_has_no_group():
    import bench
    assert bench.reduce_over_ranks(3.5, "max") == 3.5
    bench.barrier()  # no process group: nothing to wait for
