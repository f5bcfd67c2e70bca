"""The multi-rank benchmark path on CPU: two gloo ranks, each timing an
independent replica; the job time is the slowest rank's and the updates add."""
import os
import socket

import pytest


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out):
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    ms, upd = bench.reduce_over_ranks(10.0 + 5.0 * rank, 1000.0 * (rank + 1), dist, "cpu")
    dist.barrier()
    out.put((rank, ms, upd))
    dist.destroy_process_group()


def test_reduce_over_two_gloo_ranks():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert res == [(0, 15.0, 3000.0), (1, 15.0, 3000.0)]


def test_reduce_without_process_group():
    import bench
    assert bench.reduce_over_ranks(3.0, 7.0) == (3.0, 7.0)
