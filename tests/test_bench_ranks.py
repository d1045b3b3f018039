"""Host logic of the multi-rank benchmark on CPU: world size 2 over gloo.  Each
rank is an independent replica; the job is timed by the slowest rank and the
whole-job value counts every rank's units."""
import os
import socket

import pytest
import torch.multiprocessing as mp


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, q):
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    ms = [12.0, 15.0][rank]
    mx = bench.max_over_ranks(ms, world)
    val = bench.job_value(1000.0, world, mx)
    dist.barrier()
    q.put((rank, mx, val))
    dist.destroy_process_group()


def test_max_over_ranks_and_job_value_gloo():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = [q.get(timeout=120) for _ in procs]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, mx, val in out:
        assert mx == 15.0
        assert abs(val - 2 * 1000.0 / 15e-3) < 1e-6


def test_single_rank_identity():
    import bench
    assert bench.max_over_ranks(3.0, 1) == 3.0
    assert bench.job_value(10.0, 1, 2.0) == 5000.0
