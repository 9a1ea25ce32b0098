"""Multi-GPU runs are replicas (independent solves, no data-path
collective); the only cross-rank step is the timing reduction.  Checked
here with two gloo ranks on the CPU."""
import os
import socket

import pytest


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, q):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    ms = [120.0, 200.0][rank]          # rank 1 is the slow replica
    ms_max, rate = bench.job_rate(dist, world, 10, ms)
    bench.barrier(dist)
    q.put((rank, ms_max, rate))
    dist.destroy_process_group()


def test_job_rate_uses_slowest_rank_and_all_units():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = [q.get(timeout=120) for _ in range(2)]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, ms_max, rate in out:
        assert ms_max == 200.0
        assert abs(rate - 2 * 10 / 0.2) < 1e-9


def test_single_process_rate():
    import bench
    ms_max, rate = bench.job_rate(None, 1, 5, 250.0)
    assert ms_max == 250.0 and abs(rate - 20.0) < 1e-12
