"""The N > 1 host logic of bench.py on CPU: two gloo ranks on 127.0.0.1.

- the slowest rank's time is taken by every rank (max over ranks) and the whole-job value is
  all ranks' units over that time (independent replicas, weak scaling);
- the reference arm runs on rank 0 only: other ranks return without work.
"""
import os
import socket
import sys

import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, ws, port, q):
    os.environ.update({"MASTER_ADDR": "127.0.0.1", "MASTER_PORT": str(port), "RANK": str(rank),
                       "WORLD_SIZE": str(ws), "LOCAL_RANK": str(rank)})
    sys.path.insert(0, ROOT)
    import torch.distributed as dist
    import bench
    dist.init_process_group("gloo", rank=rank, world_size=ws)
    try:
        ms = 10.0 + 5.0 * rank                 # rank 1 is the slower one
        m = bench.max_over_ranks(ms, ws)
        v = bench.weak_value(1000.0, ws, m * 1e-3)
        assert bench.dist_env() == (ws, rank, rank)
        # the reference arm: only rank 0 would run the oracle
        class A:
            warmup, steps = 0, 0
        if rank != 0:
            assert bench.run_reference(A()) is None
        q.put((rank, m, v))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_take_the_slowest_time():
    ws, port = 2, _free_port()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_worker, args=(r, ws, port, q)) for r in range(ws)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
    assert all(p.exitcode == 0 for p in procs), [p.exitcode for p in procs]
    got = sorted(q.get(timeout=5) for _ in range(ws))
    for rank, m, v in got:
        assert m == 15.0
        assert abs(v - 1000.0 * 2 / 15e-3) <= 1e-9 * v


def test_single_rank_needs_no_process_group():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.max_over_ranks(3.5, 1) == 3.5
    assert bench.weak_value(10.0, 1, 2.0) == 5.0
