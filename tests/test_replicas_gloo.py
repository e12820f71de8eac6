"""The multi-GPU launch of bench.py on the host side: N replicas, one process per
GPU, with a barrier before the timed region and the maximum time over ranks.
Run here as two gloo processes on the CPU (no GPU, no data-path collective)."""

import os
import socket

import pytest
import torch.multiprocessing as mp


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _rank(rank, world, port, q):
    import sys
    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    os.environ.update({"RANK": str(rank), "WORLD_SIZE": str(world), "MASTER_ADDR": "127.0.0.1",
                       "MASTER_PORT": str(port)})
    import bench
    r, w, dist = bench.dist_setup(world)
    dist.barrier()
    worst = bench.max_over_ranks(10.0 + 5.0 * r, dist)     # rank r "took" 10 + 5 r ms
    q.put((r, w, worst))
    dist.barrier()
    dist.destroy_process_group()


def test_two_replicas_report_the_slowest_rank():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    got = sorted(q.get(timeout=5) for _ in range(2))
    assert got == [(0, 2, 15.0), (1, 2, 15.0)]


def test_single_rank_needs_no_process_group():
    import sys
    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    import bench
    assert bench.dist_setup(1) == (0, 1, None)
    assert bench.max_over_ranks(3.5, None) == 3.5
