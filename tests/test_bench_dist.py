"""The benchmark's multi-rank host logic (replicas on N GPUs, timed as the
slowest rank) on two gloo ranks on the CPU: the barrier lets every rank
through and the max over ranks returns the slowest rank's time on all
ranks; one rank alone returns its own value without a process group."""
import os
import socket
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, ws, port, out):
    import torch.distributed as tdist
    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    tdist.init_process_group("gloo", rank=rank, world_size=ws)
    try:
        bench.rank_barrier(ws)
        t = bench.rank_max(1.5 + rank, ws)
        bench.rank_barrier(ws)
        out.put((rank, t))
    finally:
        tdist.destroy_process_group()


def test_rank_max_over_two_gloo_ranks():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = dict(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert res == {0: 2.5, 1: 2.5}


def test_single_rank_needs_no_process_group():
    import bench
    bench.rank_barrier(1)
    assert bench.rank_max(3.25, 1) == 3.25
