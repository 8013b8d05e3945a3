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


def test_partition_units_longest_first():
    import bench
    # 5 -> rank 0, 4 -> rank 1, the 3s to the least-loaded rank in turn
    assert bench.partition_units([5, 4, 3, 3, 3], 2) == [[0, 3], [1, 2, 4]]
    assert bench.partition_units([1, 1, 1], 3) == [[0], [1], [2]]
    with pytest.raises(ValueError):
        bench.partition_units([1, 2], 3)
    with pytest.raises(ValueError):
        bench.partition_units([1, 2], 0)


def test_partition_units_within_the_lpt_bound():
    """Every unit on exactly one rank, and the largest load within
    (4/3 - 1/(3m)) of the best split, found here by brute force."""
    import itertools

    import numpy as np

    import bench
    rng = np.random.default_rng(7)
    for _ in range(40):
        n = int(rng.integers(2, 8))
        m = int(rng.integers(2, min(n, 3) + 1))
        costs = [float(x) for x in rng.integers(1, 50, size=n)]
        parts = bench.partition_units(costs, m)
        assert sorted(i for p in parts for i in p) == list(range(n))
        got = max(sum(costs[i] for i in p) for p in parts)
        best = min(max(sum(c for c, r in zip(costs, asg) if r == k) for k in range(m))
                   for asg in itertools.product(range(m), repeat=n))
        assert got <= (4 / 3 - 1 / (3 * m)) * best + 1e-9


def test_batch_split_balances_the_batched_workload():
    """The batched workload's grid mix (7 of 32^3, 10 of 48^3, 7 of 64^3, 8
    of 96^3) split over 2, 4 and 8 ranks: no rank above 1.1x the mean."""
    import bench
    sizes = [32] * 7 + [48] * 10 + [64] * 7 + [96] * 8
    costs = [bench.rve_cost((s, s, s)) for s in sizes]
    for m in (2, 4, 8):
        loads = [sum(costs[i] for i in p) for p in bench.partition_units(costs, m)]
        assert max(loads) <= 1.1 * sum(loads) / m


def _split_rank(rank, ws, port, costs, out):
    import torch.distributed as tdist
    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    tdist.init_process_group("gloo", rank=rank, world_size=ws)
    try:
        mine = bench.partition_units(costs, ws)[rank]
        total = bench.rank_sum(sum(costs[i] for i in mine), ws)
        count = bench.rank_sum(len(mine), ws)
        got = [None] * ws
        tdist.all_gather_object(got, mine)
        out.put((rank, total, count, got))
    finally:
        tdist.destroy_process_group()


def test_batch_split_over_two_gloo_ranks():
    """Each rank takes its share of the units with no exchange; the sums
    over the ranks give the whole job's units and cost on every rank."""
    import torch.multiprocessing as mp
    costs = [9.0, 1.0, 4.0, 4.0, 2.0, 7.0, 3.0]
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_split_rank, args=(r, 2, port, costs, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = {}
    for _ in procs:
        rank, total, count, got = q.get(timeout=120)
        res[rank] = (total, count, got)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank in (0, 1):
        total, count, got = res[rank]
        assert total == sum(costs) and count == len(costs)
        assert sorted(got[0] + got[1]) == list(range(len(costs)))
        assert not set(got[0]) & set(got[1])


def test_batch_line_names_the_split():
    import argparse

    import bench
    a = argparse.Namespace(config="batch32", steps=10, warmup=3, tol="paper", no_classes=False,
                           batch_threads=None)
    common = dict(sizes={32: 7, 96: 8}, Ntot=1000, total_s=2.0, value=5000.0, e2e_s=None,
                  serial_s=None, launches=10, roof=None, clocks=None, its=4, cuts=0, cls=[],
                  variants={}, vits=40)
    one = bench.batch_line(a, 1, 0, 15, **common)
    assert one["scaling"] == "weak" and one["ms_per_step"] == 200.0
    two = bench.batch_line(a, 2, 0, 15, split=True, **common)
    assert two["scaling"] == "strong" and "split over 2 ranks" in two["config"]["workload"]
    assert "no data exchanged" in two["config"]["parallelism"]
    weak = bench.batch_line(a, 2, 0, 30, **common)
    assert weak["scaling"] == "weak" and "on each of 2 ranks" in weak["config"]["workload"]
    assert bench.batch_line(a, 2, 1, 30, **common) is None
