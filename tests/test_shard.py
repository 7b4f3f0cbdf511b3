"""Splitting one batch over ranks (paper_2401_07378_gb300/shard.py), on CPU.

Checks the partition (every pair exactly once, the longest-processing-time
bound on the largest load) and, with two gloo ranks, that the costs
gathered to every rank in pair order equal a single-rank run.  The CPU
oracle stands in for each rank's GPU solve: the host logic under test is the
same."""
import os
import socket

import numpy as np
import pytest

import oracle
from paper_2401_07378_gb300 import shard
from paper_2401_07378_gb300 import workloads as wl


def test_partition_covers_every_pair_once_and_balances():
    rng = np.random.default_rng(0)
    for ranks in (1, 2, 3, 4, 8):
        for _ in range(5):
            work = rng.integers(1, 10 ** 6, size=int(rng.integers(1, 400)))
            shares = shard.partition(work, ranks)
            assert len(shares) == ranks
            allp = np.sort(np.concatenate(shares))
            assert np.array_equal(allp, np.arange(work.size))
            for s in shares:
                assert np.all(np.diff(s) > 0)
            loads = [int(work[s].sum()) for s in shares]
            lower = max(work.sum() / ranks, work.max())      # no split does better than this
            assert max(loads) <= (4.0 / 3.0 - 1.0 / (3 * ranks)) * lower + 1e-9 * lower or max(loads) == work.max()


def test_partition_is_deterministic_and_handles_fewer_pairs_than_ranks():
    work = np.array([5, 5, 5], np.int64)
    a, b = shard.partition(work, 4), shard.partition(work, 4)
    assert all(np.array_equal(x, y) for x, y in zip(a, b))
    assert sorted(int(s.size) for s in a) == [0, 1, 1, 1]


def test_sub_batch_gathers_the_pairs_it_names():
    batch = wl.random_batch(9, seed=3, d=3, lo=5, hi=40)
    ids = np.array([7, 0, 4], np.int64)
    sb = shard.sub_batch(batch, ids)
    for k, p in enumerate(ids):
        got = wl.Batch(sb.x, sb.a, sb.x_off, sb.y, sb.b, sb.y_off).pair(k)
        want = batch.pair(int(p))
        for u, v in ((got.x, want.x), (got.a, want.a), (got.y, want.y), (got.b, want.b)):
            assert np.array_equal(u, v)


def test_pair_work_is_m_times_n():
    batch = wl.random_batch(6, seed=5, d=2, lo=3, hi=30)
    w = shard.pair_work(batch.x_off, batch.y_off)
    for p in range(6):
        q = batch.pair(p)
        assert w[p] == q.m * q.n
    assert np.array_equal(shard.pair_work(batch.x_off, n_shared=7), np.diff(batch.x_off) * 7)


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, q):
    import torch
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        batch = wl.random_batch(23, seed=11, d=2, lo=10, hi=120)
        shares = shard.partition(shard.pair_work(batch.x_off, batch.y_off), world)
        sb = shard.sub_batch(batch, shares[rank])
        local = [oracle.solve_pair(wl.Batch(sb.x, sb.a, sb.x_off, sb.y, sb.b, sb.y_off).pair(k), "l2").cost
                 for k in range(sb.num_pairs)]
        costs = shard.gather_costs(torch.tensor(local, dtype=torch.float64), shares, batch.num_pairs, rank)
        q.put((rank, costs.tolist()))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_gather_the_single_rank_costs():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    got = dict(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    batch = wl.random_batch(23, seed=11, d=2, lo=10, hi=120)
    want = [oracle.solve_pair(batch.pair(k), "l2").cost for k in range(batch.num_pairs)]
    assert got[0] == want
    assert got[1] == want
