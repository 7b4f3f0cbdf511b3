"""The multi-core twin of the oracle returns exactly what the serial oracle
returns: R, Alg. 1's sequential R, the plan in the same order, the residuals,
rounds, pair evaluations, the per-round NN trace and the near-tie counts.
It is what times the oracle on all host cores and checks the large parity
cases, so it is held to the serial oracle bit for bit."""
import numpy as np
import pytest

import oracle
from paper_2401_07378_gb300 import workloads as wl


def _same(r1, r2):
    assert r1.cost == r2.cost
    assert r1.cost_seq == r2.cost_seq
    assert np.array_equal(r1.plan_i, r2.plan_i)
    assert np.array_equal(r1.plan_j, r2.plan_j)
    assert np.array_equal(r1.plan_f, r2.plan_f)
    assert np.array_equal(r1.plan_term, r2.plan_term)
    assert np.array_equal(r1.s_left, r2.s_left) and np.array_equal(r1.c_left, r2.c_left)
    assert (r1.rounds, r1.pair_evals, r1.near_ties, r1.violations) == (r2.rounds, r2.pair_evals, r2.near_ties,
                                                                      r2.violations)
    assert r1.max_rel_gap == r2.max_rel_gap
    assert np.array_equal(r1.m_t, r2.m_t) and np.array_equal(r1.n_t, r2.n_t)


def _grid_pair(m, n, d, seed):
    """Integer grid points with many exact ties and duplicates, 30 % zero weights."""
    rng = np.random.default_rng(seed)
    x = rng.integers(0, 4, size=(m, d)).astype(np.float32)
    y = rng.integers(0, 4, size=(n, d)).astype(np.float32)
    a = rng.integers(0, 3, size=m).astype(np.float64)
    b = rng.integers(0, 3, size=n).astype(np.float64)
    a[0] = b[0] = 1.0
    return wl.Pair(x, a, y, b)


@pytest.mark.parametrize("metric", ["l2", "sql2", "l1"])
@pytest.mark.parametrize("decide", ["fp32", "fp64"])
def test_twin_equals_serial_oracle_on_random_pairs(metric, decide):
    for k, (m, n, d) in enumerate([(1, 1, 2), (1, 40, 3), (37, 1, 5), (300, 700, 2), (513, 257, 8), (120, 90, 64)]):
        p = wl.uniform_pair(m, n, d, 500 + k, "dirichlet")
        _same(oracle.solve_pair(p, metric, decide, trace=True),
              oracle.solve_pair(p, metric, decide, trace=True, threads=4))
        r = oracle.solve_pair(p, metric, decide, threads=0)
        assert np.array_equal(r.plan_f, oracle.solve_pair(p, metric, decide).plan_f)


def test_twin_equals_serial_oracle_on_ties_duplicates_and_zero_weights():
    for seed in range(6):
        p = _grid_pair(200 + 31 * seed, 150 + 17 * seed, 2 + seed % 3, seed)
        for metric in ("l2", "l1"):
            _same(oracle.solve_pair(p, metric, trace=True), oracle.solve_pair(p, metric, trace=True, threads=3))


def test_twin_equals_serial_oracle_under_the_random_protocol():
    p = wl.uniform_pair(400, 650, 3, 77, "dirichlet")
    for seed in (0, 1, 12345):
        _same(oracle.solve_pair(p, "l2", protocol="random", seed=seed, trace=True),
              oracle.solve_pair(p, "l2", protocol="random", seed=seed, trace=True, threads=5))


def test_twin_equals_serial_oracle_on_a_colour_cluster_pair():
    p = wl.color_transfer(seed=3, n=3000)
    _same(oracle.solve_pair(p, "sql2", trace=True), oracle.solve_pair(p, "sql2", trace=True, threads=0))


def test_solve_many_keeps_the_pair_order():
    batch = wl.random_batch(12, seed=4, d=3, lo=20, hi=90)
    pairs = [batch.pair(k) for k in range(batch.num_pairs)]
    many = oracle.solve_many(pairs, "l2", workers=4)
    for p, r in zip(pairs, many):
        assert r.cost == oracle.solve_pair(p, "l2").cost
