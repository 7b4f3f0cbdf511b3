"""Pins of the CPU oracle against what the paper and the mathematics fix.

None of these compares the oracle with itself: each check is a hand-worked
value, a brute-force optimum, a closed form, an invariant or a special case of
the paper's theorems (Lemma 1, Thm. 1, Thm. 2), chosen so that a plausible
mistake in the oracle (a flipped tie-break, a reversed greedy order, a skipped
consumer, a dropped distance term, a lost weight update) fails at least one of
them -- ``test_mutants_are_caught`` plants such mistakes to show it.
"""
import itertools
import math
import os
import shutil
import subprocess
import tempfile
from fractions import Fraction

import numpy as np
import pytest

import oracle
from golden_io import all_golden
from paper_2401_07378_gb300 import workloads as wl

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def dist_matrix(x, y, metric):
    """Ground distances D_ij in float64 by numpy broadcasting."""
    diff = x.astype(np.float64)[:, None, :] - y.astype(np.float64)[None, :, :]
    if metric == "l1":
        return np.abs(diff).sum(-1)
    d2 = (diff * diff).sum(-1)
    return np.sqrt(d2) if metric == "l2" else d2


_PERMS = {k: np.array(list(itertools.permutations(range(k))), np.int64) for k in range(1, 9)}


def exact_emd_equal_weights(x, y, metric):
    """Exact EMD for n=m and equal weights: by Birkhoff-von Neumann the
    optimum of the transport LP is a permutation, so enumerate them all."""
    k = x.shape[0]
    D = dist_matrix(x, y, metric)
    perms = _PERMS[k]
    costs = D[np.arange(k)[None, :], perms].sum(1) / k
    best = int(np.argmin(costs))
    return float(costs[best]), perms[best]


# ---------------------------------------------------------------------------
# the correctly rounded total used for normalisation (Sec. II-A)
# ---------------------------------------------------------------------------

def test_fsum_is_correctly_rounded():
    rng = np.random.default_rng(7)
    cases = [rng.random(n) * 10.0 ** rng.integers(-300, 300, n) for n in (1, 2, 7, 100, 1000)]
    cases += [rng.exponential(1.0, 5000), [1.0, 2.0 ** -53], [1.0, 2.0 ** -53, 2.0 ** -105],
              [2.0 ** -1074] * 3, [1e308, 1e308 * 0.5, -0.0 + 1e-300], [0.1] * 10]
    for v in cases:
        v = [float(t) for t in v]
        exact = float(sum((Fraction(t) for t in v), Fraction(0)))
        assert math.fsum(v) == exact


# ---------------------------------------------------------------------------
# P6: hand-worked examples
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("g", all_golden(GOLDEN), ids=lambda g: g.name)
@pytest.mark.parametrize("decide", ["fp32", "fp64"])
def test_golden_examples(g, decide):
    assert g.cost == pytest.approx(g.cost_from_expr(), rel=1e-15)
    r = oracle.solve(g.x, g.a, g.y, g.b, g.metric, decide, trace=True)
    assert r.rounds == g.rounds
    # per-round nearest-neighbour choices
    off = 0
    for t in range(r.rounds):
        nt = int(r.n_t[t])
        assert list(r.trace_nn[off:off + nt]) == g.nn[t + 1], f"round {t + 1}"
        off += nt
    got = sorted(zip(r.plan_i.tolist(), r.plan_j.tolist(), r.plan_f.tolist()))
    assert got == sorted(g.plan)
    assert r.cost == pytest.approx(g.cost, rel=2e-16, abs=0)
    assert r.cost_seq == pytest.approx(g.cost, rel=4e-16, abs=0)
    # Thm. 1 lower side
    assert r.cost >= g.emd * (1 - 1e-15)


# ---------------------------------------------------------------------------
# P3 + Thm. 1: never below the exact EMD, and within the theorem's bound
# ---------------------------------------------------------------------------

def _thm1_bound(r, x, y, metric, perm, k):
    """Right-hand side of Thm. 1 with F^opt the optimal permutation plan:
    sum_i D_{i,j*_i} * sum_{j in J_i} (c_j - F^opt_ij)."""
    D = dist_matrix(x, y, metric)
    c = np.full(k, 1.0 / k)
    bound = 0.0
    for i in range(k):
        sel = r.plan_i == i
        J = r.plan_j[sel][r.plan_f[sel] > 0]
        if J.size == 0:
            continue
        jstar_d = D[i, J].max()
        fopt = np.where(perm[i] == J, 1.0 / k, 0.0)
        bound += jstar_d * float(np.sum(c[J] - fopt))
    return bound


@pytest.mark.parametrize("metric", ["l2", "sql2", "l1"])
def test_never_below_bruteforce_emd(metric):
    rng = np.random.default_rng({"l2": 1, "sql2": 2, "l1": 3}[metric])
    for case in range(700):
        k = int(rng.integers(1, 9))
        d = int(rng.integers(1, 4))
        kind = case % 3
        if kind == 0:
            x = rng.random((k, d)).astype(np.float32)
            y = rng.random((k, d)).astype(np.float32)
        else:  # small integer grid: many exact ties and duplicate points
            x = rng.integers(0, 3, (k, d)).astype(np.float32)
            y = rng.integers(0, 3, (k, d)).astype(np.float32)
        w = np.ones(k)
        emd, perm = exact_emd_equal_weights(x, y, metric)
        for decide in ("fp64", "fp32"):
            r = oracle.solve(x, w, y, w, metric, decide)
            assert r.cost >= emd - 1e-12 * max(1.0, emd), (case, r.cost, emd)
            slack = _thm1_bound(r, x, y, metric, perm, k)
            assert r.cost - emd <= slack + 1e-12 * max(1.0, emd), (case, r.cost, emd, slack)


# ---------------------------------------------------------------------------
# P1, P2, P7: feasibility (Lemma 1), cost identity, termination bounds
# ---------------------------------------------------------------------------

def _random_problem(rng, m, n, d, weights):
    x = rng.random((m, d)).astype(np.float32)
    y = rng.random((n, d)).astype(np.float32)
    if weights == "dirichlet":
        a, b = rng.exponential(1.0, m), rng.exponential(1.0, n)
    elif weights == "sparse":
        a, b = rng.exponential(1.0, m), rng.exponential(1.0, n)
        a[rng.random(m) < 0.3] = 0.0
        b[rng.random(n) < 0.3] = 0.0
        a[0] = max(a[0], 0.1)
        b[0] = max(b[0], 0.1)
    else:
        a, b = np.ones(m), np.ones(n)
    return x, a, y, b


@pytest.mark.parametrize("metric", ["l2", "sql2", "l1"])
@pytest.mark.parametrize("weights", ["uniform", "dirichlet", "sparse"])
def test_feasible_plan_and_cost_identity(metric, weights):
    rng = np.random.default_rng(["l2", "sql2", "l1"].index(metric) * 10 + ["uniform", "dirichlet", "sparse"].index(weights))
    for _ in range(12):
        m = int(rng.integers(1, 120))
        n = int(rng.integers(1, 120))
        d = int(rng.integers(1, 9))
        x, a, y, b = _random_problem(rng, m, n, d, weights)
        r = oracle.solve(x, a, y, b, metric, "fp64")
        # Lemma 1: row sums = s_i and column sums = c_j, up to what is left
        rows = np.zeros(m)
        cols = np.zeros(n)
        np.add.at(rows, r.plan_i, r.plan_f)
        np.add.at(cols, r.plan_j, r.plan_f)
        np.testing.assert_allclose(rows + r.s_left, r.s, rtol=0, atol=1e-13)
        np.testing.assert_allclose(cols + r.c_left, r.c, rtol=0, atol=1e-13)
        assert np.all(r.plan_f > 0)
        # termination: one side is spent exactly, and the rest is rounding
        assert np.all(r.s_left == 0) or np.all(r.c_left == 0)
        assert r.leftover <= 1e-13
        # Eq. (objective): R = sum_ij F_ij D_ij, recomputed independently
        D = dist_matrix(x, y, metric)
        ref = math.fsum((r.plan_f * D[r.plan_i, r.plan_j]).tolist())
        assert r.cost == pytest.approx(ref, rel=1e-13, abs=1e-300)
        # rounds and plan size are at most m+n-1; no (i,j) gets flow twice
        mm, nn = int(np.count_nonzero(a)), int(np.count_nonzero(b))
        assert 1 <= r.rounds <= mm + nn - 1
        assert r.plan_f.size <= mm + nn - 1
        assert len(set(zip(r.plan_i.tolist(), r.plan_j.tolist()))) == r.plan_f.size
        # zero-weight points never take part
        assert np.all(a[r.plan_i] > 0) and np.all(b[r.plan_j] > 0)
        # work count: sum over rounds of m_t * n_t, first round is all points
        assert r.pair_evals == int(np.sum(r.m_t * r.n_t))
        assert r.m_t[0] == mm and r.n_t[0] == nn


# ---------------------------------------------------------------------------
# P4, P5: closed forms and Thm. 2 special cases
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("metric", ["l2", "sql2", "l1"])
def test_identical_inputs_cost_zero(metric):
    rng = np.random.default_rng(11)
    for k in (1, 5, 64, 300):
        x = rng.random((k, 3)).astype(np.float32)
        x[k // 2:] = x[: k - k // 2]          # duplicated points
        a = rng.exponential(1.0, k)
        r = oracle.solve(x, a, x.copy(), a.copy(), metric, "fp32")
        assert r.cost == 0.0
        assert r.rounds >= 1


@pytest.mark.parametrize("metric", ["l2", "sql2", "l1"])
def test_single_supplier_or_consumer_closed_form(metric):
    rng = np.random.default_rng(12)
    for k in (1, 2, 17, 200):
        x = rng.random((1, 4)).astype(np.float32)
        y = rng.random((k, 4)).astype(np.float32)
        b = rng.exponential(1.0, k)
        D = dist_matrix(x, y, metric)[0]
        c = b / math.fsum(b.tolist())
        r = oracle.solve(x, [3.0], y, b, metric)          # m = 1
        assert r.cost == pytest.approx(math.fsum((c * D).tolist()), rel=1e-13)
        assert r.rounds == 1 and r.plan_f.size == k
        r2 = oracle.solve(y, b, x, [3.0], metric)         # n = 1
        assert r2.cost == pytest.approx(math.fsum((c * D).tolist()), rel=1e-13)


def test_separated_mutual_pairs_are_exact():
    """Thm. 2: no consumer of a supplier received mass earlier -> R = EMD."""
    rng = np.random.default_rng(13)
    for _ in range(50):
        k = int(rng.integers(1, 9))
        centres = rng.permutation(64)[:k].astype(np.float32)[:, None] * np.float32(10.0)
        x = centres + rng.random((k, 1)).astype(np.float32)
        y = centres + rng.random((k, 1)).astype(np.float32)
        w = np.ones(k)
        emd, _ = exact_emd_equal_weights(x, y, "l2")
        r = oracle.solve(x, w, y, w, "l2")
        assert r.rounds == 1
        assert r.cost == pytest.approx(emd, rel=1e-14)


# ---------------------------------------------------------------------------
# P8, P9: invariances and the uniform equal-size structure
# ---------------------------------------------------------------------------

def test_invariances():
    rng = np.random.default_rng(14)
    x = (rng.integers(0, 4096, (80, 3)) / 4096.0).astype(np.float32)
    y = (rng.integers(0, 4096, (70, 3)) / 4096.0).astype(np.float32)
    a, b = rng.exponential(1.0, 80), rng.exponential(1.0, 70)
    base = {m: oracle.solve(x, a, y, b, m) for m in ("l2", "sql2", "l1")}
    # translation by an exactly representable offset
    shift = np.float32(0.5)
    for m in base:
        assert oracle.solve(x + shift, a, y + shift, b, m).cost == base[m].cost
    # scaling by 2 (exact): L2 and L1 double, squared L2 quadruples
    two = np.float32(2.0)
    assert oracle.solve(x * two, a, y * two, b, "l2").cost == 2 * base["l2"].cost
    assert oracle.solve(x * two, a, y * two, b, "l1").cost == 2 * base["l1"].cost
    assert oracle.solve(x * two, a, y * two, b, "sql2").cost == 4 * base["sql2"].cost
    # weight scaling is undone by the normalisation
    assert oracle.solve(x, a * 8, y, b * 0.25, "l2").cost == base["l2"].cost
    # relabelling points (continuous coordinates: no ties) keeps R
    xc = rng.random((90, 2)).astype(np.float32)
    yc = rng.random((60, 2)).astype(np.float32)
    ac, bc = rng.exponential(1.0, 90), rng.exponential(1.0, 60)
    r0 = oracle.solve(xc, ac, yc, bc, "l2")
    pi, pj = rng.permutation(90), rng.permutation(60)
    r1 = oracle.solve(xc[pi], ac[pi], yc[pj], bc[pj], "l2")
    assert r1.cost == r0.cost and r1.rounds == r0.rounds


def test_uniform_equal_size_plan_is_a_permutation():
    p = wl.single_pair(seed=0)
    r = oracle.solve_pair(p, "l2")
    assert r.plan_f.size == 256
    assert np.all(r.plan_f == 1.0 / 256)
    assert sorted(r.plan_i.tolist()) == list(range(256))
    assert sorted(r.plan_j.tolist()) == list(range(256))


# ---------------------------------------------------------------------------
# the NNS step against a brute-force argmin; FP32 decisions vs FP64
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("metric", ["l2", "l1"])
def test_first_round_nn_is_bruteforce_argmin(metric):
    rng = np.random.default_rng(15)
    for grid in (False, True):
        if grid:
            x = rng.integers(0, 5, (60, 2)).astype(np.float32)
            y = rng.integers(0, 5, (50, 2)).astype(np.float32)
        else:
            x = rng.random((60, 5)).astype(np.float32)
            y = rng.random((50, 5)).astype(np.float32)
        a, b = rng.exponential(1.0, 60), rng.exponential(1.0, 50)
        r = oracle.solve(x, a, y, b, metric, "fp64", trace=True)
        D = dist_matrix(x, y, metric)
        want = np.argmin(D, axis=0)          # first (lowest) index on ties
        assert np.array_equal(r.trace_nn[:50], want)
        assert np.array_equal(r.trace_j[:50], np.arange(50))


def test_fp32_decisions_match_fp64_up_to_near_ties():
    for pair, metric in ((wl.single_pair(0), "l2"), (wl.color_transfer(0, n=2048), "sql2"),
                         (wl.uniform_pair(500, 300, 8, 3, "dirichlet"), "l1")):
        r32 = oracle.solve_pair(pair, metric, "fp32")
        r64 = oracle.solve_pair(pair, metric, "fp64")
        assert r32.violations == 0
        assert abs(r32.cost - r64.cost) <= 1e-5 * r64.cost


# ---------------------------------------------------------------------------
# input errors
# ---------------------------------------------------------------------------

def test_errors():
    x = np.zeros((2, 2), np.float32)
    with pytest.raises(oracle.OracleError):
        oracle.solve(x, [1, -1], x, [1, 1])
    with pytest.raises(oracle.OracleError):
        oracle.solve(x, [0, 0], x, [1, 1])
    with pytest.raises(oracle.OracleError):
        oracle.solve(np.array([[0, np.nan], [0, 0]], np.float32), [1, 1], x, [1, 1])
    with pytest.raises(oracle.OracleError):
        oracle.solve(x, [1, np.inf], x, [1, 1])


# ---------------------------------------------------------------------------
# the pins above catch planted mistakes
# ---------------------------------------------------------------------------

MUTANTS = {
    "argmin_ties_to_highest": ("if (best64_i < 0 || k < best64)", "if (best64_i < 0 || k <= best64)"),
    "greedy_descending": ("if (a->k64 < b->k64) return -1;", "if (a->k64 < b->k64) return 1;"),
    "skips_last_consumer": ("for (int64_t l = 0; l < L && s[i] > 0.0; ++l)",
                            "for (int64_t l = 0; l + 1 < L && s[i] > 0.0; ++l)"),
    "drops_first_dim": ("double acc = t * t;", "double acc = 0.0 * t;"),
    "no_consumer_update": ("c[j] = c[j] - f;", "c[j] = c[j];"),
    "cost_without_sqrt": ("return metric == METRIC_L2 ? sqrt(k) : k;", "return k;"),
}


def _mutant_lib(tmp, name):
    src = open(os.path.join(os.path.dirname(oracle.__file__), "nnsemd_oracle.c")).read()
    old, new = MUTANTS[name]
    assert src.count(old) == 1, name
    path = os.path.join(tmp, f"{name}.c")
    with open(path, "w") as fh:
        fh.write(src.replace(old, new))
    so = os.path.join(tmp, f"lib{name}.so")
    subprocess.run(["gcc", "-std=c11", "-O2", "-ffp-contract=off", "-fPIC", "-shared", "-o", so, path, "-lm"],
                   check=True)
    return so


def _pins_pass() -> bool:
    """A quick subset of the pins above, returning False at the first failure."""
    try:
        for g in all_golden(GOLDEN):
            r = oracle.solve(g.x, g.a, g.y, g.b, g.metric, "fp64", trace=True)
            got = sorted(zip(r.plan_i.tolist(), r.plan_j.tolist(), r.plan_f.tolist()))
            if got != sorted(g.plan) or abs(r.cost - g.cost) > 1e-12 * g.cost:
                return False
            if r.rounds != g.rounds or list(r.trace_nn[: int(r.n_t[0])]) != g.nn[1]:
                return False
        rng = np.random.default_rng(5)
        for _ in range(200):
            k = int(rng.integers(1, 7))
            x = rng.integers(0, 3, (k, 2)).astype(np.float32)
            y = rng.integers(0, 3, (k, 2)).astype(np.float32)
            emd, _ = exact_emd_equal_weights(x, y, "l2")
            r = oracle.solve(x, np.ones(k), y, np.ones(k), "l2", "fp64")
            if r.cost < emd - 1e-12:
                return False
    except Exception:
        return False
    return True


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_mutants_are_caught(name, monkeypatch):
    import ctypes
    tmp = tempfile.mkdtemp()
    try:
        so = _mutant_lib(tmp, name)
        lib = ctypes.CDLL(so)
        real = oracle._load()
        lib.oracle_nnsemd.argtypes = real.oracle_nnsemd.argtypes
        lib.oracle_nnsemd.restype = ctypes.c_int
        assert _pins_pass()                       # the real oracle passes
        monkeypatch.setattr(oracle, "_lib", lib)
        assert not _pins_pass(), f"mutant {name} slipped through the pins"
    finally:
        shutil.rmtree(tmp, ignore_errors=True)
