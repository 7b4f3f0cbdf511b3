"""Parity of the CUDA path with the CPU oracle (through the C ABI).

The FP32 path takes its decisions (argmin, greedy order) on FP32 distances
with the same fixed operation order as the oracle's ``decide="fp32"`` mode,
keeps the mass bookkeeping in FP64 in the algorithm's own order, and returns
R as a correctly rounded sum.  So everything is compared bit for bit: the
cost, the plan (as a set of (i, j, f)), the number of rounds and the NNS work.
The oracle also checks, on the CPU, that every FP32 decision agrees with the
FP64 one up to a documented near-tie (gap < 1e-6 relative).
"""
import numpy as np
import pytest

import oracle
from golden_io import all_golden
from paper_2401_07378_gb300 import workloads as wl

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

GOLDEN = __import__("os").path.join(__import__("os").path.dirname(__file__), "golden")


@pytest.fixture(scope="module")
def ctx():
    from paper_2401_07378_gb300 import nnsemd
    c = nnsemd.Context(0)
    yield c
    c.close()


def dev(a, dt):
    return torch.as_tensor(np.ascontiguousarray(a), dtype=dt).cuda()


def gpu_solve(ctx, x, a, y, b, metric, plan=True):
    return ctx.solve(dev(x, torch.float32), dev(a, torch.float64), dev(y, torch.float32), dev(b, torch.float64),
                     metric=metric, plan=plan)


def plan_set(i, j, f):
    i = np.asarray(i.cpu() if hasattr(i, "cpu") else i)
    j = np.asarray(j.cpu() if hasattr(j, "cpu") else j)
    f = np.asarray(f.cpu() if hasattr(f, "cpu") else f)
    order = np.lexsort((j, i))
    return i[order], j[order], f[order]


def assert_parity(res, ref):
    assert res.cost == ref.cost, (res.cost, ref.cost)
    gi, gj, gf = plan_set(res.plan_i, res.plan_j, res.plan_f)
    oi, oj, of = plan_set(ref.plan_i, ref.plan_j, ref.plan_f)
    assert np.array_equal(gi, oi) and np.array_equal(gj, oj)
    assert np.array_equal(gf, of)
    assert res.stats["rounds"] == ref.rounds
    assert res.stats["pair_evals"] == ref.pair_evals
    assert ref.violations == 0
    assert abs(res.stats["leftover_mass"] - ref.leftover) <= 1e-15


@pytest.mark.parametrize("g", all_golden(GOLDEN), ids=lambda g: g.name)
def test_golden_examples_on_gpu(ctx, g):
    ref = oracle.solve(g.x, g.a, g.y, g.b, g.metric, "fp32")
    res = gpu_solve(ctx, g.x, g.a, g.y, g.b, g.metric)
    assert_parity(res, ref)
    assert res.cost == pytest.approx(g.cost, rel=2e-16)


def test_single_pair_256_d2(ctx):
    p = wl.single_pair(0)
    ref = oracle.solve_pair(p, "l2")
    assert_parity(gpu_solve(ctx, p.x, p.a, p.y, p.b, "l2"), ref)


@pytest.mark.parametrize("d", [1, 2, 3, 4, 5, 6, 7, 8])
@pytest.mark.parametrize("metric", ["l2", "sql2", "l1"])
def test_random_pairs_all_d(ctx, d, metric):
    rng = np.random.default_rng(100 + d)
    for m, n, w in ((1, 1, "uniform"), (1, 37, "dirichlet"), (53, 1, "dirichlet"), (300, 700, "dirichlet"),
                    (1500, 1100, "uniform"), (2500, 3100, "dirichlet")):
        p = wl.uniform_pair(m, n, d, int(rng.integers(1 << 30)), w)
        ref = oracle.solve_pair(p, metric)
        assert_parity(gpu_solve(ctx, p.x, p.a, p.y, p.b, metric), ref)


def test_multi_round_colour_clusters(ctx):
    # large enough for several multi-CTA rounds before the one-CTA tail;
    # sizes not multiples of any tile
    p = wl.color_transfer(seed=3, n=20011)
    ref = oracle.solve_pair(p, "sql2")
    assert_parity(gpu_solve(ctx, p.x, p.a, p.y, p.b, "sql2"), ref)


@pytest.mark.parametrize("ratio", [4, 12, 25, 60])
def test_group_sizes_in_multi_cta_rounds(ctx, ratio):
    # n / m consumers per supplier on average: groups of a few (one thread
    # each), of 9..32 (one warp each) and beyond 32 (one CTA each) in the
    # multi-CTA rounds
    n = 6000
    p = wl.uniform_pair(n // ratio, n, 2, 1000 + ratio, "dirichlet")
    for metric in ("l2", "sql2"):
        ref = oracle.solve_pair(p, metric)
        assert_parity(gpu_solve(ctx, p.x, p.a, p.y, p.b, metric), ref)


def test_zero_weights_and_duplicates(ctx):
    rng = np.random.default_rng(5)
    x = rng.integers(0, 4, (3000, 2)).astype(np.float32)   # many exact ties / duplicates
    y = rng.integers(0, 4, (2000, 2)).astype(np.float32)
    a = rng.exponential(1.0, 3000)
    b = rng.exponential(1.0, 2000)
    a[rng.random(3000) < 0.4] = 0.0
    b[rng.random(2000) < 0.4] = 0.0
    for metric in ("l2", "l1"):
        ref = oracle.solve(x, a, y, b, metric)
        assert_parity(gpu_solve(ctx, x, a, y, b, metric), ref)


def test_identical_sets_cost_zero(ctx):
    p = wl.color_transfer(seed=1, n=5000)
    res = gpu_solve(ctx, p.x, p.a, p.x, p.a, "l2")
    assert res.cost == 0.0


def test_one_heavy_supplier_long_groups(ctx):
    # one supplier holds most of the mass: its group spans far more than a
    # warp, which exercises the CTA-level sort of long groups
    rng = np.random.default_rng(6)
    x = rng.random((40, 3)).astype(np.float32)
    y = rng.random((9000, 3)).astype(np.float32)
    a = np.full(40, 1e-3)
    a[7] = 50.0
    b = np.ones(9000)
    ref = oracle.solve(x, a, y, b, "l2")
    assert_parity(gpu_solve(ctx, x, a, y, b, "l2"), ref)


def test_host_entry_point_matches_device(ctx):
    p = wl.uniform_pair(4000, 3500, 3, 9, "dirichlet")
    dev_res = gpu_solve(ctx, p.x, p.a, p.y, p.b, "l2")
    host_res = ctx.solve_host(p.x, p.a, p.y, p.b, metric="l2", plan=True)
    assert host_res.cost == dev_res.cost
    a = plan_set(host_res.plan_i, host_res.plan_j, host_res.plan_f)
    b = plan_set(dev_res.plan_i, dev_res.plan_j, dev_res.plan_f)
    assert all(np.array_equal(u, v) for u, v in zip(a, b))


@pytest.mark.parametrize("d", [2, 3])
def test_batched_small_pairs(ctx, d):
    batch = wl.random_batch(40, seed=d, d=d, lo=1, hi=1024)
    costs, stats = ctx.solve_batched(dev(batch.x, torch.float32), dev(batch.a, torch.float64), batch.x_off,
                                     dev(batch.y, torch.float32), dev(batch.b, torch.float64), batch.y_off,
                                     metric="l2")
    costs = costs.cpu().numpy()
    rounds = 0
    for p in range(batch.num_pairs):
        ref = oracle.solve_pair(batch.pair(p), "l2")
        assert costs[p] == ref.cost, p
        rounds += ref.rounds
    assert stats["rounds"] == rounds


def test_batched_mixes_small_and_large_pairs(ctx):
    pairs = [wl.uniform_pair(m, n, 2, s, "dirichlet") for s, (m, n) in
             enumerate([(10, 20), (1500, 900), (1024, 1024), (3000, 2500), (1, 1)])]
    batch = wl.Batch.pack(pairs)
    costs, _ = ctx.solve_batched(dev(batch.x, torch.float32), dev(batch.a, torch.float64), batch.x_off,
                                 dev(batch.y, torch.float32), dev(batch.b, torch.float64), batch.y_off,
                                 metric="sql2")
    costs = costs.cpu().numpy()
    for p, pr in enumerate(pairs):
        assert costs[p] == oracle.solve_pair(pr, "sql2").cost


@pytest.mark.parametrize("metric", ["l2", "l1"])
def test_batched_high_d_both_kernels(ctx, metric):
    # d > 8, FP32: pairs of at most 512 points per side run on the 256-thread
    # kernel, larger ones on the 1,024-thread kernel, beyond 2,048 multi-CTA
    sizes = [(1, 1), (3, 700), (512, 512), (513, 40), (200, 300), (60, 480), (900, 1100), (2100, 300), (37, 12)]
    pairs = [wl.uniform_pair(m, n, 24, 500 + s, "dirichlet") for s, (m, n) in enumerate(sizes)]
    rb = wl.random_batch(40, 77, 24, 5, 520)
    pairs += [rb.pair(k) for k in range(rb.num_pairs)]
    batch = wl.Batch.pack(pairs)
    costs, stats = ctx.solve_batched(dev(batch.x, torch.float32), dev(batch.a, torch.float64), batch.x_off,
                                     dev(batch.y, torch.float32), dev(batch.b, torch.float64), batch.y_off,
                                     metric=metric)
    costs = costs.cpu().numpy()
    rounds = 0
    for p, pr in enumerate(pairs):
        ref = oracle.solve_pair(pr, metric)
        assert costs[p] == ref.cost, p
        rounds += ref.rounds
    assert stats["rounds"] == rounds


def test_errors_are_reported(ctx):
    from paper_2401_07378_gb300.nnsemd import NNSEMDError
    x = np.zeros((4, 2), np.float32)
    w = np.ones(4)
    bad = x.copy()
    bad[1, 1] = np.nan
    with pytest.raises(NNSEMDError) as e:
        gpu_solve(ctx, bad, w, x, w, "l2")
    assert e.value.status == 2
    with pytest.raises(NNSEMDError) as e:
        gpu_solve(ctx, x, np.array([1.0, -1.0, 1.0, 1.0]), x, w, "l2")
    assert e.value.status == 3
    with pytest.raises(NNSEMDError) as e:
        gpu_solve(ctx, x, np.zeros(4), x, w, "l2")
    assert e.value.status == 3
    with pytest.raises(NNSEMDError) as e:
        ctx.solve(dev(x, torch.float32), dev(w, torch.float64), dev(x, torch.float32), dev(w, torch.float64),
                  metric="l2", precision="fp8")
    assert e.value.status == 8
    bad9 = np.zeros((4, 9), np.float32)
    bad9[2, 7] = np.inf
    with pytest.raises(NNSEMDError) as e:
        gpu_solve(ctx, bad9, w, np.zeros((4, 9), np.float32), w, "l2")
    assert e.value.status == 2
    # the context stays usable after errors
    p = wl.single_pair(2)
    assert gpu_solve(ctx, p.x, p.a, p.y, p.b, "l2").cost == oracle.solve_pair(p, "l2").cost


def test_errors_in_multi_round_solves(ctx):
    # large enough for the multi-CTA rounds: the packing's count kernel
    # reports a non-finite coordinate, also on a point of zero weight
    from paper_2401_07378_gb300.nnsemd import NNSEMDError
    p = wl.uniform_pair(3000, 2500, 3, 17, "dirichlet")
    for zero_weight in (False, True):
        x, a = p.x.copy(), p.a.copy()
        x[1234, 2] = np.nan
        if zero_weight:
            a[1234] = 0.0
        with pytest.raises(NNSEMDError) as e:
            gpu_solve(ctx, x, a, p.y, p.b, "l2")
        assert e.value.status == 2
        y = p.y.copy()
        y[77, 0] = np.inf
        with pytest.raises(NNSEMDError) as e:
            gpu_solve(ctx, p.x, p.a, y, p.b, "sql2")
        assert e.value.status == 2
    assert gpu_solve(ctx, p.x, p.a, p.y, p.b, "l2").cost == oracle.solve_pair(p, "l2").cost


def test_colour_transfer_full_size(ctx):
    """The benchmark's workload (65,536 colours per image, d=3, squared
    Euclidean, full plan) in the benchmark's launch configuration, compared
    bit for bit with the oracle."""
    p = wl.color_transfer(seed=0)
    res = gpu_solve(ctx, p.x, p.a, p.y, p.b, "sql2")
    # properties that hold at any size, checked first
    gi, gj, gf = plan_set(res.plan_i, res.plan_j, res.plan_f)
    assert gf.size == 65536 and np.all(gf == 1.0 / 65536)
    assert np.array_equal(np.sort(gi), np.arange(65536)) and np.array_equal(np.sort(gj), np.arange(65536))
    ref = oracle.solve_pair(p, "sql2")
    assert_parity(res, ref)


# ---------------------------------------------------------------------------
# d > 8: tiled FP32 NNS, index-only active lists, high-d tail and batches
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("d", [9, 16, 64, 130])
@pytest.mark.parametrize("metric", ["l2", "l1"])
def test_random_pairs_high_d(ctx, d, metric):
    rng = np.random.default_rng(200 + d)
    for m, n, w in ((1, 50, "dirichlet"), (70, 1, "uniform"), (257, 190, "dirichlet"), (2100, 1900, "dirichlet")):
        p = wl.uniform_pair(m, n, d, int(rng.integers(1 << 30)), w)
        ref = oracle.solve_pair(p, metric)
        assert_parity(gpu_solve(ctx, p.x, p.a, p.y, p.b, metric), ref)


def test_gmm_pair_d64(ctx):
    p = wl.gmm_pair(seed=1, n=6000, d=64)
    ref = oracle.solve_pair(p, "l2")
    assert_parity(gpu_solve(ctx, p.x, p.a, p.y, p.b, "l2"), ref)


def test_batched_documents_d300(ctx):
    batch = wl.doc_knn(num_docs=48, seed=3, vocab_size=5000)
    costs, stats = ctx.solve_batched(dev(batch.x, torch.float32), dev(batch.a, torch.float64), batch.x_off,
                                     dev(batch.y, torch.float32), dev(batch.b, torch.float64), batch.y_off,
                                     metric="l2")
    costs = costs.cpu().numpy()
    rounds = 0
    for k in range(batch.num_pairs):
        ref = oracle.solve_pair(batch.pair(k), "l2")
        assert costs[k] == ref.cost, k
        rounds += ref.rounds
    assert stats["rounds"] == rounds


def test_batched_retrieval_signatures_d128(ctx):
    batch = wl.retrieval(num_pairs=6, seed=4, lo=256, hi=2048)
    costs, _ = ctx.solve_batched(dev(batch.x, torch.float32), dev(batch.a, torch.float64), batch.x_off,
                                 dev(batch.y, torch.float32), dev(batch.b, torch.float64), batch.y_off,
                                 metric="l2")
    costs = costs.cpu().numpy()
    for k in range(batch.num_pairs):
        assert costs[k] == oracle.solve_pair(batch.pair(k), "l2").cost, k


# ---------------------------------------------------------------------------
# reduced precision: tcgen05 contraction proposes, FP32 re-rank decides,
# certificate or FP32 rescan -- the result must equal the FP32 path's
# ---------------------------------------------------------------------------

def gpu_solve_prec(ctx, x, a, y, b, metric, precision):
    return ctx.solve(dev(x, torch.float32), dev(a, torch.float64), dev(y, torch.float32), dev(b, torch.float64),
                     metric=metric, precision=precision, plan=True)


@pytest.mark.parametrize("precision", ["bf16", "fp16", "fp8", "bf16x3"])
def test_reduced_precision_small_pair(ctx, precision):
    p = wl.uniform_pair(300, 260, 64, 31, "dirichlet")
    ref = oracle.solve_pair(p, "l2")
    res = gpu_solve_prec(ctx, p.x, p.a, p.y, p.b, "l2", precision)
    assert_parity(res, ref)


@pytest.mark.parametrize("precision", ["bf16", "fp16", "fp8", "bf16x3"])
@pytest.mark.parametrize("shape", ["gmm64", "sift128", "words300"])
def test_reduced_precision_equals_fp32(ctx, precision, shape):
    if precision == "bf16x3" and shape == "words300":
        pytest.skip("BF16X3 serves d <= 128 (test_bf16x3_beyond_its_dimension_is_unsupported)")
    if shape == "gmm64":
        p = wl.gmm_pair(seed=2, n=5000, d=64)
    elif shape == "sift128":
        p = wl.retrieval(num_pairs=1, seed=5, lo=2000, hi=2048).pair(0)
    else:
        b = wl.doc_knn(num_docs=1, seed=6, vocab_size=3000, median=400, lo=300, hi=500)
        p = b.pair(0)
    for metric in ("l2", "sql2"):
        ref = oracle.solve_pair(p, metric)
        res = gpu_solve_prec(ctx, p.x, p.a, p.y, p.b, metric, precision)
        assert_parity(res, ref)
        s = res.stats
        assert s["certified"] + s["fallbacks"] > 0
        if precision in ("bf16", "fp16") and shape != "words300":
            assert s["certified"] >= 0.5 * (s["certified"] + s["fallbacks"]), s


def test_bf16x3_certifies_where_bf16_cannot(ctx):
    # points far from the origin relative to their spread (a common offset
    # of 20 against unit noise in d = 16): the error of one BF16 copy,
    # about 2^-7 |x||y|, dwarfs the distance gaps and leaves the searches to
    # the FP32 rescan; the split form's 3 * 2^-16 |x||y| certifies them
    p = wl.uniform_pair(3000, 2500, 16, 4, "dirichlet")
    rng = np.random.default_rng(4)
    p.x = (20.0 + rng.normal(0, 1, p.x.shape)).astype(np.float32)
    p.y = (20.0 + rng.normal(0, 1, p.y.shape)).astype(np.float32)
    ref = oracle.solve_pair(p, "l2")
    one = gpu_solve_prec(ctx, p.x, p.a, p.y, p.b, "l2", "bf16")
    split = gpu_solve_prec(ctx, p.x, p.a, p.y, p.b, "l2", "bf16x3")
    assert_parity(one, ref)
    assert_parity(split, ref)
    s = split.stats
    assert s["fallbacks"] <= 0.05 * (s["certified"] + s["fallbacks"]), s
    assert one.stats["fallbacks"] >= 0.5 * (one.stats["certified"] + one.stats["fallbacks"]), one.stats


def test_bf16x3_beyond_its_dimension_is_unsupported(ctx):
    from paper_2401_07378_gb300.nnsemd import NNSEMDError
    p = wl.uniform_pair(40, 30, 300, 8)
    with pytest.raises(NNSEMDError) as e:
        gpu_solve_prec(ctx, p.x, p.a, p.y, p.b, "l2", "bf16x3")
    assert e.value.status == 8


def test_reduced_precision_rejections(ctx):
    from paper_2401_07378_gb300.nnsemd import NNSEMDError
    p = wl.uniform_pair(50, 40, 16, 7)
    with pytest.raises(NNSEMDError) as e:
        gpu_solve_prec(ctx, p.x, p.a, p.y, p.b, "l1", "bf16")
    assert e.value.status == 8
