"""Batched reduced-precision solves (one persistent launch, tensor-core NNS
inside every pair's CTA), the autotuner and CUDA-graph replay: every cost
must equal the CPU oracle's bit for bit (the FP32 re-rank + certificate +
FP32 rescan make the reduced-precision path exact)."""
import numpy as np
import pytest

import oracle
from paper_2401_07378_gb300 import workloads as wl

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    from paper_2401_07378_gb300 import nnsemd
    c = nnsemd.Context(0)
    yield c
    c.close()


def dev(a, dt):
    return torch.as_tensor(np.ascontiguousarray(a), dtype=dt).cuda()


def run_batch(ctx, batch, metric, precision, flags=0):
    return ctx.solve_batched(dev(batch.x, torch.float32), dev(batch.a, torch.float64), batch.x_off,
                             dev(batch.y, torch.float32), dev(batch.b, torch.float64), batch.y_off,
                             metric=metric, precision=precision, flags=flags)


@pytest.mark.parametrize("precision", ["bf16", "fp16", "fp8"])
def test_batched_documents_reduced_precision(ctx, precision):
    batch = wl.doc_knn(num_docs=40, seed=8, vocab_size=4000)
    costs, stats = run_batch(ctx, batch, "l2", precision)
    costs = costs.cpu().numpy()
    rounds = 0
    for k in range(batch.num_pairs):
        ref = oracle.solve_pair(batch.pair(k), "l2")
        assert costs[k] == ref.cost, k
        rounds += ref.rounds
    assert stats["rounds"] == rounds
    assert stats["certified"] + stats["fallbacks"] > 0


def test_batched_bf16x3_small_pairs(ctx):
    batch = wl.random_batch(20, seed=12, d=48, lo=20, hi=400)
    costs, stats = run_batch(ctx, batch, "l2", "bf16x3")
    costs = costs.cpu().numpy()
    for k in range(batch.num_pairs):
        assert costs[k] == oracle.solve_pair(batch.pair(k), "l2").cost, k
    assert stats["fallbacks"] <= 0.01 * (stats["certified"] + stats["fallbacks"]), stats


@pytest.mark.parametrize("precision", ["bf16", "fp16", "fp8"])
def test_batched_retrieval_reduced_precision(ctx, precision):
    batch = wl.retrieval(num_pairs=5, seed=9, lo=600, hi=2048)
    costs, stats = run_batch(ctx, batch, "sql2", precision)
    costs = costs.cpu().numpy()
    for k in range(batch.num_pairs):
        assert costs[k] == oracle.solve_pair(batch.pair(k), "sql2").cost, k
    if precision != "fp8":
        assert stats["certified"] >= 0.5 * (stats["certified"] + stats["fallbacks"]), stats


def test_batched_mixed_sizes_with_large_pairs(ctx):
    # pairs above 2,048 points go through the single-pair tensor-core path
    pairs = [wl.uniform_pair(m, n, 24, s, "dirichlet") for s, (m, n) in
             enumerate([(10, 30), (700, 300), (2500, 2100), (1, 1), (2048, 2048)])]
    batch = wl.Batch.pack(pairs)
    costs, _ = run_batch(ctx, batch, "l2", "bf16")
    costs = costs.cpu().numpy()
    for k, p in enumerate(pairs):
        assert costs[k] == oracle.solve_pair(p, "l2").cost, k


def test_autotune_and_graph_replay(ctx):
    from paper_2401_07378_gb300 import nnsemd
    batch = wl.retrieval(num_pairs=12, seed=10, lo=200, hi=900)
    x, a = dev(batch.x, torch.float32), dev(batch.a, torch.float64)
    y, b = dev(batch.y, torch.float32), dev(batch.b, torch.float64)
    costs = torch.empty(batch.num_pairs, dtype=torch.float64, device="cuda")
    flags = nnsemd.FLAG_AUTOTUNE | nnsemd.FLAG_GRAPH
    want = np.array([oracle.solve_pair(batch.pair(k), "l2").cost for k in range(batch.num_pairs)])
    for _ in range(3):  # tune + capture, then two replays
        costs.fill_(float("nan"))
        ctx.solve_batched(x, a, batch.x_off, y, b, batch.y_off, metric="l2", precision="fp16", costs=costs,
                          flags=flags)
        assert np.array_equal(costs.cpu().numpy(), want)
    # new weights in the same buffers: the replayed graph reads them
    rng = np.random.default_rng(11)
    a2 = rng.exponential(1.0, batch.a.shape[0])
    a.copy_(torch.as_tensor(a2))
    ctx.solve_batched(x, a, batch.x_off, y, b, batch.y_off, metric="l2", precision="fp16", costs=costs,
                      flags=flags)
    got = costs.cpu().numpy()
    for k in range(batch.num_pairs):
        p = batch.pair(k)
        xs, xe = int(batch.x_off[k]), int(batch.x_off[k + 1])
        assert got[k] == oracle.solve(p.x, a2[xs:xe], p.y, p.b, "l2").cost, k


def test_single_pair_reduced_precision_through_host_entry(ctx):
    p = wl.gmm_pair(seed=3, n=3000, d=64)
    res = ctx.solve_host(p.x, p.a, p.y, p.b, metric="l2", precision="bf16", plan=True)
    ref = oracle.solve_pair(p, "l2")
    assert res.cost == ref.cost
    assert res.stats["certified"] > 0
