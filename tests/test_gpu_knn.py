"""EMD-kNN on the GPU: nnsemd_solve_one_to_many's distances equal the CPU
oracle's bit for bit and equal nnsemd_solve_batched's with the query
replicated, so the kNN decisions are the oracle's."""
import numpy as np
import pytest

import oracle
from paper_2401_07378_gb300 import knn, workloads as wl

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    from paper_2401_07378_gb300 import nnsemd
    c = nnsemd.Context(0)
    yield c
    c.close()


@pytest.mark.parametrize("d,precision", [(2, "fp32"), (32, "fp32"), (32, "bf16")])
def test_distances_and_decisions(ctx, d, precision):
    docs = wl.labelled_documents(classes=3, docs_per_class=10, queries_per_class=2, seed=5, d=d)
    model = knn.EMDKNN(ctx, docs.x, docs.a, docs.x_off, docs.labels, precision=precision)
    P = len(docs.labels)
    for (y, b), lab in zip(docs.queries, docs.query_labels):
        dist = model.distances(y, b)
        ref = np.array([oracle.solve(docs.x[docs.x_off[p]:docs.x_off[p + 1]],
                                     docs.a[docs.x_off[p]:docs.x_off[p + 1]], y, b, "l2").cost for p in range(P)])
        assert np.array_equal(dist, ref)
        assert knn.vote(dist, docs.labels, 3) == knn.vote(ref, docs.labels, 3)
        assert model.classify(y, b) == lab
    # the same distances through the replicated-query batch
    y, b = docs.queries[0]
    t = lambda v, dt: torch.from_numpy(np.ascontiguousarray(v)).to("cuda", dt)
    rep_y = np.concatenate([y] * P)
    rep_b = np.concatenate([b] * P)
    y_off = np.arange(P + 1, dtype=np.int64) * len(b)
    costs, _ = ctx.solve_batched(t(docs.x, torch.float32), t(docs.a, torch.float64), docs.x_off,
                                 t(rep_y, torch.float32), t(rep_b, torch.float64), y_off, precision=precision)
    assert np.array_equal(costs.cpu().numpy(), model.distances(y, b))


def test_large_query_uses_the_multi_cta_path(ctx):
    # a query larger than the one-CTA capacity: every pair takes the
    # multi-CTA path with the shared consumer rows
    rng = np.random.default_rng(9)
    y = rng.random((2600, 3)).astype(np.float32)
    b = rng.exponential(1.0, 2600)
    xs = [rng.random((m, 3)).astype(np.float32) for m in (50, 1200, 3000)]
    ws = [rng.exponential(1.0, len(x)) for x in xs]
    x_off = np.concatenate([[0], np.cumsum([len(x) for x in xs])]).astype(np.int64)
    model = knn.EMDKNN(ctx, np.concatenate(xs), np.concatenate(ws), x_off, np.zeros(3, int), metric="sql2")
    dist = model.distances(y, b)
    for p in range(3):
        assert dist[p] == oracle.solve(xs[p], ws[p], y, b, "sql2").cost
