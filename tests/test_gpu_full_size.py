"""Parity at the sizes the benchmark workloads are quoted at.

- Documents: the whole batch of 4,096 documents against one query (d = 300,
  50,000-word vocabulary), BF16 distances with FP32 re-rank, replayed as a
  CUDA graph: every pair's R equals the oracle's.
- Retrieval: the whole 10,000-pair batch (d = 128, 256..2,048 descriptors
  per side), FP16 distances with autotuned tiles: every R equals the FP32
  GPU path's, and a seeded 200-pair subset equals the oracle's.
- GMM with the learned proposal at the configuration's size (4,096 cells,
  hidden width 256, trained on 200 seeded plain runs): a 16,384-point pair
  (the largest the oracle finishes in seconds on the host cores) solved with
  the FP32 and the BF16 fallback gives the oracle's plan bit for bit.

The pairs are independent problems (Sec. III-D), so the oracle solves them
in parallel on the host (one process per pair, or its multi-core twin for a
single large pair).
"""
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


@pytest.fixture(scope="module")
def pool():
    with oracle.process_pool() as p:
        yield p


def dev(a, dt):
    return torch.as_tensor(np.ascontiguousarray(a), dtype=dt).cuda()


def batch_on_device(batch):
    return (dev(batch.x, torch.float32), dev(batch.a, torch.float64), dev(batch.y, torch.float32),
            dev(batch.b, torch.float64))


def test_full_document_batch_bf16_graph_equals_oracle(ctx, pool):
    from paper_2401_07378_gb300 import nnsemd
    batch = wl.doc_knn(num_docs=4096, seed=0)
    x, a, y, b = batch_on_device(batch)
    costs = torch.empty(batch.num_pairs, dtype=torch.float64, device="cuda")
    first = None
    for _ in range(2):  # capture, then replay of the captured graph
        costs.fill_(float("nan"))
        _, stats = ctx.solve_batched(x, a, batch.x_off, y, b, batch.y_off, metric="l2", precision="bf16",
                                     costs=costs, flags=nnsemd.FLAG_GRAPH)
        got = costs.cpu().numpy().copy()
        if first is None:
            first = got
    assert np.array_equal(got, first)
    ref = oracle.solve_many([batch.pair(k) for k in range(batch.num_pairs)], "l2", pool=pool)
    want = np.array([r.cost for r in ref])
    bad = np.nonzero(got != want)[0]
    assert bad.size == 0, (bad[:10], got[bad[:10]], want[bad[:10]])
    assert stats["rounds"] == sum(r.rounds for r in ref)


def test_full_retrieval_batch_fp16_autotuned(ctx, pool):
    from paper_2401_07378_gb300 import nnsemd
    batch = wl.retrieval(num_pairs=10000, seed=0)
    x, a, y, b = batch_on_device(batch)
    costs, stats = ctx.solve_batched(x, a, batch.x_off, y, b, batch.y_off, metric="l2", precision="fp16",
                                     flags=nnsemd.FLAG_AUTOTUNE)
    got = costs.cpu().numpy()
    plain, _ = ctx.solve_batched(x, a, batch.x_off, y, b, batch.y_off, metric="l2", precision="fp32")
    assert np.array_equal(got, plain.cpu().numpy())
    assert stats["certified"] + stats["fallbacks"] > 0
    del x, a, y, b
    ids = sorted(int(p) for p in np.random.default_rng(0).choice(batch.num_pairs, size=200, replace=False))
    ref = oracle.solve_many([batch.pair(k) for k in ids], "l2", pool=pool)
    for k, r in zip(ids, ref):
        assert got[k] == r.cost, k


@pytest.fixture(scope="module")
def full_prop(ctx):
    """The proposal of the GMM configuration: 4,096 cells, hidden 256, trained
    on round-one traces of 200 seeded plain runs."""
    from paper_2401_07378_gb300 import proposal_training
    prop, info = proposal_training.build_gmm_proposal(ctx)
    assert info["cells"] == 4096 and info["hidden"] == 256 and info["runs"] == 200
    yield prop
    prop.close()


@pytest.mark.parametrize("precision", ["fp32", "bf16"])
def test_learned_gmm_at_the_configured_size_equals_oracle(ctx, full_prop, precision):
    p = wl.gmm_pair(seed=0, n=16384)
    t = [dev(v, dt) for v, dt in ((p.x, torch.float32), (p.a, torch.float64), (p.y, torch.float32),
                                  (p.b, torch.float64))]
    res = ctx.solve(*t, metric="l2", precision=precision, plan=True, proposal=full_prop)
    ref = oracle.solve_pair(p, "l2", threads=0)
    assert res.cost == ref.cost
    assert res.stats["rounds"] == ref.rounds
    assert res.stats["pair_evals"] == ref.pair_evals
    got = sorted(zip(res.plan_i.cpu().tolist(), res.plan_j.cpu().tolist(), res.plan_f.cpu().tolist()))
    want = sorted(zip(ref.plan_i.tolist(), ref.plan_j.tolist(), ref.plan_f.tolist()))
    assert got == want
    assert res.stats["certified"] > 0
