"""Solve options on the GPU: rerank_k (how many reduced-precision candidates
the exact FP32 re-rank sees) changes only how often the certificate holds,
never a result; its range is checked; the near-tie count of the
reduced-precision scan is reported, and is 0 on the FP32 paths."""
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


def pair_dev(p):
    return dev(p.x, torch.float32), dev(p.a, torch.float64), dev(p.y, torch.float32), dev(p.b, torch.float64)


def test_rerank_k_changes_certification_not_results(ctx):
    p = wl.gmm_pair(seed=5, n=6000)
    ref = oracle.solve_pair(p, "l2")
    t = pair_dev(p)
    fallbacks = {}
    for k in (1, 2, 4, 8, 16, 0):
        r = ctx.solve(*t, metric="l2", precision="bf16", rerank_k=k, plan=True)
        assert r.cost == ref.cost, k
        assert r.stats["rounds"] == ref.rounds
        assert r.stats["near_ties"] >= 0
        fallbacks[k] = r.stats["fallbacks"]
    # a smaller re-rank set can only weaken the certificate (0 = all 16)
    assert fallbacks[1] >= fallbacks[2] >= fallbacks[4] >= fallbacks[8] >= fallbacks[16] == fallbacks[0]


def test_rerank_k_in_the_batched_kernel(ctx):
    batch = wl.doc_knn(num_docs=24, seed=3, vocab_size=3000)
    x, a, y, b = dev(batch.x, torch.float32), dev(batch.a, torch.float64), dev(batch.y, torch.float32), dev(
        batch.b, torch.float64)
    want = [oracle.solve_pair(batch.pair(k), "l2").cost for k in range(batch.num_pairs)]
    for k in (1, 3, 8, 16):
        costs, stats = ctx.solve_batched(x, a, batch.x_off, y, b, batch.y_off, metric="l2", precision="fp16",
                                         rerank_k=k)
        assert costs.cpu().numpy().tolist() == want, k
        assert stats["near_ties"] >= 0


def test_rerank_k_outside_its_range_is_rejected(ctx):
    from paper_2401_07378_gb300 import nnsemd
    p = wl.gmm_pair(seed=6, n=500)
    t = pair_dev(p)
    for k in (-1, 17):
        with pytest.raises(nnsemd.NNSEMDError) as e:
            ctx.solve(*t, metric="l2", precision="bf16", rerank_k=k)
        assert e.value.status == 1


def test_fp32_paths_report_no_near_ties(ctx):
    for p, metric in ((wl.uniform_pair(3000, 2500, 3, 1, "dirichlet"), "l2"), (wl.gmm_pair(seed=2, n=3000), "l2")):
        r = ctx.solve(*pair_dev(p), metric=metric)
        assert r.stats["near_ties"] == 0
        assert r.cost == oracle.solve_pair(p, metric).cost
