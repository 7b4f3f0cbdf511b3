"""The seeded input generators match the recipes they state (the stand-ins
for the paper's workloads): shapes, dtypes, ranges, weight laws, length
laws, determinism.  CPU only; small instances of each generator."""
import numpy as np
import pytest

from paper_2401_07378_gb300 import workloads as wl


def test_single_pair_recipe():
    p = wl.single_pair(0)
    assert p.x.shape == (256, 2) and p.y.shape == (256, 2)
    assert p.x.dtype == np.float32 and p.a.dtype == np.float64
    assert p.x.min() >= 0.0 and p.x.max() < 1.0 and p.y.min() >= 0.0 and p.y.max() < 1.0
    assert np.all(p.a == 1.0) and np.all(p.b == 1.0)
    q = wl.single_pair(0)
    assert np.array_equal(p.x, q.x) and np.array_equal(p.y, q.y)  # seeded
    assert not np.array_equal(p.x, wl.single_pair(1).x)


def test_colour_transfer_recipe():
    p = wl.color_transfer(seed=3, n=20000)
    for v in (p.x, p.y):
        assert v.shape == (20000, 3) and v.dtype == np.float32
        assert v.min() >= 0.0 and v.max() < 1.0  # clipped to [0, 1)
    assert np.all(p.a == 1.0) and np.all(p.b == 1.0)
    # eight shared centres: every point lies within a few sigma of one of
    # them, measured on the points that were not clipped
    rng = np.random.default_rng(3)
    centres = rng.random((8, 3))
    for v in (p.x, p.y):
        inner = v[np.all((v > 0.0) & (v < np.float32(1.0) - 1e-6), axis=1)].astype(np.float64)
        dist = np.sqrt(((inner[:, None, :] - centres[None]) ** 2).sum(-1)).min(1)
        assert np.quantile(dist, 0.99) < 5 * 0.08 * np.sqrt(3)


def test_gmm_recipe():
    p = wl.gmm_pair(seed=1, n=4096, d=64)
    assert p.x.shape == (4096, 64) and p.x.dtype == np.float32
    assert np.all(p.a > 0) and np.all(p.b > 0)
    # Dirichlet(0.5) as normalised Gamma(0.5) draws: mean 0.5, variance 0.5
    assert abs(p.a.mean() - 0.5) < 0.05 and abs(p.a.var() - 0.5) < 0.1
    # both clouds use the same 256 means (fixed mixture seed): the nearest
    # mean of a point is within a few standard deviations (0.5 per axis)
    means = np.random.default_rng(12345).normal(0.0, 2.0, (256, 64))
    v = p.y[:512].astype(np.float64)
    d2 = ((v[:, None, :] - means[None]) ** 2).sum(-1).min(1)
    assert np.all(d2 < 64 * 0.25 * 2.0)


def test_document_recipe():
    b = wl.doc_knn(num_docs=300, seed=2, vocab_size=5000, d=32)
    lengths = np.diff(b.x_off)
    assert b.num_pairs == 300 and lengths.min() >= 20 and lengths.max() <= 500
    assert 45 <= np.median(lengths) <= 75  # LogNormal(ln 60, 0.6), clipped
    norms = np.linalg.norm(b.x.astype(np.float64), axis=1)
    assert np.allclose(norms, 1.0, atol=1e-5)  # L2-normalised word vectors
    assert np.all(b.a > 0) and np.all(b.a <= 1.0)  # rank^-1.1 weights
    # every pair holds the same query document as consumers
    q = b.pair(0)
    for k in (1, 150, 299):
        assert np.array_equal(b.pair(k).y, q.y) and np.array_equal(b.pair(k).b, q.b)


def test_retrieval_recipe():
    b = wl.retrieval(num_pairs=40, seed=4)
    m, n = np.diff(b.x_off), np.diff(b.y_off)
    assert m.min() >= 256 and m.max() <= 2048 and n.min() >= 256 and n.max() <= 2048
    assert b.x.shape[1] == 128 and b.x.min() >= 0.0  # |N(0,1)|, nonnegative
    assert np.allclose(np.linalg.norm(b.x.astype(np.float64), axis=1), 512.0, rtol=1e-5)
    assert np.all(b.a > 0) and abs(b.a.mean() - 1.0) < 0.05  # Exp(1) draws


@pytest.mark.parametrize("weights", ["uniform", "dirichlet"])
def test_batch_pack_round_trip(weights):
    pairs = [wl.uniform_pair(m, n, 3, 10 + m, weights) for m, n in ((5, 7), (1, 1), (40, 3))]
    b = wl.Batch.pack(pairs)
    assert b.num_pairs == 3 and b.x_off.tolist() == [0, 5, 6, 46] and b.y_off.tolist() == [0, 7, 8, 11]
    for k, p in enumerate(pairs):
        q = b.pair(k)
        assert np.array_equal(q.x, p.x) and np.array_equal(q.a, p.a)
        assert np.array_equal(q.y, p.y) and np.array_equal(q.b, p.b)
