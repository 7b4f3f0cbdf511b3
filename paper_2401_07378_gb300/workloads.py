"""Seeded synthetic inputs shaped like the NNS-EMD paper's workloads.

This module holds no NNS-EMD arithmetic: it only draws point sets and raw
weights.  Both the CUDA path (through the tests and the benchmark) and the
CPU oracle are fed from here, so the two sides always see the same inputs.

The paper's datasets (MNIST, CIFAR-10, DOTmark, 20news, Amazon, NUS-WIDE,
Paris-6k and the seasonal colour-transfer set) are not available; each
generator below stands in for one of them with the shape, size and value
distribution the paper describes (Sec. IV-A "Histogram Initialization",
Table "Datasets description"):

* ``single_pair``       -- a spatial-location histogram pair (pixels as bins).
* ``color_transfer``    -- colour-intensity histograms of two RGB images
                           (Sec. IV-D), 8 colour clusters.
* ``doc_knn``           -- word-embedding histograms of documents
                           (Sec. IV-B, document classification).
* ``retrieval``         -- signatures of image descriptors (Sec. IV-C).
* ``gmm``               -- large Gaussian-mixture clouds in d=64.

Coordinates are float32 (row-major ``[points, d]``); weights are float64 and
not normalised (the solver normalises them, Sec. II-A).
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np

_ONE_MINUS = np.float32(np.nextafter(np.float32(1.0), np.float32(0.0)))


@dataclass
class Pair:
    """One EMD problem: suppliers ``x``/``a`` and consumers ``y``/``b``."""

    x: np.ndarray  # float32 [m, d]  suppliers S
    a: np.ndarray  # float64 [m]
    y: np.ndarray  # float32 [n, d]  consumers C
    b: np.ndarray  # float64 [n]

    @property
    def m(self) -> int:
        return int(self.x.shape[0])

    @property
    def n(self) -> int:
        return int(self.y.shape[0])

    @property
    def d(self) -> int:
        return int(self.x.shape[1])


@dataclass
class Batch:
    """Many EMD problems packed back to back (CSR-style offsets)."""

    x: np.ndarray      # float32 [sum m, d]
    a: np.ndarray      # float64 [sum m]
    x_off: np.ndarray  # int64 [P+1]
    y: np.ndarray      # float32 [sum n, d]
    b: np.ndarray      # float64 [sum n]
    y_off: np.ndarray  # int64 [P+1]

    @property
    def num_pairs(self) -> int:
        return int(self.x_off.shape[0] - 1)

    @property
    def d(self) -> int:
        return int(self.x.shape[1])

    def pair(self, p: int) -> Pair:
        xs, xe = int(self.x_off[p]), int(self.x_off[p + 1])
        ys, ye = int(self.y_off[p]), int(self.y_off[p + 1])
        return Pair(self.x[xs:xe], self.a[xs:xe], self.y[ys:ye], self.b[ys:ye])

    @staticmethod
    def pack(pairs: list[Pair]) -> "Batch":
        d = pairs[0].d
        x_off = np.zeros(len(pairs) + 1, np.int64)
        y_off = np.zeros(len(pairs) + 1, np.int64)
        x_off[1:] = np.cumsum([p.m for p in pairs])
        y_off[1:] = np.cumsum([p.n for p in pairs])
        x = np.ascontiguousarray(np.concatenate([p.x for p in pairs]).reshape(-1, d), np.float32)
        y = np.ascontiguousarray(np.concatenate([p.y for p in pairs]).reshape(-1, d), np.float32)
        a = np.ascontiguousarray(np.concatenate([p.a for p in pairs]), np.float64)
        b = np.ascontiguousarray(np.concatenate([p.b for p in pairs]), np.float64)
        return Batch(x, a, x_off, y, b, y_off)


def _clip01(v: np.ndarray) -> np.ndarray:
    return np.clip(v.astype(np.float32), np.float32(0.0), _ONE_MINUS)


def uniform_pair(m: int, n: int, d: int, seed: int, weights: str = "uniform") -> Pair:
    """Points iid Uniform[0,1)^d; weights uniform (1 each) or Dirichlet(1)."""
    rng = np.random.default_rng(seed)
    x = rng.random((m, d), dtype=np.float32)
    y = rng.random((n, d), dtype=np.float32)
    if weights == "uniform":
        a = np.ones(m, np.float64)
        b = np.ones(n, np.float64)
    elif weights == "dirichlet":
        a = rng.exponential(1.0, m)
        b = rng.exponential(1.0, n)
    else:
        raise ValueError(weights)
    return Pair(x, a, y, b)


def single_pair(seed: int = 0, n: int = 256, d: int = 2) -> Pair:
    """Spatial-location histogram pair: n=m=256 points in d=2, Uniform[0,1),
    uniform weights (the paper's grayscale-pixel formulation, Sec. II-A)."""
    return uniform_pair(n, n, d, seed)


def color_transfer(seed: int = 0, n: int = 65536, clusters: int = 8, sigma: float = 0.08) -> Pair:
    """Colour-intensity histograms of two RGB images (Sec. IV-D): 65,536
    points each in d=3.  Cluster centres ~ Uniform[0,1)^3 (drawn first, shared
    by both images), points = centre + N(0, sigma^2 I) clipped to [0,1),
    uniform weights."""
    rng = np.random.default_rng(seed)
    centres = rng.random((clusters, 3))
    pts = []
    for _ in range(2):
        lab = rng.integers(0, clusters, n)
        p = centres[lab] + rng.normal(0.0, sigma, (n, 3))
        pts.append(_clip01(p))
    return Pair(pts[0], np.ones(n), pts[1], np.ones(n))


def gmm_pair(seed: int = 0, n: int = 262144, d: int = 64, components: int = 256,
             mixture_seed: int = 12345, alpha: float = 0.5) -> Pair:
    """Gaussian-mixture clouds: means ~ N(0, 4I) (fixed mixture seed), points
    ~ N(mu, 0.25 I), Dirichlet(alpha) weights (as normalised Gamma draws)."""
    mrng = np.random.default_rng(mixture_seed)
    means = mrng.normal(0.0, 2.0, (components, d))
    rng = np.random.default_rng(seed)
    out = []
    for _ in range(2):
        lab = rng.integers(0, components, n)
        p = means[lab] + rng.normal(0.0, 0.5, (n, d))
        w = rng.gamma(alpha, 1.0, n)
        out.append((p.astype(np.float32), w))
    return Pair(out[0][0], out[0][1], out[1][0], out[1][1])


# --------------------------------------------------------------------------
# document kNN (Sec. IV-B): 1 query document against many documents
# --------------------------------------------------------------------------

def vocabulary(size: int = 50000, d: int = 300, seed: int = 0) -> np.ndarray:
    """Word vectors iid N(0,1) then L2-normalised (float32)."""
    rng = np.random.default_rng(seed)
    v = rng.standard_normal((size, d))
    v /= np.linalg.norm(v, axis=1, keepdims=True)
    return v.astype(np.float32)


def _zipf_probs(size: int, s: float) -> np.ndarray:
    p = np.arange(1, size + 1, dtype=np.float64) ** (-s)
    return p / p.sum()


def _document(rng: np.random.Generator, vocab: np.ndarray, probs: np.ndarray,
              median: float, sigma: float, lo: int, hi: int, s: float):
    length = int(np.clip(np.round(rng.lognormal(np.log(median), sigma)), lo, hi))
    ids = rng.choice(vocab.shape[0], size=length, replace=False, p=probs)
    w = (ids.astype(np.float64) + 1.0) ** (-s)  # term weight ~ vocab rank^-s
    return vocab[ids], w


def doc_knn(num_docs: int = 4096, seed: int = 0, vocab_size: int = 50000, d: int = 300,
            median: float = 60.0, sigma: float = 0.6, lo: int = 20, hi: int = 500,
            s: float = 1.1, vocab_seed: int = 0) -> Batch:
    """One query document (consumer) against ``num_docs`` documents
    (suppliers).  Document lengths are LogNormal(ln median, sigma) clipped to
    [lo, hi]; words are distinct ids drawn with probability ~ rank^-s; a
    word's weight is ~ rank^-s (a Zipf term frequency)."""
    vocab = vocabulary(vocab_size, d, vocab_seed)
    probs = _zipf_probs(vocab_size, s)
    rng = np.random.default_rng(seed)
    qy, qb = _document(rng, vocab, probs, median, sigma, lo, hi, s)
    pairs = []
    for _ in range(num_docs):
        dx, da = _document(rng, vocab, probs, median, sigma, lo, hi, s)
        pairs.append(Pair(dx, da, qy, qb))
    return Batch.pack(pairs)


@dataclass
class LabelledDocs:
    """A labelled collection for EMD-kNN: documents packed as suppliers
    (x, a, x_off) with one class label each, and held-out queries of known
    class."""

    x: np.ndarray
    a: np.ndarray
    x_off: np.ndarray
    labels: np.ndarray
    queries: list          # [(y [n, d] float32, b [n] float64)]
    query_labels: np.ndarray


def labelled_documents(classes: int = 3, docs_per_class: int = 20, queries_per_class: int = 2, seed: int = 0,
                       vocab_size: int = 2000, d: int = 32, topic_words: int = 150, on_topic: float = 0.8,
                       median: float = 40.0, sigma: float = 0.5, lo: int = 10, hi: int = 120,
                       s: float = 1.1) -> LabelledDocs:
    """Synthetic labelled documents (stand-in for a labelled corpus such as
    20news, Sec. IV-B): each class owns a topic, the ``topic_words`` words
    whose vectors point most along a random class direction (so a topic is a
    region of the word-vector space); a document of the class draws a share
    ``on_topic`` of its distinct words from its topic, Zipf over the topic's
    ranking, weighted by that rank's Zipf term frequency, and the rest from
    the whole vocabulary, Zipf over the vocabulary, weighted likewise."""
    vocab = vocabulary(vocab_size, d, seed + 1)
    rng = np.random.default_rng(seed)
    topics = []
    for _ in range(classes):
        u = rng.standard_normal(d)
        topics.append(np.argsort(-(vocab.astype(np.float64) @ u), kind="stable")[:topic_words])
    p_all = _zipf_probs(vocab_size, s)
    p_top = _zipf_probs(topic_words, s)

    def doc(c: int):
        length = int(np.clip(np.round(rng.lognormal(np.log(median), sigma)), lo, hi))
        k_top = min(topic_words, int(round(on_topic * length)))
        ranks = rng.choice(topic_words, size=k_top, replace=False, p=p_top)
        weight = {int(topics[c][r]): (r + 1.0) ** (-s) for r in ranks}
        while len(weight) < length:
            i = int(rng.choice(vocab_size, p=p_all))
            weight.setdefault(i, (i + 1.0) ** (-s))
        ids = np.array(sorted(weight))
        return vocab[ids], np.array([weight[i] for i in ids.tolist()])

    xs, ws, labels = [], [], []
    for c in range(classes):
        for _ in range(docs_per_class):
            x, w = doc(c)
            xs.append(x)
            ws.append(w)
            labels.append(c)
    x_off = np.concatenate([[0], np.cumsum([len(w) for w in ws])]).astype(np.int64)
    queries, qlabels = [], []
    for c in range(classes):
        for _ in range(queries_per_class):
            queries.append(doc(c))
            qlabels.append(c)
    return LabelledDocs(np.concatenate(xs).astype(np.float32), np.concatenate(ws), x_off, np.array(labels),
                        queries, np.array(qlabels))


def retrieval(num_pairs: int = 10000, seed: int = 0, d: int = 128, lo: int = 256, hi: int = 2048) -> Batch:
    """Signature pairs of SIFT-like descriptors: m, n ~ Uniform{lo..hi}
    independently; descriptors |N(0,1)| then L2-normalised and scaled by 512;
    weights Dirichlet(1) (normalised Exp(1) draws).  All sizes are drawn
    first, then all descriptors (vectorised: the full 10,000-pair batch holds
    about 23 million descriptors)."""
    rng = np.random.default_rng(seed)
    m = rng.integers(lo, hi + 1, num_pairs)
    n = rng.integers(lo, hi + 1, num_pairs)
    x_off = np.concatenate([[0], np.cumsum(m)]).astype(np.int64)
    y_off = np.concatenate([[0], np.cumsum(n)]).astype(np.int64)

    def descriptors(count: int) -> np.ndarray:
        out = np.empty((count, d), np.float32)
        step = 1 << 20
        for s in range(0, count, step):
            v = np.abs(rng.standard_normal((min(step, count - s), d), dtype=np.float32))
            v /= np.linalg.norm(v, axis=1, keepdims=True)
            v *= np.float32(512.0)
            out[s:s + v.shape[0]] = v
        return out

    x = descriptors(int(x_off[-1]))
    y = descriptors(int(y_off[-1]))
    a = rng.exponential(1.0, int(x_off[-1]))
    b = rng.exponential(1.0, int(y_off[-1]))
    return Batch(x, a, x_off, y, b, y_off)


def random_batch(num_pairs: int, seed: int, d: int, lo: int, hi: int, weights: str = "dirichlet") -> Batch:
    """Small uneven batches of uniform point sets (test cases)."""
    rng = np.random.default_rng(seed)
    pairs = []
    for p in range(num_pairs):
        m = int(rng.integers(lo, hi + 1))
        n = int(rng.integers(lo, hi + 1))
        pairs.append(uniform_pair(m, n, d, seed * 100003 + p, weights))
    return Batch.pack(pairs)
