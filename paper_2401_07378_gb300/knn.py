"""EMD-kNN: classification and retrieval of histograms under NNS-EMD, the
workload of the paper's experiments (Sec. IV-B documents and images,
Sec. IV-C retrieval).

A query is compared with every histogram of a collection in one call of
nnsemd_solve_one_to_many (collection = suppliers, query = consumers, the
query stored once); the distances come back to the host, where the k
smallest (ties by collection index) vote on the label.
"""
from __future__ import annotations

import numpy as np


def nearest(dist: np.ndarray, k: int) -> np.ndarray:
    """Indices of the k smallest distances, ascending, ties by index."""
    dist = np.asarray(dist)
    order = np.lexsort((np.arange(dist.shape[0]), dist))
    return order[:k]


def vote(dist: np.ndarray, labels: np.ndarray, k: int) -> int:
    """Majority label among the k nearest; a tie between labels goes to the
    label whose tied neighbours have the smaller summed distance, then to the
    smaller label."""
    nn = nearest(dist, k)
    best = None
    for lab in np.unique(labels[nn]):
        members = nn[labels[nn] == lab]
        key = (-len(members), float(np.sum(dist[members])), int(lab))
        if best is None or key < best[0]:
            best = (key, int(lab))
    return best[1]


class EMDKNN:
    """A device-resident collection of histograms with labels.

    x [N_points, d] float32, a [N_points] float64 (device tensors or numpy),
    x_off (host, P+1) delimit the P histograms; labels [P] (host)."""

    def __init__(self, ctx, x, a, x_off, labels, metric: str = "l2", precision: str = "fp32",
                 protocol: str = "greedy", seed: int = 0):
        import torch
        self.ctx = ctx
        self.x = torch.as_tensor(x, dtype=torch.float32).cuda().contiguous()
        self.a = torch.as_tensor(a, dtype=torch.float64).cuda().contiguous()
        self.x_off = np.ascontiguousarray(x_off, np.int64)
        self.labels = np.asarray(labels)
        self.metric, self.precision, self.protocol, self.seed = metric, precision, protocol, seed

    def distances(self, y, b) -> np.ndarray:
        """NNS-EMD from the query (y [n, d], b [n]) to every histogram."""
        import torch
        y = torch.as_tensor(y, dtype=torch.float32).cuda().contiguous()
        b = torch.as_tensor(b, dtype=torch.float64).cuda().contiguous()
        costs, _ = self.ctx.solve_one_to_many(self.x, self.a, self.x_off, y, b, metric=self.metric,
                                              precision=self.precision, stats=False, protocol=self.protocol,
                                              seed=self.seed)
        return costs.cpu().numpy()

    def classify(self, y, b, k: int = 3) -> int:
        return vote(self.distances(y, b), self.labels, k)

    def retrieve(self, y, b, top: int = 10) -> np.ndarray:
        return nearest(self.distances(y, b), top)
