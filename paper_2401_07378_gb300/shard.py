"""Splitting one batch of EMD pairs over several GPUs (one process per GPU).

The pairs of a batch are independent problems (Sec. III-D, batch
processing), so a batch shards without any exchange on the data path: the
pair list is partitioned by its estimated NNS work, every rank solves its
share with ``nnsemd_solve_batched`` on its own GPU, and the P costs are
gathered to rank 0 in pair order (the only collective).

Work estimate of a pair: m * n, the first round's NNS work; the work of a
whole solve grows with it (Sec. III-C).  The partition is greedy
longest-processing-time (Graham 1969): pairs in decreasing work (ties by
index) each go to the least-loaded rank so far (ties to the lower rank).  Its
largest load is at most (4/3 - 1/(3G)) times the best possible one.  Every
rank computes the same partition from the offsets alone, so no partition is
communicated.

Host logic only: every solve still runs in the CUDA library.
"""
from __future__ import annotations

import heapq
from dataclasses import dataclass

import numpy as np


def pair_work(x_off, y_off=None, n_shared: int | None = None) -> np.ndarray:
    """Estimated work m * n of every pair of a packed batch (int64)."""
    x_off = np.asarray(x_off, np.int64)
    m = np.diff(x_off)
    n = np.diff(np.asarray(y_off, np.int64)) if y_off is not None else np.full_like(m, int(n_shared))
    return m * n


def partition(work, ranks: int) -> list[np.ndarray]:
    """Greedy longest-processing-time split of the pairs over ``ranks``;
    returns, per rank, its pair indices in ascending order."""
    work = np.asarray(work, np.int64)
    if ranks < 1:
        raise ValueError("ranks must be >= 1")
    order = sorted(range(work.size), key=lambda p: (-int(work[p]), p))
    heap = [(0, r) for r in range(ranks)]
    shares: list[list[int]] = [[] for _ in range(ranks)]
    for p in order:
        load, r = heapq.heappop(heap)
        shares[r].append(p)
        heapq.heappush(heap, (load + int(work[p]), r))
    return [np.array(sorted(s), np.int64) for s in shares]


@dataclass
class SubBatch:
    """The packed arrays of the pairs ``ids`` of a batch, in that order."""
    ids: np.ndarray
    x: np.ndarray
    a: np.ndarray
    x_off: np.ndarray
    y: np.ndarray
    b: np.ndarray
    y_off: np.ndarray

    @property
    def num_pairs(self) -> int:
        return int(self.ids.size)


def sub_batch(batch, ids) -> SubBatch:
    """Gather pairs ``ids`` (any order) of a packed batch (``x``, ``a``,
    ``x_off``, ``y``, ``b``, ``y_off``) into packed arrays of their own."""
    ids = np.asarray(ids, np.int64)

    def take(v, off):
        off = np.asarray(off, np.int64)
        lens = off[ids + 1] - off[ids]
        new_off = np.zeros(ids.size + 1, np.int64)
        new_off[1:] = np.cumsum(lens)
        rows = np.concatenate([np.arange(off[p], off[p + 1]) for p in ids]) if ids.size else np.zeros(0, np.int64)
        return np.ascontiguousarray(v[rows]), new_off, rows

    x, x_off, rx = take(batch.x, batch.x_off)
    y, y_off, ry = take(batch.y, batch.y_off)
    return SubBatch(ids, x, np.ascontiguousarray(batch.a[rx]), x_off, y, np.ascontiguousarray(batch.b[ry]), y_off)


def gather_costs(local_costs, ids_per_rank: list[np.ndarray], num_pairs: int, rank: int, device=None):
    """All-gather every rank's costs (a float64 tensor in the order of its
    ids) and return the P costs in pair order (a CPU float64 numpy array, on
    every rank).  One collective: an all-gather of the shares padded to the
    largest one.  With one rank (or no process group) it only reorders."""
    import torch
    import torch.distributed as dist
    ranks = len(ids_per_rank)
    out = np.empty(num_pairs, np.float64)
    if ranks == 1 or not (dist.is_available() and dist.is_initialized()):
        out[ids_per_rank[rank]] = local_costs.detach().cpu().numpy()
        return out
    width = max(int(s.size) for s in ids_per_rank)
    dev = device if device is not None else local_costs.device
    mine = torch.full((width,), float("nan"), dtype=torch.float64, device=dev)
    mine[: local_costs.numel()] = local_costs.to(dev)
    parts = [torch.empty(width, dtype=torch.float64, device=dev) for _ in range(ranks)]
    dist.all_gather(parts, mine)
    for r, ids in enumerate(ids_per_rank):
        out[ids] = parts[r][: ids.size].cpu().numpy()
    return out
