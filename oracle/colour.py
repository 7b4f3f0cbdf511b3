"""TEST INFRASTRUCTURE -- CPU oracle of the colour-transfer application
(Sec. IV-D): k-means colour quantisation of both images, NNS-EMD between
the palettes (reference palette = suppliers, source palette = consumers),
and the recolouring of the source by the plan's barycentric map.  Only the
tests may import this module.

Definitions (the paper gives the pipeline, not these details):
  k-means   initial centroids: the points at indices floor((2c + 1) N / 2k);
            assignment: nearest centroid by the FP32 squared-distance key of
            the NNS operation, lowest index on ties; update: centroid =
            float32(exact sum / count) per coordinate (the sum correctly
            rounded, so independent of the order of the points); a centroid
            with no point keeps its value; weights = point counts.
  map       y'_j = float32(S_j / W_j), S_j = exact sum over the flows into
            consumer j of f * x_i (each product an FP64 multiply), W_j =
            exact sum of those f; a consumer with no flow keeps its colour.
  recolour  every source pixel takes the mapped colour of its palette entry.
"""
from __future__ import annotations

import ctypes
import math

import numpy as np

from . import _load, solve


def assign(pts: np.ndarray, cent: np.ndarray) -> np.ndarray:
    lib = _load()
    f = lib.oracle_assign
    f.argtypes = [ctypes.c_void_p, ctypes.c_int64, ctypes.c_void_p, ctypes.c_int64, ctypes.c_int32, ctypes.c_void_p]
    f.restype = None
    pts = np.ascontiguousarray(pts, np.float32)
    cent = np.ascontiguousarray(cent, np.float32)
    out = np.empty(pts.shape[0], np.int32)
    f(pts.ctypes.data, pts.shape[0], cent.ctypes.data, cent.shape[0], pts.shape[1], out.ctypes.data)
    return out


def kmeans(pts: np.ndarray, k: int, iters: int):
    """Returns (centroids float32 [k, d], assignment int32 [N], counts int64 [k])."""
    pts = np.ascontiguousarray(pts, np.float32)
    N, d = pts.shape
    idx = ((2 * np.arange(k, dtype=np.int64) + 1) * N) // (2 * k)
    cent = pts[idx].copy()
    lab = assign(pts, cent)
    for _ in range(iters):
        for c in range(k):
            members = pts[lab == c].astype(np.float64)
            if members.shape[0] == 0:
                continue
            for t in range(d):
                cent[c, t] = np.float32(math.fsum(members[:, t].tolist()) / members.shape[0])
        lab = assign(pts, cent)
    counts = np.bincount(lab, minlength=k).astype(np.int64)
    return cent, lab, counts


def barycentric(plan_i, plan_j, plan_f, x: np.ndarray, y: np.ndarray) -> np.ndarray:
    x = np.asarray(x, np.float32)
    out = np.asarray(y, np.float32).copy()
    for j in np.unique(plan_j):
        sel = plan_j == j
        f = plan_f[sel]
        xi = x[plan_i[sel]].astype(np.float64)
        w = math.fsum(f.tolist())
        for t in range(x.shape[1]):
            out[j, t] = np.float32(math.fsum((f * xi[:, t]).tolist()) / w)
    return out


def transfer(src: np.ndarray, ref: np.ndarray, k: int, iters: int, metric: str = "sql2"):
    """The whole application on the CPU: returns (recoloured source pixels,
    source palette, reference palette, the solve's result, source labels)."""
    cs, ls, ns = kmeans(src, k, iters)
    cr, lr, nr = kmeans(ref, k, iters)
    used_r = nr > 0
    used_s = ns > 0
    r = solve(cr[used_r], nr[used_r].astype(np.float64), cs[used_s], ns[used_s].astype(np.float64), metric)
    mapped_used = barycentric(r.plan_i, r.plan_j, r.plan_f, cr[used_r], cs[used_s])
    mapped = cs.copy()
    mapped[used_s] = mapped_used
    return mapped[ls], cs, cr, r, ls
