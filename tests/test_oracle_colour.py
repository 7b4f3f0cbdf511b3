"""Pins of the colour-transfer oracle (Sec. IV-D pipeline): k-means against
the exact cluster means of separated clusters, the identity transfer, the
plan's marginals carried into the recoloured palette, and single flows."""
import math

import numpy as np
import pytest

from oracle import colour


def clusters(seed, k=4, per=200, sigma=1e-3):
    rng = np.random.default_rng(seed)
    centres = np.array([[0.1, 0.1, 0.1], [0.9, 0.1, 0.5], [0.2, 0.8, 0.9], [0.7, 0.7, 0.2]])[:k]
    pts = np.concatenate([c + sigma * rng.standard_normal((per, 3)) for c in centres]).astype(np.float32)
    return pts, np.repeat(np.arange(k), per)


def test_kmeans_recovers_separated_cluster_means():
    pts, truth = clusters(0)
    cent, lab, counts = colour.kmeans(pts, 4, 5)
    # every true cluster is one k-means cluster, and its centroid is the
    # correctly rounded mean of its points
    for c in range(4):
        members = lab[truth == c]
        assert np.all(members == members[0])
        got = cent[members[0]]
        want = [np.float32(math.fsum(pts[truth == c, t].astype(np.float64).tolist()) / 200) for t in range(3)]
        assert got.tolist() == want
    assert sorted(counts.tolist()) == [200] * 4


def test_identity_transfer_keeps_the_quantised_colours():
    rng = np.random.default_rng(1)
    img = rng.random((3000, 3)).astype(np.float32)
    out, cs, cr, r, ls = colour.transfer(img, img, 24, 3)
    assert np.array_equal(out, cs[ls])
    assert r.cost == 0.0


def test_recoloured_palette_keeps_the_reference_mean():
    rng = np.random.default_rng(2)
    src = rng.random((4000, 3)).astype(np.float32)
    ref = (0.5 * rng.random((3000, 3)) + 0.3).astype(np.float32)
    out, cs, cr, r, ls = colour.transfer(src, ref, 16, 3)
    # sum_j c_j y'_j = sum_ij F_ij x_i = sum_i s_i x_i (the plan's marginals)
    used_r = np.bincount(colour.assign(ref, cr), minlength=16) > 0
    mapped_mean = out.astype(np.float64).mean(axis=0)
    ref_mean = (r.s[:, None] * cr[used_r].astype(np.float64)).sum(axis=0)
    np.testing.assert_allclose(mapped_mean, ref_mean, rtol=0, atol=1e-6)


def test_single_flows_copy_the_supplier_colour():
    x = np.array([[0.1, 0.2, 0.3], [0.9, 0.8, 0.7]], np.float32)
    y = np.zeros((3, 3), np.float32)
    out = colour.barycentric(np.array([1, 0]), np.array([0, 2]), np.array([0.25, 0.5]), x, y)
    assert out[0].tolist() == x[1].tolist() and out[2].tolist() == x[0].tolist()
    assert out[1].tolist() == [0.0, 0.0, 0.0]  # no flow: unchanged
