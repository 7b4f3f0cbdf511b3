"""The colour-transfer application (Sec. IV-D) on the GPU against its CPU
oracle: k-means palettes, labels and counts, the NNS-EMD between the
palettes, the barycentric map and the recoloured pixels, all bit for bit."""
import numpy as np
import pytest

from oracle import colour
from paper_2401_07378_gb300 import colour_transfer, workloads as wl

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    from paper_2401_07378_gb300 import nnsemd
    c = nnsemd.Context(0)
    yield c
    c.close()


def test_kmeans_equals_oracle(ctx):
    pts = wl.color_transfer(seed=2, n=12000).x
    cent, lab, cnt = ctx.kmeans(torch.from_numpy(pts).cuda(), 48, 4)
    rc, rl, rn = colour.kmeans(pts, 48, 4)
    assert np.array_equal(cent.cpu().numpy(), rc)
    assert np.array_equal(lab.cpu().numpy(), rl)
    assert np.array_equal(cnt.cpu().numpy(), rn)


@pytest.mark.parametrize("k", [16, 64])
def test_transfer_equals_oracle(ctx, k):
    src = wl.color_transfer(seed=5, n=20000).x
    rng = np.random.default_rng(6)
    ref = np.clip(0.6 * wl.color_transfer(seed=7, n=15000).x + 0.3 * rng.random((15000, 3)), 0, 1).astype(np.float32)
    got = colour_transfer.transfer(ctx, src, ref, k=k, iters=4)
    want_pixels, cs, cr, r, ls = colour.transfer(src, ref, k, 4)
    assert np.array_equal(got.source_palette.cpu().numpy(), cs)
    assert np.array_equal(got.reference_palette.cpu().numpy(), cr)
    assert got.cost == r.cost
    assert np.array_equal(got.pixels.cpu().numpy(), want_pixels)


def test_identity_transfer(ctx):
    img = wl.color_transfer(seed=9, n=8000).x
    got = colour_transfer.transfer(ctx, img, img, k=32, iters=3)
    assert got.cost == 0.0
    assert torch.equal(got.mapped_palette, got.source_palette)
