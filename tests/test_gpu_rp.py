"""The random protocol (Sec. III-A) on the GPU: every path that orders a
supplier's group (multi-CTA rounds with thread / warp / CTA serving, the
one-CTA tail, the one-launch small solve, the batched kernels, the
reduced-precision NNS) against the CPU oracle, bit for bit."""
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


def dev(v, dt):
    return torch.from_numpy(np.ascontiguousarray(v)).to("cuda", dt)


def gpu(ctx, x, a, y, b, metric, seed, **kw):
    return ctx.solve(dev(x, torch.float32), dev(a, torch.float64), dev(y, torch.float32), dev(b, torch.float64),
                     metric=metric, plan=True, protocol="random", seed=seed, **kw)


def same(res, ref):
    assert res.cost == ref.cost
    assert res.stats["rounds"] == ref.rounds
    gi = np.lexsort((res.plan_j.cpu().numpy(), res.plan_i.cpu().numpy()))
    oi = np.lexsort((ref.plan_j, ref.plan_i))
    assert np.array_equal(res.plan_i.cpu().numpy()[gi], ref.plan_i[oi])
    assert np.array_equal(res.plan_j.cpu().numpy()[gi], ref.plan_j[oi])
    assert np.array_equal(res.plan_f.cpu().numpy()[gi], ref.plan_f[oi])


def test_hand_worked_case_all_seeds(ctx):
    x = np.array([[0, 0], [10, 0]], np.float32)
    y = np.array([[1, 0], [0, 2]], np.float32)
    w = np.array([0.5, 0.5])
    for seed in range(16):
        same(gpu(ctx, x, w, y, w, "l2", seed), oracle.solve(x, w, y, w, "l2", protocol="random", seed=seed))


@pytest.mark.parametrize("d", [2, 3, 16])
@pytest.mark.parametrize("metric", ["l2", "l1"])
def test_random_pairs(ctx, d, metric):
    rng = np.random.default_rng(40 + d)
    for m, n in ((1, 30), (300, 700), (1500, 1100), (2500, 3100)):
        p = wl.uniform_pair(m, n, d, int(rng.integers(1 << 30)), "dirichlet")
        seed = int(rng.integers(1 << 62))
        same(gpu(ctx, p.x, p.a, p.y, p.b, metric, seed), oracle.solve_pair(p, metric, protocol="random", seed=seed))


@pytest.mark.parametrize("ratio", [4, 25, 60])
def test_group_sizes(ctx, ratio):
    n = 6000
    p = wl.uniform_pair(n // ratio, n, 2, 77 + ratio, "dirichlet")
    same(gpu(ctx, p.x, p.a, p.y, p.b, "sql2", 123), oracle.solve_pair(p, "sql2", protocol="random", seed=123))


def test_colour_clusters(ctx):
    p = wl.color_transfer(seed=4, n=20011)
    ref = oracle.solve_pair(p, "sql2", protocol="random", seed=2024)
    same(gpu(ctx, p.x, p.a, p.y, p.b, "sql2", 2024), ref)
    # and the protocol changes the answer here (groups are contested)
    assert ref.cost != oracle.solve_pair(p, "sql2").cost


@pytest.mark.parametrize("precision", ["fp32", "bf16"])
def test_high_d(ctx, precision):
    p = wl.gmm_pair(seed=5, n=5000, d=64)
    same(gpu(ctx, p.x, p.a, p.y, p.b, "l2", 9, precision=precision),
         oracle.solve_pair(p, "l2", protocol="random", seed=9))


@pytest.mark.parametrize("d,precision", [(2, "fp32"), (24, "fp32"), (24, "bf16")])
def test_batched(ctx, d, precision):
    rng = np.random.default_rng(d)
    sizes = [(1, 1), (40, 700), (512, 512), (600, 30), (900, 1100), (37, 12), (200, 300)]
    pairs = [wl.uniform_pair(m, n, d, int(rng.integers(1 << 30)), "dirichlet") for m, n in sizes]
    batch = wl.Batch.pack(pairs)
    costs, stats = ctx.solve_batched(dev(batch.x, torch.float32), dev(batch.a, torch.float64), batch.x_off,
                                     dev(batch.y, torch.float32), dev(batch.b, torch.float64), batch.y_off,
                                     metric="l2", precision=precision, protocol="random", seed=31)
    costs = costs.cpu().numpy()
    for k, pr in enumerate(pairs):
        assert costs[k] == oracle.solve_pair(pr, "l2", protocol="random", seed=31).cost, k
