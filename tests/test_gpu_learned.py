"""The learned candidate proposal on the GPU: its gradient against the CPU
oracle network, its training, and solves that use it -- which must equal the
CPU oracle bit for bit (certified choices equal the full scan's; the rest
fall back to it) -- plus what the trained network gains over an untrained
one."""
import os
import tempfile

import numpy as np
import pytest

import oracle
from oracle import mlp
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
def small_prop(ctx):
    """A trained proposal with 256 cells (quick to build)."""
    from paper_2401_07378_gb300 import proposal_training
    prop, info = proposal_training.build_gmm_proposal(ctx, cells=256, hidden=64, runs=40, n_per_run=2048,
                                                       fit_runs=2, fit_n=16384, epochs=6, batch=2048, lr=3e-3)
    return prop, info


def test_gradient_matches_cpu_oracle(ctx):
    from paper_2401_07378_gb300 import nnsemd
    d, h, k, n = 16, 32, 64, 96
    prop = nnsemd.Proposal(ctx, d, cells=k, hidden=h, seed=3)
    rng = np.random.default_rng(4)
    theta = rng.normal(0, 0.3, prop.nparams).astype(np.float32)
    prop.set_params(theta)
    y = rng.normal(0, 1, (n, d)).astype(np.float32)
    labels = rng.integers(0, k, n).astype(np.int32)
    loss, grad = prop.loss_grad(torch.from_numpy(y).cuda(), torch.from_numpy(labels).cuda())
    ref_loss, ref_grad = mlp.loss_and_grad(theta.astype(np.float64), y.astype(np.float64), labels, d, h, k)
    assert loss == pytest.approx(ref_loss, rel=1e-5)
    g = grad.cpu().numpy().astype(np.float64)
    np.testing.assert_allclose(g, ref_grad, rtol=2e-3, atol=2e-6)
    prop.close()


def test_training_lowers_the_loss(ctx, small_prop):
    prop, info = small_prop
    assert np.isfinite(info["final_loss"])
    assert info["final_loss"] < np.log(256) * 0.7, info


@pytest.mark.parametrize("metric", ["l2", "sql2"])
def test_learned_solve_equals_oracle(ctx, small_prop, metric):
    prop, _ = small_prop
    p = wl.gmm_pair(seed=0, n=6000, d=64)
    t = lambda v: torch.from_numpy(v).cuda()
    res = ctx.solve(t(p.x), t(p.a), t(p.y), t(p.b), metric=metric, plan=True, proposal=prop)
    ref = oracle.solve_pair(p, metric)
    assert res.cost == ref.cost
    assert res.stats["rounds"] == ref.rounds and res.stats["pair_evals"] == ref.pair_evals
    gi = np.lexsort((res.plan_j.cpu().numpy(), res.plan_i.cpu().numpy()))
    oi = np.lexsort((ref.plan_j, ref.plan_i))
    assert np.array_equal(res.plan_f.cpu().numpy()[gi], ref.plan_f[oi])
    assert res.stats["certified"] > 0


def test_trained_network_beats_untrained(ctx, small_prop):
    """What the trained network gains: more consumer searches certified from
    its own candidates (certified - widened: the second tier, the bound
    list's further cells, is not the network's doing) than the same
    architecture with its initial weights, on the same codebook."""
    from paper_2401_07378_gb300 import nnsemd
    prop, _ = small_prop
    untrained = nnsemd.Proposal(ctx, 64, cells=256, hidden=64, seed=99)
    with tempfile.TemporaryDirectory() as tmp:
        path = os.path.join(tmp, "p.bin")
        prop.save(path)
        loaded = nnsemd.Proposal.load(ctx, path)
    trained = loaded.params()
    assert np.array_equal(trained, prop.params())
    p = wl.gmm_pair(seed=0, n=6000, d=64)
    t = lambda v: torch.from_numpy(v).cuda()
    args = (t(p.x), t(p.a), t(p.y), t(p.b))
    # the loaded copy keeps the trained codebook; swap in the initial weights
    loaded.set_params(untrained.params())
    r_untrained = ctx.solve(*args, metric="l2", proposal=loaded)
    loaded.set_params(trained)
    r_trained = ctx.solve(*args, metric="l2", proposal=loaded)
    assert r_trained.cost == r_untrained.cost  # both exact
    def own(st):
        total = st["certified"] + st["fallbacks"]
        assert 0 <= st["widened"] <= st["certified"]
        return (st["certified"] - st["widened"]) / max(1, total)
    ft, fu = own(r_trained.stats), own(r_untrained.stats)
    assert ft > fu, (ft, fu)
    untrained.close()
    loaded.close()


@pytest.mark.parametrize("precision", ["bf16", "fp16"])
def test_learned_with_reduced_precision_fallback_equals_oracle(ctx, small_prop, precision):
    """Consumers the proposal cannot certify go to the tensor-core scan
    (its own certificate, FP32 rescan of the rest): still the oracle's
    result bit for bit."""
    prop, _ = small_prop
    p = wl.gmm_pair(seed=0, n=6000, d=64)
    t = lambda v: torch.from_numpy(v).cuda()
    res = ctx.solve(t(p.x), t(p.a), t(p.y), t(p.b), metric="l2", precision=precision, plan=True, proposal=prop)
    ref = oracle.solve_pair(p, "l2")
    assert res.cost == ref.cost
    assert res.stats["rounds"] == ref.rounds
    gi = np.lexsort((res.plan_j.cpu().numpy(), res.plan_i.cpu().numpy()))
    oi = np.lexsort((ref.plan_j, ref.plan_i))
    assert np.array_equal(res.plan_f.cpu().numpy()[gi], ref.plan_f[oi])
    assert res.stats["certified"] > 0


def test_learned_host_entry_point(ctx, small_prop):
    prop, _ = small_prop
    p = wl.gmm_pair(seed=2, n=3000, d=64)
    res = ctx.solve_host(p.x, p.a, p.y, p.b, metric="l2", proposal=prop)
    assert res.cost == oracle.solve_pair(p, "l2").cost


@pytest.mark.parametrize("d,precision", [(48, "fp32"), (48, "bf16x3"), (100, "fp32"), (100, "bf16")])
def test_learned_solve_at_other_widths_equals_oracle(ctx, d, precision):
    """The learned path's other branches: at d = 48 the scan runs one warp
    per consumer while the network, the assignment and the cell bounds run
    on the tensor cores; at d = 100 (not a multiple of 16) the network's two
    narrow layers, the assignment and the cell bounds take their FP32 forms.
    Either way the result is the oracle's, bit for bit."""
    from paper_2401_07378_gb300 import proposal_training
    prop, _ = proposal_training.build_gmm_proposal(ctx, d=d, cells=128, hidden=64, runs=12, n_per_run=1024,
                                                    fit_runs=1, fit_n=8192, epochs=3, batch=1024, lr=3e-3)
    p = wl.gmm_pair(seed=3, n=3000, d=d)
    t = lambda v: torch.from_numpy(v).cuda()
    res = ctx.solve(t(p.x), t(p.a), t(p.y), t(p.b), metric="l2", precision=precision, plan=True, proposal=prop)
    ref = oracle.solve_pair(p, "l2")
    assert res.cost == ref.cost
    assert res.stats["rounds"] == ref.rounds
    gi = np.lexsort((res.plan_j.cpu().numpy(), res.plan_i.cpu().numpy()))
    oi = np.lexsort((ref.plan_j, ref.plan_i))
    assert np.array_equal(res.plan_f.cpu().numpy()[gi], ref.plan_f[oi])
    assert res.stats["certified"] > 0
    prop.close()
