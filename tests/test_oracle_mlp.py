"""Pins of the CPU oracle of the proposal network: its backpropagated
gradient against central finite differences of its loss, and its loss
against a closed form (uniform logits give log K)."""
import numpy as np
import pytest

from oracle import mlp


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_gradient_matches_finite_differences(seed):
    rng = np.random.default_rng(seed)
    d, h, k, n = 5, 7, 6, 9
    nparam = h * d + h + h * h + h + k * h + k
    theta = rng.normal(0, 0.7, nparam)
    X = rng.normal(0, 1, (n, d))
    labels = rng.integers(0, k, n)
    loss, grad = mlp.loss_and_grad(theta, X, labels, d, h, k)
    eps = 1e-6
    num = np.empty(nparam)
    for i in range(nparam):
        tp, tm = theta.copy(), theta.copy()
        tp[i] += eps
        tm[i] -= eps
        num[i] = (mlp.loss_only(tp, X, labels, d, h, k) - mlp.loss_only(tm, X, labels, d, h, k)) / (2 * eps)
    np.testing.assert_allclose(grad, num, rtol=1e-5, atol=1e-8)


def test_uniform_logits_give_log_k():
    d, h, k, n = 3, 4, 10, 5
    theta = np.zeros(h * d + h + h * h + h + k * h + k)
    X = np.random.default_rng(3).normal(0, 1, (n, d))
    loss, grad = mlp.loss_and_grad(theta, X, np.arange(n) % k, d, h, k)
    assert loss == pytest.approx(np.log(k), rel=1e-15)
    # with all weights zero only the output bias moves: softmax - onehot
    gb3 = grad[-k:]
    want = np.full(k, 1.0 / k) - np.bincount(np.arange(n) % k, minlength=k) / n
    np.testing.assert_allclose(gb3, want, atol=1e-15)
