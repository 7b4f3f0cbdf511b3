"""TEST INFRASTRUCTURE -- CPU oracle of the learned proposal's network.

Only the tests may import this module.  A plain FP64 numpy restatement of
the MLP d -> h -> h -> K with ReLU and the mean softmax cross-entropy, and
its gradient by backpropagation written out layer by layer, in the
parameter layout of nnsemd_proposal_params:

    W1 [h][d], b1 [h], W2 [h][h], b2 [h], W3 [K][h], b3 [K]

Inputs are standardised as the library does: (y - mean) * scale.
The gradient is pinned against central finite differences in the tests.
"""
from __future__ import annotations

import numpy as np


def unpack(theta: np.ndarray, d: int, h: int, k: int):
    theta = np.asarray(theta, np.float64)
    o = 0
    parts = []
    for shape in ((h, d), (h,), (h, h), (h,), (k, h), (k,)):
        size = int(np.prod(shape))
        parts.append(theta[o:o + size].reshape(shape))
        o += size
    assert o == theta.size
    return parts


def loss_and_grad(theta, X, labels, d: int, h: int, k: int):
    """Mean softmax cross-entropy of the network on rows of X (already
    standardised) with integer labels, and its gradient (same layout)."""
    W1, b1, W2, b2, W3, b3 = unpack(theta, d, h, k)
    X = np.asarray(X, np.float64)
    n = X.shape[0]
    a1 = X @ W1.T + b1
    h1 = np.maximum(a1, 0.0)
    a2 = h1 @ W2.T + b2
    h2 = np.maximum(a2, 0.0)
    z = h2 @ W3.T + b3
    zmax = z.max(axis=1, keepdims=True)
    e = np.exp(z - zmax)
    s = e.sum(axis=1, keepdims=True)
    loss = float(np.mean(np.log(s[:, 0]) + zmax[:, 0] - z[np.arange(n), labels]))
    dz = e / s
    dz[np.arange(n), labels] -= 1.0
    dz /= n
    gW3 = dz.T @ h2
    gb3 = dz.sum(axis=0)
    dh2 = (dz @ W3) * (a2 > 0)
    gW2 = dh2.T @ h1
    gb2 = dh2.sum(axis=0)
    dh1 = (dh2 @ W2) * (a1 > 0)
    gW1 = dh1.T @ X
    gb1 = dh1.sum(axis=0)
    grad = np.concatenate([g.ravel() for g in (gW1, gb1, gW2, gb2, gW3, gb3)])
    return loss, grad


def loss_only(theta, X, labels, d, h, k):
    return loss_and_grad(theta, X, labels, d, h, k)[0]
