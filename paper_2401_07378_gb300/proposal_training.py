"""Build a learned candidate proposal for the Gaussian-mixture workload.

Everything runs through the C ABI (nnsemd_proposal_*, nnsemd_nearest); this
module only draws the seeded training inputs and moves them to the device.

1. Codebook: k-means of supplier points drawn from training seeds
   (seeds 1..fit_runs of the generator; the evaluation instance is seed 0).
2. Traces: for seeds 1..runs, one plain-method NNS round (nnsemd_nearest,
   round one of Alg. 1) gives each consumer its nearest supplier.
3. Training: minibatch Adam on the cell of that supplier (GPU kernels).
"""
from __future__ import annotations

import time

import numpy as np

from . import workloads


def build_gmm_proposal(ctx, d: int = 64, cells: int = 4096, hidden: int = 256, runs: int = 200,
                       n_per_run: int = 4096, fit_runs: int = 4, fit_n: int = 65536, kmeans_iters: int = 10,
                       epochs: int = 4, batch: int = 4096, lr: float = 2e-3, seed: int = 7):
    import torch

    from .nnsemd import Proposal
    t0 = time.perf_counter()
    prop = Proposal(ctx, d, cells, hidden, seed=seed)
    fit = np.concatenate([workloads.gmm_pair(seed=s, n=fit_n, d=d).x for s in range(1, fit_runs + 1)])
    prop.fit(torch.from_numpy(fit).cuda(), iters=kmeans_iters, seed=seed)
    ys, xs = [], []
    for s in range(1, runs + 1):
        p = workloads.gmm_pair(seed=1000 + s, n=n_per_run, d=d)
        x = torch.from_numpy(p.x).cuda()
        y = torch.from_numpy(p.y).cuda()
        nn = ctx.nearest(x, y, "l2").long()
        ys.append(y)
        xs.append(x[nn])
    y_all = torch.cat(ys).contiguous()
    x_all = torch.cat(xs).contiguous()
    loss = prop.train(y_all, x_all, epochs=epochs, batch=batch, lr=lr, seed=seed)
    torch.cuda.synchronize()
    info = {"train_samples": int(y_all.shape[0]), "final_loss": loss, "seconds": time.perf_counter() - t0,
            "runs": runs, "n_per_run": n_per_run, "cells": cells, "hidden": hidden, "epochs": epochs}
    return prop, info
