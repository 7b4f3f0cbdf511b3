"""Colour transfer with NNS-EMD (Sec. IV-D), on the GPU through the C ABI.

    recoloured = transfer(ctx, source_pixels, reference_pixels, k=256, iters=8)

source / reference: [N, 3] float32 colours in [0, 1] (an image's pixels in
any order).  Both images are quantised to k colours (nnsemd_kmeans), the
NNS-EMD plan moves the reference palette (suppliers, weights = cluster
sizes) onto the source palette (consumers), each source palette colour is
replaced by the barycentre of the reference colours it receives
(nnsemd_barycentric), and the source pixels are recoloured
(nnsemd_recolour).  Palette entries without pixels take no part.
"""
from __future__ import annotations

from dataclasses import dataclass


@dataclass
class TransferResult:
    pixels: object          # [N_src, 3] recoloured source (device)
    source_palette: object  # [k, 3]
    reference_palette: object
    mapped_palette: object  # [k, 3] source palette after the map
    labels: object          # [N_src] source pixel -> palette entry
    cost: float             # NNS-EMD between the palettes
    stats: dict


def transfer(ctx, src, ref, k: int = 256, iters: int = 8, metric: str = "sql2") -> TransferResult:
    import torch
    src = torch.as_tensor(src, dtype=torch.float32).cuda().contiguous()
    ref = torch.as_tensor(ref, dtype=torch.float32).cuda().contiguous()
    cs, ls, ns = ctx.kmeans(src, k, iters)
    cr, lr, nr = ctx.kmeans(ref, k, iters)
    used_s = ns > 0
    used_r = nr > 0
    ys, bs = cs[used_s].contiguous(), ns[used_s].to(torch.float64).contiguous()
    xr, ar = cr[used_r].contiguous(), nr[used_r].to(torch.float64).contiguous()
    res = ctx.solve(xr, ar, ys, bs, metric=metric, plan=True)
    mapped_used = ctx.barycentric(res.plan_i, res.plan_j, res.plan_f, xr, ys)
    mapped = cs.clone()
    mapped[used_s] = mapped_used
    pixels = ctx.recolour(ls, mapped)
    return TransferResult(pixels, cs, cr, mapped, ls, res.cost, res.stats)
