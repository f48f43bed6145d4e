"""torch.autograd binding of the rasterizer (differentiation pattern).

`rasterize(params, n, deg, cams, ctx)` returns the batch image buffer
([view][3][H][W] concatenated, FP32) as a differentiable function of the
[P, stride] parameter tensor.  The forward runs gs_project, gs_bin_sort and
gs_raster_fwd; the backward runs gs_raster_bwd, which re-walks each tile's
sorted list from every pixel's last contributor and recomputes alpha per
pair, so only T_final and the last-contributor index are kept per pixel
(no per-pixel contributor lists).

The context keeps the sorted state of the last forward, so each in-flight
forward needs its own context; `rasterize` checks that the backward runs
against the forward that produced it and raises otherwise.
"""
from __future__ import annotations

import torch

from . import gs


class _Rasterize(torch.autograd.Function):
    @staticmethod
    def forward(fctx, params, n, deg, cams, gctx, token):
        gctx.gs_project(params, n, deg, cams)
        gctx.gs_bin_sort()
        _, total = gs.image_offsets(cams)
        img = torch.empty(total, device=params.device, dtype=torch.float32)
        gctx.gs_raster_fwd(img)
        fctx.save_for_backward(params)
        fctx.n, fctx.deg, fctx.gctx, fctx.token = n, deg, gctx, token
        gctx._autograd_token = token
        return img

    @staticmethod
    def backward(fctx, dimg):
        (params,) = fctx.saved_tensors
        gctx = fctx.gctx
        if getattr(gctx, "_autograd_token", None) is not fctx.token:
            raise RuntimeError("the rasterizer context was reused by another forward before this backward; "
                               "use one context per in-flight forward")
        grads = torch.empty_like(params)
        gctx.gs_raster_bwd(params, fctx.n, fctx.deg, dimg.contiguous(), grads)
        return grads, None, None, None, None, None


def rasterize(params: torch.Tensor, n: int, deg: int, cams, ctx: gs.Context) -> torch.Tensor:
    """Differentiable batch render of `cams` (list of camera dicts)."""
    return _Rasterize.apply(params, n, deg, cams, ctx, object())


class Adam:
    """Per-group Adam over the plane layout, through gs_adam."""

    DEFAULTS = dict(lr_mean=1.6e-4, lr_scale=5e-3, lr_quat=1e-3, lr_opacity=0.05, lr_sh_dc=2.5e-3,
                    lr_sh_rest=2.5e-3 / 20, beta1=0.9, beta2=0.999, eps=1e-15)

    def __init__(self, params: torch.Tensor, n: int, deg: int, ctx: gs.Context, **hp):
        self.p, self.n, self.deg, self.ctx = params, n, deg, ctx
        self.hp = dict(self.DEFAULTS, **hp)
        self.m = torch.zeros_like(params)
        self.v = torch.zeros_like(params)
        self.t = 0

    def step(self, grad: torch.Tensor):
        self.t += 1
        self.ctx.gs_adam(self.p, grad, self.m, self.v, self.n, self.deg, self.hp, self.t)
