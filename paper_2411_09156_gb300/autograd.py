"""torch.autograd wrapper: forward = ges_preprocess + ges_bin + ges_render_fwd,
backward = ges_render_bwd (front-to-back replay from t_final and last)."""
from __future__ import annotations

import torch

from .api import Rasterizer


class GESRasterize(torch.autograd.Function):
    """Differentiable GES rasterization of one scene into the rasterizer's views.

    Inputs: pos_op [N,4], lscale_beta [N,4], quat [N,4], color ([N,3] or [N,K,3]),
    all float32 CUDA tensors, and a Rasterizer holding the views and buffers.
    Returns (color [3P], depth [P], alpha [P], normal [3P]) concatenated over views
    (colour and normal planar per view). The returned tensors are copies, so the
    rasterizer's buffers can be reused by the next call.
    """

    @staticmethod
    def forward(ctx, pos_op, lscale_beta, quat, color, rast: Rasterizer):
        out = rast.forward(pos_op, lscale_beta, quat, color)
        ctx.rast = rast
        ctx.save_for_backward(pos_op, lscale_beta, quat, color)
        return out["color"].clone(), out["depth"].clone(), out["alpha"].clone(), out["normal"].clone()

    @staticmethod
    def backward(ctx, g_color, g_depth, g_alpha, g_normal):
        pos_op, lscale_beta, quat, color = ctx.saved_tensors
        rast = ctx.rast
        cont = lambda g: None if g is None else g.contiguous()
        grads = rast.backward(pos_op, lscale_beta, quat, color, cont(g_color), cont(g_depth), cont(g_alpha),
                              cont(g_normal))
        # the colour gradient is float32; autograd wants the input's element type
        return grads["g_pos_op"], grads["g_lscale_beta"], grads["g_quat"], grads["g_color"].to(color.dtype), None


def rasterize(pos_op, lscale_beta, quat, color, rast: Rasterizer):
    return GESRasterize.apply(pos_op, lscale_beta, quat, color, rast)
