"""torch.autograd.Function over the C ABI: forward = nerfxl_render_fwd,
backward = nerfxl_render_bwd (hand-written adjoint kernels; per-sample
activations recomputed from the saved chunk partials)."""
from __future__ import annotations

import torch

from . import api


class RenderFunction(torch.autograd.Function):
    @staticmethod
    def forward(ctx, tables, mlp, rays_o, rays_d, field: api.PartitionedField, samp: api.Sampling):
        if tables.data_ptr() != field.tables.data_ptr() or mlp.data_ptr() != field.mlp.data_ptr():
            raise ValueError("tables/mlp must be the field's own parameter tensors")
        ws = api.alloc_workspace(field, samp, rays_o.shape[0], for_backward=True)
        out = api.render_fwd(field, samp, rays_o, rays_d, workspace=ws)
        ctx.field, ctx.samp = field, samp
        ctx.save_for_backward(rays_o, rays_d, ws)
        return out["rgb"], out["depth"], out["opacity"], out["dist"]

    @staticmethod
    def backward(ctx, g_rgb, g_depth, g_opacity, g_dist):
        rays_o, rays_d, ws = ctx.saved_tensors
        gt, gm = api.render_bwd(ctx.field, ctx.samp, rays_o, rays_d, ws, g_rgb, g_depth, g_opacity, g_dist)
        return gt, gm, None, None, None, None


def render(field: api.PartitionedField, samp: api.Sampling, rays_o, rays_d):
    """Differentiable render w.r.t. field.tables and field.mlp (FP32)."""
    o, d = api._rays(rays_o, rays_d, field.device)
    return RenderFunction.apply(field.tables, field.mlp, o, d, field, samp)
