"""PyTorch autograd over the hand-written adjoint kernels.

``mapping_loss(density, sh, ...)`` is the RGB-D loss of a ray batch
(L = L_p + lambda_d L_g, Sec. 5.2, Eq. 4, 5, 11) as a differentiable function
of the grid values. Its gradient is the analytic adjoint of Eq. 6-10
(``plx_render_backward_grid``). The loss and the gradient come out of the same
pass (the adjoint kernel produces both), so the forward stores the gradient
and the backward only scales it by the incoming gradient. Options naming a
sample cache (``plx.SampleCache.opts``) make the adjoint read back the
forward's compositing samples instead of re-marching the rays; per-sample
transmittance is recomputed either way.
"""
from __future__ import annotations

import torch

from . import plx


class MappingLoss(torch.autograd.Function):
    @staticmethod
    def forward(ctx, density, sh, grid, cams, opts, rgb_target, depth_target, rays):
        grid.upload(density.detach().float(), sh.detach().float().reshape(-1, 27))
        out = plx.render_forward(grid, cams, opts, rays=rays)
        grad, loss = plx.render_backward_grid(grid, cams, opts, rgb_target, depth_target,
                                              out["rgb"], out["depth"], rays=rays)
        ctx.save_for_backward(grad)
        ctx.sh_shape = sh.shape
        ctx.mark_non_differentiable(out["rgb"], out["depth"])
        return loss[0], out["rgb"], out["depth"]

    @staticmethod
    def backward(ctx, g_loss, _g_rgb, _g_depth):
        (grad,) = ctx.saved_tensors
        s = g_loss.to(grad.dtype)
        gd = grad[:, 0] * s
        gs = (grad[:, 1:28] * s).reshape(ctx.sh_shape)
        return gd, gs, None, None, None, None, None, None


def mapping_loss(density: torch.Tensor, sh: torch.Tensor, grid: "plx.Grid",
                 cams: "plx.CameraSet", opts, rgb_target: torch.Tensor,
                 depth_target: torch.Tensor, rays=None):
    """Loss (FP64 scalar) of the rays, rendered colour and depth; differentiable
    in ``density`` [n_alloc] and ``sh`` [n_alloc, 27] (the values are uploaded
    into ``grid``, whose links fix the sparsity)."""
    return MappingLoss.apply(density, sh, grid, cams, opts, rgb_target, depth_target, rays)
