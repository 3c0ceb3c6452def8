"""PyTorch autograd over the hand-written adjoint kernels.

``mapping_loss(density, sh, ...)`` is the RGB-D loss of a ray batch
(L = L_p + lambda_d L_g, Sec. 5.2, Eq. 4, 5, 11) as a differentiable function
of the grid values; its gradient is the analytic adjoint of Eq. 6-10
(``plx_render_backward_grid``). The forward renders (``plx_render_forward``)
and takes the loss alone (the adjoint entry with no gradient buffer); the
adjoint runs only when autograd asks for the gradient, from the forward's
colour and depth, recomputing the per-sample transmittance over each ray's
compositing range (the forward writes it, 8 bytes per ray, unless the options
name a ``plx.RayRange`` already; the same gradient as a full re-march). Options naming a
sample cache (``plx.SampleCache.opts``) make that adjoint read back the
forward's compositing samples instead of re-marching (the cache must not be
refilled between the forward and the backward). The values are uploaded into
the grid only when they are not the ones it holds already (same tensors,
unchanged since the last upload).

``pose_loss(xi, ...)`` is the same loss of one camera's rays as a function of
a left perturbation xi = (rho, phi) of its pose, T <- exp(xi^) T (Sec. 5.3,
Eq. 12-14); its gradient is 2 J^T W r from ``plx_render_backward_pose``, the
derivative with respect to a perturbation of the evaluated pose exp(xi^) T.
That is d loss / d xi exactly at xi = 0; a caller that optimises xi applies
it with ``retract`` (pose <- exp(xi^) pose, on the device) and restarts from
xi = 0, as the trackers do.
"""
from __future__ import annotations

import weakref

import torch

from . import plx


def _upload_if_changed(grid, density, sh):
    """Upload density / sh into ``grid`` unless they are the very tensor
    objects uploaded last (held by weak reference, so a new tensor that reuses
    a freed one's memory is not mistaken for it) and their version counters
    say they are unchanged since."""
    last = getattr(grid, "_autograd_values", None)
    if last is not None:
        d_ref, d_ver, s_ref, s_ver = last
        if d_ref() is density and s_ref() is sh and density._version == d_ver \
                and sh._version == s_ver:
            return
    grid.upload(density.detach().float().contiguous(),
                sh.detach().float().reshape(-1, 27).contiguous())
    grid._autograd_values = (weakref.ref(density), density._version, weakref.ref(sh),
                             sh._version)


class MappingLoss(torch.autograd.Function):
    @staticmethod
    def forward(ctx, density, sh, grid, cams, opts, rgb_target, depth_target, rays):
        _upload_if_changed(grid, density, sh)
        if not opts.ray_range:  # the options copy keeps the range alive for backward
            n = cams.n_pixels() if rays is None else int(rays[1].shape[0])
            opts = plx.RayRange(n, device=rgb_target.device).opts(opts)
        out = plx.render_forward(grid, cams, opts, rays=rays, state=False)
        _, loss = plx.render_backward_grid(grid, cams, opts, rgb_target, depth_target,
                                           out["rgb"], out["depth"], rays=rays, grad=False)
        ctx.save_for_backward(rgb_target, depth_target, out["rgb"], out["depth"])
        ctx.args = (grid, cams, opts, rays)
        ctx.sh_shape = sh.shape
        ctx.mark_non_differentiable(out["rgb"], out["depth"])
        return loss[0], out["rgb"], out["depth"]

    @staticmethod
    def backward(ctx, g_loss, _g_rgb, _g_depth):
        rgb_target, depth_target, rgb, depth = ctx.saved_tensors
        grid, cams, opts, rays = ctx.args
        grad, _ = plx.render_backward_grid(grid, cams, opts, rgb_target, depth_target, rgb, depth,
                                           rays=rays)
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


def _apply_twist(pose, xi):
    """pose (device float64 [12]) <- exp(xi^) pose, through plx_pose_step with
    the identity system (its solve returns xi itself)."""
    eye = torch.eye(6, dtype=torch.float64, device=pose.device)
    plx.pose_step(eye, -xi.detach().to(torch.float64).contiguous(), pose)


class PoseLoss(torch.autograd.Function):
    @staticmethod
    def forward(ctx, xi, grid, cams, cam, opts, rgb_target, depth_target, rays):
        base = cams.poses[cam].clone()
        try:
            _apply_twist(cams.poses[cam], xi)
            H, b, loss = plx.render_backward_pose(grid, cams, cam, opts, rgb_target, depth_target,
                                                  rays=rays)
        finally:
            cams.poses[cam].copy_(base)
        ctx.save_for_backward(b)
        return loss[0]

    @staticmethod
    def backward(ctx, g_loss):
        (b,) = ctx.saved_tensors
        return 2.0 * b * g_loss.to(b.dtype), None, None, None, None, None, None, None


def pose_loss(xi: torch.Tensor, grid: "plx.Grid", cams: "plx.CameraSet", cam: int, opts,
              rgb_target: torch.Tensor, depth_target: torch.Tensor, rays=None):
    """Loss (FP64 scalar) of camera ``cam``'s rays at the pose exp(xi^) T,
    differentiable in ``xi`` (float64 [6] on the device, translation first)."""
    return PoseLoss.apply(xi, grid, cams, cam, opts, rgb_target, depth_target, rays)


def retract(cams: "plx.CameraSet", cam: int, xi: torch.Tensor) -> None:
    """Apply a perturbation to the stored pose, T <- exp(xi^) T, and zero xi
    (in place, no autograd history)."""
    with torch.no_grad():
        _apply_twist(cams.poses[cam], xi)
        xi.zero_()
