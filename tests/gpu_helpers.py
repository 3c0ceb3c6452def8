"""Helpers shared by the GPU parity tests: run the CUDA path through the C ABI
binding and the oracle on the same seeded inputs, and measure the difference."""
import numpy as np
import torch

from paper_2307_03404_b300 import plx


def rel_err(x, ref, floor=1e-3):
    """max over elements of |x - ref| / max(|ref|, floor)."""
    x, ref = np.asarray(x, np.float64), np.asarray(ref, np.float64)
    if x.size == 0:
        return 0.0
    return float(np.max(np.abs(x - ref) / np.maximum(np.abs(ref), floor)))


def norm_err(x, ref):
    """||x - ref||_inf / ||ref||_inf (gradients: elementwise relative error is
    ill-posed where they are near zero)."""
    x, ref = np.asarray(x, np.float64), np.asarray(ref, np.float64)
    den = np.abs(ref).max()
    return float(np.abs(x - ref).max() / (den if den > 0 else 1.0))


def dev(a, dtype=torch.float32):
    return torch.as_tensor(np.ascontiguousarray(a)).to("cuda", dtype)


class GpuCase:
    """A grid handle + cameras for one scene."""

    def __init__(self, grid, cams, storage="f32"):
        self.grid_np = grid
        self.cams_np = list(cams)
        self.grid = plx.Grid.from_scene(grid, storage)
        self.cams = plx.CameraSet(self.cams_np)

    def forward(self, opts, rays=None, counts=True):
        o = plx.opts_from_dict(opts)
        rr = None if rays is None else (dev(rays[0], torch.int32), dev(rays[1], torch.int32))
        out = plx.render_forward(self.grid, self.cams, o, rays=rr, counts=counts)
        torch.cuda.synchronize()
        self.grid.check()
        return {k: (v.cpu().numpy() if v is not None else None) for k, v in out.items()}

    def backward_grid(self, opts, rgb_t, depth_t, rays=None, cache_cap=None, ray_range=False):
        """Forward then grid adjoint; with cache_cap, through a sample cache
        of that many samples per ray (self.cache keeps it for inspection);
        with ray_range, the forward writes each ray's compositing range and
        the re-marching adjoint marches only that (self.range keeps it)."""
        o = plx.opts_from_dict(opts)
        rr = None if rays is None else (dev(rays[0], torch.int32), dev(rays[1], torch.int32))
        n = self.cams.n_pixels() if rays is None else len(rays[1])
        if cache_cap is not None:
            self.cache = plx.SampleCache(n, cache_cap)
            o = self.cache.opts(o)
        if ray_range:
            self.range = plx.RayRange(n)
            o = self.range.opts(o)
        out = plx.render_forward(self.grid, self.cams, o, rays=rr)
        grad, loss = plx.render_backward_grid(self.grid, self.cams, o, dev(rgb_t), dev(depth_t),
                                              out["rgb"], out["depth"], rays=rr)
        torch.cuda.synchronize()
        self.grid.check()
        g = grad.cpu().numpy()
        return g[:, 0], g[:, 1:28], g[:, 28:], loss.cpu().numpy()

    def backward_pose(self, opts, cam, rgb_t, depth_t, pixels=None):
        o = plx.opts_from_dict(opts)
        pr = None if pixels is None else dev(pixels, torch.int32)
        H, b, loss = plx.render_backward_pose(self.grid, self.cams, cam, o, dev(rgb_t),
                                              dev(depth_t), rays=pr)
        torch.cuda.synchronize()
        self.grid.check()
        return H.cpu().numpy(), b.cpu().numpy(), loss.cpu().numpy()

    def close(self):
        self.grid.close()
