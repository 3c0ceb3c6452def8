"""The allocation-free pose entry point against the regular one.

``plx_render_backward_pose_noalloc`` is for callers that cannot allocate
device memory while they run (a real-time tracking loop, or an application
whose device memory belongs to another allocator). It takes the grid as plain
arrays and keeps its scratch in a static device array of the library. This
file is collected last so that a run stopping at the first failure has run
every other test; it also passes alone in a fresh process.
"""
import ctypes as C

import numpy as np
import pytest
import torch

import oracle
from paper_2307_03404_b300 import plx, scenes

pytestmark = pytest.mark.gpu


def _norm_err(x, ref):
    return float(np.abs(x - ref).max() / max(np.abs(ref).max(), 1e-300))


def test_noalloc_pose_matches_regular_entry_twice_in_a_row():
    g, cam, _ = scenes.sphere_scene()
    opts = dict(step=0.5 * g.h[0], lambda_d=0.8, depth_is_z=False, bg=(0.1, 0.1, 0.2))
    ref_t = oracle.render(g, [cam], opts)
    T0 = scenes.perturb_pose(cam.T_wc, 0.03, 2.0, np.random.default_rng(9))
    cams = plx.CameraSet([cam.with_pose(T0)])
    o = plx.opts_from_dict(opts)
    rgb_t = torch.tensor(ref_t.rgb, dtype=torch.float32, device="cuda")
    depth_t = torch.tensor(ref_t.depth, dtype=torch.float32, device="cuda")

    grid = plx.Grid.from_scene(g, "f32")
    H_ref, b_ref, l_ref = plx.render_backward_pose(grid, cams, 0, o, rgb_t, depth_t)
    torch.cuda.synchronize()

    # the same grid as caller-owned arrays in the F32 record layout
    links = torch.from_numpy(g.links).cuda()
    dens = torch.from_numpy(g.density).cuda()
    sh = torch.from_numpy(g.sh).cuda()
    records = torch.cat([dens[:, None], sh, torch.zeros(g.n_alloc, 4, device="cuda")], 1)
    records = records.contiguous()
    desc = plx.GridDesc()
    desc.res[:] = list(g.res)
    desc.lo[:] = [float(v) for v in g.lo]
    desc.hi[:] = [float(v) for v in g.hi]
    desc.n_alloc = g.n_alloc
    desc.storage = plx.STORE_F32
    rays = plx.Rays()
    cs = cams.struct()
    stream = C.c_void_p(torch.cuda.current_stream().cuda_stream)
    for call in range(2):
        H = torch.full((6, 6), np.nan, dtype=torch.float64, device="cuda")
        b = torch.full((6,), np.nan, dtype=torch.float64, device="cuda")
        loss = torch.full((2,), np.nan, dtype=torch.float64, device="cuda")
        st = plx._lib.plx_render_backward_pose_noalloc(
            C.byref(desc), C.c_void_p(links.data_ptr()), C.c_void_p(records.data_ptr()),
            C.byref(cs), 0, C.byref(rays), C.byref(o), C.c_void_p(rgb_t.data_ptr()),
            C.c_void_p(depth_t.data_ptr()), C.c_void_p(H.data_ptr()), C.c_void_p(b.data_ptr()),
            C.c_void_p(loss.data_ptr()), stream)
        assert st == 0, plx._lib.plx_last_error()
        torch.cuda.synchronize()
        assert loss[1].item() == l_ref[1].item()
        assert abs(loss[0].item() - l_ref[0].item()) <= 1e-5 * l_ref[0].item()
        assert _norm_err(H.cpu().numpy(), H_ref.cpu().numpy()) <= 1e-4, call
        assert _norm_err(b.cpu().numpy(), b_ref.cpu().numpy()) <= 1e-4, call
    grid.close()
