"""The batched persistent launch against the separate entry points and the
oracle: uneven frame sizes, a camera used twice, mapping and tracking mixed."""
import numpy as np
import pytest
import torch

import oracle
from gpu_helpers import dev, norm_err
from paper_2307_03404_b300 import plx, scenes

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("cache", [None, "all", "part"])
def test_batch_matches_separate_calls_and_oracle(cache):
    """cache "all": a sample cache row for every thread slot; "part": rows
    for 100 slots only and 2 samples each, so most mapping rays re-march and
    the rest overflow or fit."""
    g = scenes.tiny_grid(9, seed=41, alloc_frac=0.7, sigma_mean=2.0, sigma_std=2.0)
    T = [scenes.look_at((2.2, 1.4, -2.6), (0, 0.1, 0)), scenes.look_at((-2.0, 0.8, 2.4), (0.1, 0, 0)),
         scenes.look_at((2.6, -1.0, 1.5), (0, 0, 0))]
    cams_np = [scenes.Camera(9.0, 9.0, 8.3, 5.4, 17, 11, T[0]),
               scenes.Camera(5.0, 5.0, 4.0, 2.0, 8, 4, T[1]),
               scenes.Camera(12.0, 12.0, 16.0, 8.0, 33, 19, T[2])]
    work = [(0, plx.WORK_MAP), (1, plx.WORK_TRACK), (2, plx.WORK_MAP), (0, plx.WORK_TRACK),
            (2, plx.WORK_TRACK), (1, plx.WORK_MAP)]
    sizes = [cams_np[c].width * cams_np[c].height for c, _ in work]
    rows = int(sum(sizes))
    rng = np.random.default_rng(8)
    rgb_t = rng.uniform(0, 1, (rows, 3)).astype(np.float32)
    depth_t = rng.uniform(1.0, 4.0, rows).astype(np.float32)
    depth_t[::13] = 0.0
    opts_d = dict(step=0.09, bg=(0.2, 0.3, 0.1), lambda_d=0.6)
    o = plx.opts_from_dict(opts_d)
    grid = plx.Grid.from_scene(g, "f32")
    cams = plx.CameraSet(cams_np)
    ob = o
    if cache == "all":
        ob = plx.SampleCache.for_batch(64).opts(o)
    elif cache == "part":
        ob = plx.SampleCache(100, 2).opts(o)
    grad, mloss, H, b, tloss = plx.render_batch(grid, cams, work, ob, dev(rgb_t), dev(depth_t))
    torch.cuda.synchronize()
    grid.check()
    offs = np.cumsum([0] + sizes)
    # mapping: one list-mode call over all mapping rows (same M)
    mrows = [np.arange(offs[i], offs[i + 1]) for i, (c, m) in enumerate(work) if m == plx.WORK_MAP]
    mcid = np.concatenate([np.full(sizes[i], c, np.int32)
                           for i, (c, m) in enumerate(work) if m == plx.WORK_MAP])
    mpix = np.concatenate([np.arange(sizes[i], dtype=np.int32)
                           for i, (c, m) in enumerate(work) if m == plx.WORK_MAP])
    mr = np.concatenate(mrows)
    rr = (dev(mcid, torch.int32), dev(mpix, torch.int32))
    f = plx.render_forward(grid, cams, o, rays=rr)
    g2, l2 = plx.render_backward_grid(grid, cams, o, dev(rgb_t[mr]), dev(depth_t[mr]), f["rgb"],
                                      f["depth"], rays=rr)
    gb, g2n = grad.cpu().numpy(), g2.cpu().numpy()
    assert mloss[1].item() == l2[1].item()
    assert abs(mloss[0].item() - l2[0].item()) <= 1e-6 * l2[0].item()
    assert norm_err(gb[:, :28], g2n[:, :28]) <= 1e-5
    ref = oracle.grad_grid(g, cams_np, opts_d, rgb_t[mr], depth_t[mr], rays=(mcid, mpix))
    assert norm_err(gb[:, 0], ref.grad_density) <= 1e-4
    assert norm_err(gb[:, 1:28], ref.grad_sh) <= 1e-4
    # tracking: each item against plx_render_backward_pose and the oracle
    tk = [(i, c) for i, (c, m) in enumerate(work) if m == plx.WORK_TRACK]
    for s, (i, c) in enumerate(tk):
        sl = slice(offs[i], offs[i + 1])
        H2, b2, l3 = plx.render_backward_pose(grid, cams, c, o, dev(rgb_t[sl]), dev(depth_t[sl]))
        assert tloss[s, 1].item() == l3[1].item()
        # small frames take the warp-per-ray pose kernel in the separate call:
        # the same per-ray terms, FP32 sums in another order
        assert norm_err(H[s].cpu().numpy(), H2.cpu().numpy()) <= 1e-5
        assert norm_err(b[s].cpu().numpy(), b2.cpu().numpy()) <= 1e-5
        pr = oracle.pose_jacobian(g, [cams_np[c]], opts_d, rgb_t[sl], depth_t[sl])
        assert norm_err(H[s].cpu().numpy(), pr.H) <= 1e-4
        assert norm_err(b[s].cpu().numpy(), pr.b) <= 1e-4
    grid.close()
