"""Launch choices change speed, not results; the autotuner picks one and
caches it."""
import json

import numpy as np
import pytest
import torch

import oracle
from gpu_helpers import GpuCase, dev, norm_err, rel_err
from paper_2307_03404_b300 import autotune, plx, scenes

pytestmark = pytest.mark.gpu


def test_every_launch_config_gives_the_oracle_result():
    g, cam, gp = scenes.sphere_scene()
    opts = dict(step=0.5 * g.h[0], lambda_d=0.7, depth_is_z=False)
    tg = oracle.render(gp, [cam], opts)
    ref = oracle.render(g, [cam], opts)
    rg = oracle.grad_grid(g, [cam], opts, tg.rgb, tg.depth)
    rp = oracle.pose_jacobian(g, [cam], opts, tg.rgb, tg.depth)
    case = GpuCase(g, [cam])
    assert case.grid.get_config() == dict(block_shift=3, forward_blocks=1, adjoint_blocks=2,
                                          pose_blocks=2, batch_blocks=1, fine_skip=14,
                                          seg_rays=16384)
    # seg_rays 0: one ray per lane; 2^24: a warp per ray (the 3,072 rays here)
    for shift, fine, seg in ((1, 0, 0), (2, 15, 1 << 24), (3, 0, 0), (4, 15, 0), (4, 0, 1 << 24),
                             (3, 5, 0), (3, 14, 1 << 24)):
        for blocks in (1, 2):
            case.grid.set_config(block_shift=shift, forward_blocks=blocks, adjoint_blocks=blocks,
                                 pose_blocks=blocks, fine_skip=fine, seg_rays=seg)
            got = case.forward(opts)
            assert rel_err(got["rgb"], ref.rgb) <= 1e-5
            np.testing.assert_array_equal(got["counts"][:, 1], ref.n_alloc)
            gd, gs, _, loss = case.backward_grid(opts, tg.rgb.astype(np.float32),
                                                 tg.depth.astype(np.float32))
            assert norm_err(gd, rg.grad_density) <= 1e-4 and norm_err(gs, rg.grad_sh) <= 1e-4
            H, b, _ = case.backward_pose(opts, 0, tg.rgb.astype(np.float32),
                                         tg.depth.astype(np.float32))
            assert norm_err(H, rp.H) <= 1e-4 and norm_err(b, rp.b) <= 1e-4
    with pytest.raises(plx.PlxError):
        case.grid.set_config(block_shift=0)
    # the forward also at 3 blocks per SM
    case.grid.set_config(block_shift=3, forward_blocks=3, adjoint_blocks=2, pose_blocks=2,
                         fine_skip=14)
    got = case.forward(opts)
    assert rel_err(got["rgb"], ref.rgb) <= 1e-5
    np.testing.assert_array_equal(got["counts"][:, 1], ref.n_alloc)
    with pytest.raises(plx.PlxError):
        case.grid.set_config(adjoint_blocks=3)
    with pytest.raises(plx.PlxError):
        case.grid.set_config(forward_blocks=4)
    with pytest.raises(plx.PlxError):
        case.grid.set_config(fine_skip=16)
    with pytest.raises(plx.PlxError):
        case.grid.set_config(seg_rays=-1)
    with pytest.raises(plx.PlxError):
        case.grid.set_config(seg_rays=(1 << 24) + 1)


def test_autotuner_picks_and_caches_a_config(tmp_path):
    g, cam, gp = scenes.sphere_scene()
    opts = dict(step=0.5 * g.h[0], lambda_d=0.7, depth_is_z=False)
    tg = oracle.render(gp, [cam], opts)
    grid = plx.Grid.from_scene(g, "f32")
    cams = plx.CameraSet([cam])
    o = plx.opts_from_dict(opts)
    cache = str(tmp_path / "tuning.json")
    r1 = autotune.tune_mapping(grid, cams, o, dev(tg.rgb), dev(tg.depth), reps=2, cache=cache)
    assert not r1["cached"] and len(r1["trials"]) >= 5
    assert r1["ms"] <= min(t for _, t in r1["trials"]) + 1e-9
    # 3,072 rays: the rays per warp are tuned too, and a warp per ray wins
    # (7x faster than one ray per lane at this size)
    assert {c["seg_rays"] for c, _ in r1["trials"]} >= {0, 16384}
    assert r1["config"]["seg_rays"] > 0
    grid2 = plx.Grid.from_scene(g, "f32")
    r2 = autotune.tune_mapping(grid2, cams, o, dev(tg.rgb), dev(tg.depth), cache=cache)
    assert r2["cached"] and grid2.get_config() == r1["config"]
    rt = autotune.tune_tracking(grid, cams, 0, o, dev(tg.rgb), dev(tg.depth), reps=2, cache=cache)
    assert rt["config"]["pose_blocks"] in (1, 2)
    assert len(json.load(open(cache))) == 2
