"""Mapping then tracking over a short synthetic sequence (Sec. 6.1's
pipeline): the dynamic grid is grown from the keyframes' depth, mapped with
RMSProp on random rays, and every frame is tracked with Adam in a CUDA graph.
Bounds are loose (a few voxels); they catch a broken step, not a regression of
a millimetre."""
import numpy as np
import pytest

from paper_2307_03404_b300 import pipeline, scenes

pytestmark = pytest.mark.gpu


def test_short_sequence_maps_and_tracks():
    sc = scenes.room_scene(128, 0.1, 20, 1002)
    out = pipeline.run(sc, n_frames=60, span=0.06, map_every=10,
                       map_cfg=pipeline.MapConfig(iters=300, rays_per_step=1 << 17),
                       track_cfg=pipeline.TrackConfig(iters=150, n_rays=2048),
                       extra_track_cfgs=[pipeline.TrackConfig(method="lm", lm_iters=10)])
    assert out["keyframes"] == 6 and out["allocated"] > 0
    first, last = out["map_loss_first_last"]
    assert last < 0.05 * first
    assert out["mapping"]["l1_depth_m"] < 0.1
    assert out["mapping"]["psnr_db"] > 20
    assert out["median_err_m"] < 0.02       # 128^3 over 6.4 m: 5 cm voxels
    assert out["max_err_m"] < 0.1
    assert np.isfinite(out["ate_m"])
    lm = out["other_trackers"][0]
    assert lm["median_err_m"] < 0.02 and lm["max_err_m"] < 0.1
