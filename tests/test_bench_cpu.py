"""Host logic of bench.py's byte model and profile scaling (no GPU)."""
import json

import numpy as np

import bench


def test_byte_model_with_and_without_the_sample_cache():
    # three rays: (marched, with an allocated corner), compositing samples kept
    counts = np.array([[100, 10], [50, 0], [300, 40]], np.int32)
    valid = np.array([True, True, False])
    fwd, bwd, s_all, s_occ = bench.bytes_model(counts, "f32", valid)
    assert fwd == (100 + 50 + 300) * 32 + (10 + 0 + 40) * 896 + 20 * 3
    assert bwd == (100 + 50) * 32 + (10 + 0) * (896 + 1792) + 32 * 2 + 4 * 3
    assert s_all == 150.0 and s_occ == 50 / 3
    # cache of cap 8: ray 0 keeps 12 (overflows: re-marched), ray 1 keeps 0
    kept = np.array([12, 0, 5])
    fwd_c, bwd_c, _, _ = bench.bytes_model(counts, "bf16", valid, kept, 8)
    assert fwd_c == (450 * 32 + 50 * 448 + 20 * 3) + 20 * (8 + 0 + 5) + 4 * 3
    # ray 0 re-marches; ray 1 fits with nothing kept; ray 2 has no valid depth
    assert bwd_c == (100 * 32 + 10 * (448 + 1792)) + 32 * 2 + 4 * 3 + 0 + 4 * 3


def test_profile_figures_scale_with_the_rays():
    rec = {"dram_bytes_per_launch": 1000, "rays_per_launch": 100}
    assert bench._per_launch(rec, "dram_bytes_per_launch", 400) == 4000
    assert bench._per_launch(rec, "dram_bytes_per_launch", None) == 1000
    assert bench._per_launch({"dram_bytes_per_launch": 7}, "dram_bytes_per_launch", 50) == 7


def test_committed_profile_records_name_their_capture():
    recs = json.load(open(bench.os.path.join(bench.ROOT, "profiles", "traffic.json")))
    for r in recs:
        assert r["command"].startswith("ncu ") and "--clock-control none" in r["command"]
        assert r["rays_per_launch"] > 0 and r["dram_bytes_per_launch"] > 0
