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


def test_roofline_bound_is_the_closest_ceiling(monkeypatch):
    """roofline_block: with an ncu record the bound is whichever fraction is
    largest (L2 reductions, L2 reads, instruction issue); without one it is
    the HBM roofline of the compulsory bytes; the no-reuse model is only a
    diagnostic beside it."""
    ceil = {"red_per_s": 200e9, "red_rows_per_s": 40e9, "gather_float4_per_s": 300e9}
    rec = {"kernel": "backward_grid", "workload": "w", "storage": "f32",
           "dram_bytes_per_launch": 1e9, "warp_instructions_per_launch": 1.2e9,
           "red_requests_per_launch": 0.5e9, "read_requests_per_launch": 1e6,
           "rays_per_launch": 1000}
    monkeypatch.setattr(bench, "measured_profile", lambda k, w, s: rec)
    monkeypatch.setattr(bench, "peaks", lambda: (6500.0, "measured"))
    clocks = {"sm_mhz": 2000.0}
    import types
    import sys

    fake_torch = types.SimpleNamespace(cuda=types.SimpleNamespace(
        current_device=lambda: 0,
        get_device_properties=lambda d: types.SimpleNamespace(multi_processor_count=100)))
    monkeypatch.setitem(sys.modules, "torch", fake_torch)
    # 5 ms launch over 2000 rays: 1e9 reductions -> 200 G/s = 1.0 of the ceiling;
    # 2.4e9 warp instructions / 5 ms = 480 G/s against 100 x 4 x 2e9 = 800 G/s
    b = bench.roofline_block("backward_grid", "w", "f32", 2000, 5.0, ceil, 1e8, 1e12, "m",
                             clocks)
    assert b["bound"] == "l2_atomic" and abs(b["frac"] - 1.0) < 1e-12
    assert abs(b["issue"]["frac"] - 0.6) < 1e-12
    assert abs(b["hbm"]["frac"] - (1e8 / 5e-3 / 1e9) / 6500.0) < 1e-12
    assert b["no_reuse"]["frac"] > 1 and b["traffic"] == 2e9
    rec["red_requests_per_launch"] = 0.1e9          # now issue is the closest
    b = bench.roofline_block("backward_grid", "w", "f32", 2000, 5.0, ceil, 1e8, 1e12, "m",
                             clocks)
    assert b["bound"] == "alu" and abs(b["frac"] - 0.6) < 1e-12
    # the sample-cache adjoint sends one coalesced request per row: its
    # requests are held against the probe's row rate (0.1e9 x 2 / 5 ms = 40 G/s
    # against 40 G/s, where the per-float4 rate gave 0.2 and "alu" won)
    b = bench.roofline_block("backward_grid_cached", "w", "f32", 2000, 5.0, ceil, 1e8, 1e12,
                             "m", clocks)
    assert b["bound"] == "l2_atomic" and abs(b["frac"] - 1.0) < 1e-12
    assert b["l2"]["red"]["peak"] == 40e9
    # with the probe's measured issue rate, instruction issue is held against
    # it instead of the nominal rate: 480 G/s against 600 G/s = 0.8
    ceil_m = dict(ceil, issue_warp_inst_per_s=600e9)
    rec["red_requests_per_launch"] = 0.1e9
    b = bench.roofline_block("backward_grid", "w", "f32", 2000, 5.0, ceil_m, 1e8, 1e12, "m",
                             clocks)
    assert b["bound"] == "alu" and abs(b["frac"] - 0.8) < 1e-12
    assert b["issue"]["peak"] == 600e9 and b["issue"]["nominal_peak"] == 800e9
    assert b["issue"]["peak_basis"].startswith("measured")
    monkeypatch.setattr(bench, "measured_profile", lambda k, w, s: None)
    b = bench.roofline_block("backward_grid", "w", "f32", 2000, 5.0, ceil, 1e8, 1e12, "m",
                             clocks)
    assert b["bound"] == "hbm" and b["unit"] == "GB/s" and b["traffic"] is None
