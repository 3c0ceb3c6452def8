"""Benchmark: mapping rays/s (forward + backward to the grid) and tracking
iterations/s at 640x480, on seeded synthetic scenes.

Workload (one step): every ray of 8 keyframes of 640x480 (2,457,600 rays)
through a 256^3 grid with 10% of vertices allocated (analytic room with 20
primitives): forward render (Eq. 1-3), RGB-D loss (Eq. 4, 5, 11) and its
gradient to every grid value (Eq. 6-10), written into a zeroed gradient
buffer. By default the forward keeps each ray's compositing samples in a
sample cache sized (untimed) by a probe forward, and the adjoint reads them
back instead of re-marching (--sample-cache off re-marches every ray).
Tracking: 100 Gauss-Newton iterations (pose Jacobian + FP64 solve + SE(3)
step) on one 640x480 frame against a 512^3 grid with 5% allocated, captured
in one CUDA graph.

Usage: python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
Under torchrun each rank maps its own 8 keyframes of the same scene (weak
scaling, no data-path collective); rank 0 prints one JSON line.
"""
import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "mapping rays/s fwd+bwd & tracking iters/s @640x480, % HBM roofline, vs FP32"
FRAMES_PER_RANK = 8
FALLBACK_HBM_GBS = 6400.0


def log(*a):
    print(*a, file=sys.stderr, flush=True)


def shard_frames(world: int, rank: int, per_rank: int = FRAMES_PER_RANK):
    """Keyframe indices of ``rank`` when ``world`` ranks each map ``per_rank``
    keyframes of one trajectory of ``world * per_rank`` keyframes."""
    return list(range(rank * per_rank, (rank + 1) * per_rank))


def rank_max(x: float, world: int, device) -> float:
    """Maximum of ``x`` over all ranks (host-side timing only; not on the data
    path)."""
    if world == 1:
        return x
    import torch
    import torch.distributed as dist

    t = torch.tensor([x], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def combine_rank_times(times_ms, units_per_rank):
    """Whole-job throughput: all ranks' units over the slowest rank's time."""
    t = max(times_ms)
    return sum(units_per_rank) / (t / 1e3), t


# the sources each profiled kernel is built from
KERNEL_SOURCES = {
    "forward": ("plx_internal.cuh", "plx_march.cuh", "plx_render.cu"),
    "backward_grid": ("plx_internal.cuh", "plx_march.cuh", "plx_render.cu"),
    "backward_grid_cached": ("plx_internal.cuh", "plx_march.cuh", "plx_render.cu"),
    "backward_pose": ("plx_internal.cuh", "plx_pose_march.cuh", "plx_pose.cu"),
}


def kernel_source_sha(kernel=None):
    """Hash of the CUDA sources (of one kernel's files, or of all): a
    DRAM-traffic record taken with ncu applies only to the kernel it was
    measured on."""
    import glob
    import hashlib

    csrc = os.path.join(ROOT, "paper_2307_03404_b300", "csrc")
    files = (sorted(glob.glob(os.path.join(csrc, "*.cu*"))) if kernel is None
             else [os.path.join(csrc, f) for f in KERNEL_SOURCES[kernel]])
    h = hashlib.sha256()
    for f in files:
        h.update(open(f, "rb").read())
    return h.hexdigest()[:16]


def measured_profile(kernel, workload, storage):
    """The ncu record of profiles/traffic.json (DRAM bytes and warp
    instructions per launch) if it was taken on the current kernel sources,
    else None."""
    p = os.path.join(ROOT, "profiles", "traffic.json")
    if not os.path.exists(p):
        return None
    for rec in json.load(open(p)):
        if (rec["kernel"] == kernel and rec["workload"] == workload
                and rec["storage"] == storage and rec["source_sha"] == kernel_source_sha(kernel)):
            return rec
    return None


def _per_launch(rec, key, n_rays):
    """A per-launch ncu figure scaled to a launch over n_rays rays when the
    capture ran on fewer (a smaller case of the same kernel, see
    rays_per_launch in the record)."""
    v = rec[key]
    if n_rays and rec.get("rays_per_launch"):
        v = v * n_rays / rec["rays_per_launch"]
    return v


def measured_traffic(kernel, workload, storage, n_rays=None, key="dram_bytes_per_launch"):
    """An ncu per-launch figure of profiles/traffic.json (DRAM bytes by
    default; ``key`` names another, e.g. red_requests_per_launch), scaled to
    n_rays rays; None if no record was taken on the current sources."""
    rec = measured_profile(kernel, workload, storage)
    return _per_launch(rec, key, n_rays) if rec and key in rec else None


def issue_roofline(kernel, ms, storage, clocks, n_rays=None, workload="room256", ceil=None):
    """Instruction-issue utilisation of a kernel: warp instructions per launch
    (ncu, profiles/traffic.json, valid for the current sources, scaled to
    n_rays rays) over the live launch time, against the issue rate plx_probe
    measures live (independent FP32 FMA chains, ``ceil["issue_warp_inst_per_s"]``);
    without that measurement, against one warp instruction per clock per SM
    sub-partition (4 per SM) at the SM clock sampled during the run."""
    import torch

    rec = measured_profile(kernel, workload, storage)
    if not rec or "warp_instructions_per_launch" not in rec:
        return None
    sms = torch.cuda.get_device_properties(torch.cuda.current_device()).multi_processor_count
    mhz = (clocks or {}).get("sm_mhz") or 2032.0
    nominal = sms * 4 * mhz * 1e6
    measured = (ceil or {}).get("issue_warp_inst_per_s")
    peak = measured or nominal
    wi = _per_launch(rec, "warp_instructions_per_launch", n_rays)
    achieved = wi / (ms / 1e3)
    basis = (f"measured: plx_probe FP32 FMA issue rate ({measured / nominal:.3f} of {sms} SMs x "
             f"4 sub-partitions x 1 warp instruction per clock x {mhz:.0f} MHz)" if measured else
             f"{sms} SMs x 4 sub-partitions x 1 warp instruction per clock x {mhz:.0f} MHz")
    return {"achieved": achieved, "peak": peak, "unit": "warp instructions/s",
            "frac": achieved / peak, "warp_instructions_per_launch": wi,
            "nominal_peak": nominal, "peak_basis": basis}


def l2_ceilings(rows=600_000, reps=5):
    """Rates the memory system sustains for the mapping kernels' L2 accesses,
    measured live with the library's probe kernels (plx_probe) over a buffer of
    ``rows`` 128-byte rows (the size of the set of vertices one room256 step
    touches, so it stays in L2): float4 reductions into random rows, 7 per
    row, sent per lane (as the re-marching adjoint's corner flush) and as one
    coalesced request per row (as the sample-cache adjoint's warp-cooperative
    flush), and float4 gathers of random rows (as the record gathers). Best of
    8 and 16 blocks of 256 threads per SM."""
    import torch

    from paper_2307_03404_b300 import plx

    buf = torch.zeros(rows, plx.GRAD_STRIDE, device="cuda")
    sms = torch.cuda.get_device_properties(buf.device).multi_processor_count
    out = {}
    # units per lane and operation: 7 float4 (RED, GATHER) or 1 row (RED_ROWS)
    for kind, name, per in ((plx.PROBE_RED, "red", 7), (plx.PROBE_GATHER, "gather", 7),
                            (plx.PROBE_RED_ROWS, "red_rows", 1)):
        best = 0.0
        for bps in (8, 16):
            blocks, ops = bps * sms, 32
            for _ in range(2):
                plx.probe(kind, buf, 1, ops, blocks)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            torch.cuda.synchronize()
            e0.record()
            for _ in range(reps):
                plx.probe(kind, buf, 1, ops, blocks)
            e1.record()
            torch.cuda.synchronize()
            ms = e0.elapsed_time(e1) / reps
            best = max(best, blocks * 256 * ops * per / (ms / 1e3))
        out[name] = best
    # instruction issue: 512 FMAs per thread and operation, no memory traffic
    # (the few loop instructions per 512 FMAs are not counted: ncu counts
    # 1.024 instructions per FMA with 128 FMAs per operation)
    # (about 20 ms of warm-up first: a lone launch of a few hundred us right
    # after other work read as low as 0.8 of the rate it settles at)
    best = 0.0
    for bps in (8, 16):
        blocks, ops = bps * sms, 64
        for _ in range(40):
            plx.probe(plx.PROBE_ISSUE, buf, 1, ops, blocks)
        for _ in range(3):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            torch.cuda.synchronize()
            e0.record()
            for _ in range(reps):
                plx.probe(plx.PROBE_ISSUE, buf, 1, ops, blocks)
            e1.record()
            torch.cuda.synchronize()
            ms = e0.elapsed_time(e1) / reps
            best = max(best, blocks * 256 // 32 * ops * 512 / (ms / 1e3))
    out["issue"] = best
    del buf
    return {"red_per_s": out["red"], "red_rows_per_s": out["red_rows"],
            "gather_float4_per_s": out["gather"], "issue_warp_inst_per_s": out["issue"],
            "buffer_MB": rows * 128 / 1e6,
            "how": "plx_probe: each lane 32 times picks a random 128-byte row of the buffer and "
                   "issues 7 float4 atomic adds (red, per float4) or 7 float4 loads (gather); "
                   "red_rows: the same rows and adds, 7 lanes per row with one float4 each "
                   "(one coalesced request per row, per row); issue: 512 independent FP32 FMAs "
                   "per thread and operation, counted as warp instructions, after 40 warm-up "
                   "launches, best of 3; best of 8 and 16 blocks of 256 threads per SM, CUDA "
                   "events over 5 launches"}


# how each adjoint kernel sends a corner's 7 float4 reductions: per lane (7 L2
# requests) or warp-cooperatively (one coalesced request per row)
SCATTER_FORM = {"backward_grid": "lanes", "backward_grid_cached": "rows"}


def l2_roofline(kernel, workload, storage, n_rays, ms, ceil):
    """The L2 rates of a kernel against the probe ceilings: reduction requests
    (lts__t_requests_srcunit_tex_op_red.sum) and read requests
    (lts__t_requests_srcunit_tex_op_read.sum) per launch from the ncu record
    of profiles/traffic.json (taken on the current sources, scaled to n_rays
    rays) over the launch time measured here. A kernel that sends each
    corner's row as one coalesced request (SCATTER_FORM "rows") is held
    against the probe's coalesced-row rate, one that sends 7 per-lane float4
    requests against the per-float4 rate. None where no record matches."""
    out = {}
    red_peak = (ceil["red_rows_per_s"] if SCATTER_FORM.get(kernel) == "rows"
                else ceil["red_per_s"])
    for key, name, peak in (("red_requests_per_launch", "red", red_peak),
                            ("read_requests_per_launch", "read", ceil["gather_float4_per_s"])):
        n = measured_traffic(kernel, workload, storage, n_rays, key=key)
        if n:
            rate = n / (ms / 1e3)
            out[name] = {"per_launch": n, "achieved": rate, "peak": peak, "frac": rate / peak,
                         "unit": "requests/s"}
    return out or None


def roofline_block(kernel, workload, storage, n_rays, ms, ceil, compulsory, no_reuse_bytes,
                   hbm_model, clocks=None):
    """The roofline object of a dominant kernel. When its ncu record exists
    the binding ceiling is whichever the kernel comes closest to: the L2
    reduction rate (the grid adjoint's scatter), the L2 gather rate (record
    gathers) or instruction issue (bound "alu": against the warp-instruction
    rate plx_probe measures for independent FP32 FMAs); the HBM figure beside
    it uses the compulsory
    bytes (what the kernel cannot avoid moving), and the fixed no-reuse
    model stays only as a diagnostic."""
    hbm, peak_kind = peaks()
    comp_gbs = compulsory / (ms / 1e3) / 1e9
    traffic = measured_traffic(kernel, workload, storage, n_rays)
    dram_gbs = traffic / (ms / 1e3) / 1e9 if traffic else None
    l2 = l2_roofline(kernel, workload, storage, n_rays, ms, ceil)
    block = {"kernel": kernel, "ms_per_launch": ms, "traffic": traffic}
    hb = {"achieved": comp_gbs, "peak": hbm, "unit": "GB/s", "frac": comp_gbs / hbm,
          "peak_kind": f"{peak_kind} copy bandwidth", "bytes_per_launch": compulsory,
          "model": hbm_model, "dram_gbs": dram_gbs,
          "dram_frac": dram_gbs / hbm if dram_gbs else None}
    nr = no_reuse_bytes / (ms / 1e3) / 1e9
    block["no_reuse"] = {
        "bytes_per_launch": no_reuse_bytes, "achieved": nr, "peak": hbm, "frac": nr / hbm,
        "model": "a diagnostic, not a roofline: the fixed no-reuse byte model (32 B of "
                 "links per marched sample, 896 B (f32) / 448 B (16-bit) per sample with an "
                 "allocated corner per gather, 1792 B of FP32 gradient read-modify-write per "
                 "such sample in the adjoint, per-ray I/O); frac > 1 means L1/L2 reuse, not HBM "
                 "use"}
    issue = issue_roofline(kernel, ms, storage, clocks, n_rays, workload, ceil)
    cands = dict(l2 or {})
    if issue:
        cands["issue"] = issue
    if cands:
        name = max(cands, key=lambda k: cands[k]["frac"])
        b = cands[name]
        block.update({"bound": {"red": "l2_atomic", "read": "l2_gather", "issue": "alu"}[name],
                      "achieved": b["achieved"], "peak": b["peak"], "unit": b["unit"],
                      "frac": b["frac"], "l2": l2, "issue": issue, "hbm": hb,
                      "basis": "the kernel moves little DRAM traffic (hbm below). Per ncu "
                               "record (profiles/traffic.json, taken on the current sources, "
                               "scaled by rays) over the launch time measured here: L2 "
                               "reduction / read requests against the rate plx_probe measures "
                               "live for the same access (float4 reductions, per lane or "
                               "coalesced per row as the kernel sends them, or gathers of "
                               "random 128-byte rows in L2), and warp instructions against "
                               "the issue rate plx_probe measures live for independent FP32 "
                               "FMAs (alu); bound = the largest of these fractions"})
    else:
        block.update({"bound": "hbm", "achieved": comp_gbs, "peak": hbm, "unit": "GB/s",
                      "frac": comp_gbs / hbm, "hbm": hb,
                      "basis": "no ncu record of this kernel's L2 requests on the current "
                               "sources: the HBM roofline of its compulsory bytes"})
    block["ceilings"] = ceil
    return block


def peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        return float(d["hbm_gbs"]), "measured"
    return FALLBACK_HBM_GBS, "fallback"


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled during the timed region."""

    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device_id):
        self.dev = device_id
        self.proc = None
        self.lines = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.dev), f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except OSError:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            self.proc.wait()
            self.t.join(timeout=2)

    def summary(self):
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for l in self.lines:
            f = [x.strip() for x in l.split(",")]
            if len(f) < 8:
                continue
            try:
                sm.append(float(f[0]))
                mx.append(float(f[1]))
            except ValueError:
                continue
            for n, v in zip(names, f[4:8]):
                if v.lower().startswith("active"):
                    reasons.add(n)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx),
                "reasons": sorted(reasons), "samples": len(sm)}


# ---------------------------------------------------------------- workload
def mapping_workload(world, rank, frames=FRAMES_PER_RANK):
    """room256 and this rank's keyframes; ``frames`` < 8 keeps only the first
    of them (a smaller case of the same kernels, for profiler captures)."""
    from paper_2307_03404_b300 import scenes

    R, occ, npr, seed = scenes.WORKLOADS["room256"]
    t = time.time()
    sc = scenes.room_scene(R, occ, npr, seed)
    cams_all = scenes.room_cameras(sc, FRAMES_PER_RANK * world, seed + 1)
    cams = [cams_all[i] for i in shard_frames(world, rank)][:frames]
    rgb_t, depth_t = scenes.sensor_frames(sc, cams, seed + 2 + rank)
    opts = dict(step=0.5 * float(sc.grid.h[0]), lambda_d=1.0, depth_is_z=True)
    log(f"[bench] room256 scene + frames in {time.time() - t:.1f}s, n_alloc {sc.grid.n_alloc}")
    return sc, cams, rgb_t, depth_t, opts


def workload_config(sc, cams, storage):
    n = sum(c.width * c.height for c in cams)
    return {"workload": f"room256: 256^3 grid, {sc.grid.n_alloc} of {256 ** 3} vertices "
                        f"allocated (10%), {len(cams)} keyframes 640x480 = {n} rays; "
                        "forward + RGB-D loss + backward to the grid",
            "storage": storage, "step_voxels": 0.5, "lambda_d": 1.0,
            "l2": "flushed between timed steps (256 MiB write)"}


# ------------------------------------------------------------------- ours
def cache_note(res, n_rays):
    """How the mapping step used the sample cache, for the JSON line."""
    if not res["cache"]:
        return "off: the adjoint re-marches every ray"
    k, cap = res["kept"], res["cache"]["cap"]
    return (f"{cap} compositing samples per ray kept by the forward for the adjoint "
            f"({res['cache']['bytes'] / 1e9:.2f} GB, sized untimed by a probe forward); "
            f"mean {k.mean():.1f}, max {int(k.max())} per ray; "
            f"{int((k > cap).sum())} of {n_rays} rays re-marched")


def bytes_model(counts, storage, valid, kept=None, cap=0):
    """Algorithmic bytes of the forward and the adjoint launch over these rays
    (no reuse: every marched sample reads its 8 links, every sample with an
    allocated corner gathers 8 records, the adjoint adds a read-modify-write of
    8 FP32 gradient rows per such sample; per-ray I/O on top). With a sample
    cache (``kept`` = compositing samples per ray, ``cap``) the forward also
    writes 20 B per kept sample and 4 B per ray, and the adjoint of a ray that
    fits reads them back and, per kept sample, its 8 links and the gradient
    rows' read-modify-write; a ray that overflows is re-marched as without."""
    n_rays = counts.shape[0]
    rec = 896.0 if storage == "f32" else 448.0
    s_all = counts[:, 0].astype(np.float64)
    s_occ = counts[:, 1].astype(np.float64)
    fwd = (s_all * 32 + s_occ * rec).sum() + 20.0 * n_rays
    full = valid if kept is None else valid & (kept > cap)
    bwd = (s_all[full] * 32 + s_occ[full] * (rec + 1792.0)).sum() + 32.0 * valid.sum() \
        + 4.0 * n_rays
    if kept is not None:
        k = kept.astype(np.float64)
        fwd += 20.0 * np.minimum(k, cap).sum() + 4.0 * n_rays
        fit = valid & (kept <= cap)
        bwd += (k[fit] * (20.0 + 32.0 + 1792.0)).sum() + 4.0 * n_rays
    return fwd, bwd, float(s_all.mean()), float(s_occ.mean())


def run_ours(args):
    import torch
    import torch.distributed as dist

    from paper_2307_03404_b300 import plx, scenes

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))

    def barrier():
        if world > 1:
            dist.barrier()
        torch.cuda.synchronize()

    sc, cams_np, rgb_np, depth_np, opts = mapping_workload(world, rank, args.map_frames)
    n_rays = rgb_np.shape[0]
    cams = plx.CameraSet(cams_np)
    o_plain = plx.opts_from_dict(opts)
    rgb_t = torch.from_numpy(rgb_np).cuda()
    depth_t = torch.from_numpy(depth_np).cuda()
    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")
    stream = torch.cuda.current_stream()

    tune_cache = os.path.join("/tmp", f"plx_tuning_{os.getpid()}.json")

    def measure(storage, K, W, with_e2e, cache_mode=None, ray_range=False):
        grid = plx.Grid.from_scene(sc.grid, storage)
        # sample cache: forward keeps each ray's compositing samples for the
        # adjoint; sized (untimed) by a probe forward so that no ray overflows
        scache = None
        o = o_plain
        cache_mode = cache_mode or args.sample_cache
        if cache_mode != "off":
            if cache_mode == "fit":
                scache = plx.SampleCache.sized_for(grid, cams, o_plain)
            else:
                scache = plx.SampleCache(n_rays, int(cache_mode))
            o = scache.opts(o_plain)
        if ray_range:  # each ray's compositing range, written by the forward
            o = plx.RayRange(n_rays).opts(o)
        tuned = None
        if not args.no_tune:
            from paper_2307_03404_b300 import autotune

            tuned = autotune.tune_mapping(grid, cams, o, rgb_t, depth_t, reps=3, cache=tune_cache)
            log(f"[bench] {storage} mapping launch config {tuned['config']} ({tuned['ms']:.2f} ms)")
        fw = {"rgb": torch.empty(n_rays, 3, device="cuda"),
              "depth": torch.empty(n_rays, device="cuda"),
              "state": torch.empty(n_rays, device="cuda"), "counts": None}
        grad = torch.zeros(grid.n_alloc, plx.GRAD_STRIDE, device="cuda")
        loss = torch.empty(2, device="cuda", dtype=torch.float64)

        def step(ev=None):
            grad.zero_()
            if ev:
                ev[0].record()
            plx.render_forward(grid, cams, o, out=fw)
            if ev:
                ev[1].record()
            plx.render_backward_grid(grid, cams, o, rgb_t, depth_t, fw["rgb"], fw["depth"],
                                     grad=grad, loss=loss)
            if ev:
                ev[2].record()

        for _ in range(W):
            step()
        barrier()
        E = [[torch.cuda.Event(enable_timing=True) for _ in range(5)] for _ in range(K)]
        for e in E:
            flush.fill_(1)
            e[3].record()
            step(e)
            e[4].record()
        barrier()
        step_ms = [e[3].elapsed_time(e[4]) for e in E]
        fwd_ms = [e[0].elapsed_time(e[1]) for e in E]
        bwd_ms = [e[1].elapsed_time(e[2]) for e in E]
        res = {"step_ms": step_ms, "fwd_ms": fwd_ms, "bwd_ms": bwd_ms,
               "loss": loss.cpu().tolist(), "launch_config": grid.get_config(),
               "tuning_trials": tuned["trials"] if tuned else None}
        if with_e2e:
            # End to end through the public API with host buffers: each step
            # copies its targets and poses from pinned host memory and reads
            # its loss back. Double-buffered: the copies of step i+1 run on a
            # copy stream while step i computes; the timed region spans all K
            # steps, from the first copy to the last loss read.
            rgb_h = torch.from_numpy(rgb_np).pin_memory()
            depth_h = torch.from_numpy(depth_np).pin_memory()
            poses_h = cams.poses.cpu().pin_memory()
            loss_h = torch.empty(2, dtype=torch.float64).pin_memory()
            rgb_d = [torch.empty_like(rgb_t) for _ in range(2)]
            depth_d = [torch.empty_like(depth_t) for _ in range(2)]
            cams_d = [plx.CameraSet(cams_np) for _ in range(2)]
            comp_s = torch.cuda.current_stream()
            copy_s = torch.cuda.Stream()
            ready = [torch.cuda.Event() for _ in range(2)]
            free = [torch.cuda.Event() for _ in range(2)]

            def prefetch(i):
                b = i % 2
                with torch.cuda.stream(copy_s):
                    copy_s.wait_event(free[b])
                    rgb_d[b].copy_(rgb_h, non_blocking=True)
                    depth_d[b].copy_(depth_h, non_blocking=True)
                    cams_d[b].poses.copy_(poses_h, non_blocking=True)
                    ready[b].record(copy_s)

            def compute(i):
                b = i % 2
                comp_s.wait_event(ready[b])
                flush.fill_(1)
                grad.zero_()
                plx.render_forward(grid, cams_d[b], o, out=fw)
                plx.render_backward_grid(grid, cams_d[b], o, rgb_d[b], depth_d[b], fw["rgb"],
                                         fw["depth"], grad=grad, loss=loss)
                free[b].record(comp_s)
                loss_h.copy_(loss, non_blocking=True)

            def run(n):
                for b in range(2):
                    free[b].record(comp_s)
                copy_s.wait_stream(comp_s)
                prefetch(0)
                for i in range(n):
                    if i + 1 < n:
                        prefetch(i + 1)
                    compute(i)

            run(W)
            barrier()
            t0, t1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            t0.record(comp_s)
            run(K)
            t1.record(comp_s)
            barrier()
            res["e2e_ms"] = [t0.elapsed_time(t1) / K] * K
            res["h2d"] = rgb_h.numel() * 4 + depth_h.numel() * 4 + poses_h.numel() * 8
            res["d2h"] = loss_h.numel() * 8
        # exact sample counts for the byte model, and the vertices the step
        # touched for the compulsory-traffic bound (untimed)
        res["kept"] = scache.counts().cpu().numpy().copy() if scache is not None else None
        res["cache"] = ({"cap": scache.cap, "bytes": plx.sample_cache_bytes(n_rays, scache.cap)}
                        if scache is not None else None)
        cnt = plx.render_forward(grid, cams, o_plain, counts=True)["counts"].cpu().numpy()
        res["counts"] = cnt
        res["touched"] = int((grad[:, :28] != 0).any(1).sum())
        grid.close()
        del scache
        return res

    K, W = args.steps, args.warmup
    dev_id = torch.cuda.current_device()
    try:
        smi_id = "GPU-" + str(torch.cuda.get_device_properties(dev_id).uuid)
    except Exception:
        smi_id = str(dev_id)
    with ClockSampler(smi_id) as clk:
        main = measure(args.storage, K, W, with_e2e=True)
        other_storage = "bf16" if args.storage == "f32" else "f32"
        other = measure(other_storage, K, W, with_e2e=False)
        # the workload's other form: the adjoint recomputes every ray (no
        # per-sample state kept between the passes, only each ray's
        # compositing range)
        recomp = (measure(args.storage, K, W, with_e2e=False, cache_mode="off", ray_range=True)
                  if main["cache"] else None)
    clocks = clk.summary()

    # whole-job numbers: max over ranks
    t_main = rank_max(sum(main["step_ms"]), world, "cuda")
    t_e2e = rank_max(sum(main["e2e_ms"]), world, "cuda")
    t_other = rank_max(sum(other["step_ms"]), world, "cuda")
    rays_job = n_rays * world * K
    value = rays_job / (t_main / 1e3)

    # byte model of the dominant kernel (grid backward) and of the step
    valid = np.isfinite(depth_np) & (depth_np > 0)
    hbm, peak_kind = peaks()

    # the method's fixed no-reuse byte model (every pass gathers what it uses),
    # and beside it the same model for the algorithm as run (with the sample
    # cache the adjoint streams the kept samples instead of re-gathering)
    cap_main = main["cache"]["cap"] if main["cache"] else 0
    fwd_b, bwd_b, s_all, s_occ = bytes_model(main["counts"], args.storage, valid)
    fwd_i, bwd_i, _, _ = bytes_model(main["counts"], args.storage, valid, main["kept"], cap_main)
    fwd_ms, bwd_ms = statistics.mean(main["fwd_ms"]), statistics.mean(main["bwd_ms"])
    # the adjoint launch that does the work: the sample-cache kernel (its
    # re-marching partner only takes overflowing rays) or the re-march
    bwd_name = "backward_grid_cached" if main["cache"] else "backward_grid"
    dom = bwd_name if bwd_ms >= fwd_ms else "forward"
    dom_b, dom_ms = (bwd_b, bwd_ms) if dom == bwd_name else (fwd_b, fwd_ms)
    dom_i = bwd_i if dom == bwd_name else fwd_i
    achieved = dom_b / (dom_ms / 1e3) / 1e9
    step_roof = (fwd_b + bwd_b) / (hbm * 1e9) * 1e3   # ms per step at the HBM roof
    fo_b, bo_b, _, _ = bytes_model(other["counts"], other_storage, valid)

    # compulsory traffic of the dominant kernel, the bytes it cannot avoid:
    # every touched vertex's FP32 gradient row (28 values) read and written
    # once and its link read once; without a sample cache also its record
    # read once; with one, the kept samples (20 B each) and the per-ray counts
    # read once; per valid ray its targets and the forward's C and D
    rec_b = 128 if args.storage == "f32" else 64
    n_valid = int(valid.sum())
    kept_fit = 0.0
    if main["kept"] is not None:
        k = main["kept"].astype(np.float64)
        kept_fit = float(k[valid & (main["kept"] <= cap_main)].sum())
    compulsory = (main["touched"] * (2 * 112 + 4) + 32.0 * n_valid
                  + (kept_fit * 20.0 + 4.0 * n_rays if main["cache"] else main["touched"] * rec_b))
    ceil = l2_ceilings()
    roofline = roofline_block(
        dom, "room256", args.storage, n_rays, dom_ms, ceil, compulsory, dom_b,
        "compulsory bytes: per touched vertex 2 x 112 B of FP32 gradient read-modify-write "
        "and 4 B of link; with the sample cache 20 B per kept sample and 4 B per ray, without "
        "it the vertex record once; 32 B per valid ray (targets, forward's C and D)", clocks)
    fwd_comp = main["touched"] * (rec_b + 4) + 20.0 * kept_fit + 20.0 * n_rays
    fwd_block = roofline_block(
        "forward", "room256", args.storage, n_rays, fwd_ms, ceil, fwd_comp, fwd_b,
        "compulsory bytes: per touched vertex its record and link once; with the sample "
        "cache 20 B per kept sample written; 20 B of outputs per ray", clocks)
    roofline.update({
        "as_run_no_reuse_frac": dom_i / (dom_ms / 1e3) / 1e9 / hbm,
        "step_no_reuse_frac": step_roof / (t_main / K),
        "S_all_mean": s_all, "S_occ_mean": s_occ, "touched_vertices": main["touched"],
        "forward": {k: fwd_block[k] for k in ("bound", "achieved", "peak", "unit", "frac",
                                              "ms_per_launch", "traffic", "l2", "issue", "hbm")
                    if k in fwd_block},
    })
    line = {
        "metric": METRIC, "value": value, "unit": "rays/s", "n_gpus": world, "steps": K,
        "warmup": W, "ms_per_step": t_main / K, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": dict(workload_config(sc, cams_np, args.storage),
                       parallelism=f"replicated grid, keyframes sharded over {world} rank(s)",
                       sample_cache=cache_note(main, n_rays)),
        "roofline": roofline,
        "e2e": {"value": rays_job / (t_e2e / 1e3), "unit": "rays/s",
                "h2d_bytes_per_step": main["h2d"], "d2h_bytes_per_step": main["d2h"],
                "timing": "K steps as one region (first copy to last loss read); copies of "
                          "step i+1 overlap step i on a second stream; L2 flushed per step "
                          "inside the region"},
        "gpu_launches": K * (4 if main["cache"] else 3),
        "clocks": clocks,
        other_storage: {"value": rays_job / (t_other / 1e3), "unit": "rays/s",
                        "ms_per_step": t_other / K,
                        "step_frac": (fo_b + bo_b) / (hbm * 1e9) * 1e3 / (t_other / K)},
        "recompute": None if recomp is None else {
            "value": rays_job / (rank_max(sum(recomp["step_ms"]), world, "cuda") / 1e3),
            "unit": "rays/s", "storage": args.storage,
            "ms_per_step": rank_max(sum(recomp["step_ms"]), world, "cuda") / K,
            "kernels_ms": {"forward": statistics.mean(recomp["fwd_ms"]),
                           "backward_grid": statistics.mean(recomp["bwd_ms"])},
            "launch_config": recomp["launch_config"],
            "note": "the same step without the sample cache: the adjoint re-marches every ray "
                    "over its compositing range (the forward keeps 8 bytes per ray: its first "
                    "and one past its last sample with sigma > 0), recomputing T_i and the "
                    "prefix sums; the headline keeps "
                    f"{main['cache']['bytes'] / 1e9:.2f} GB of kept samples instead"},
        "loss": main["loss"],
        "kernels_ms": {"forward": fwd_ms, "backward_grid": bwd_ms},
        "launch_config": {"autotuned": not args.no_tune, args.storage: main["launch_config"],
                          other_storage: other["launch_config"]},
        "tuning_trials": main["tuning_trials"],
        "kernel_source_sha": kernel_source_sha(),
    }
    if not args.no_small:
        line["small"] = run_small_bench(args, barrier)
    if not args.no_tracking:
        line["tracking"] = run_tracking(args, world, rank, barrier, clocks)
    if not args.no_batch:
        line["batched"] = run_batch_bench(args, barrier)
    if not args.no_large:
        line["large"] = run_large_bench(args, barrier)
    if not args.no_pipeline:
        from paper_2307_03404_b300 import pipeline

        # warm-up: a short sequence first, so first-call costs stay out of the timings
        pipeline.run(sc, n_frames=40, span=0.04, map_cfg=pipeline.MapConfig(iters=50),
                     track_cfg=pipeline.TrackConfig(iters=10))
        t = time.time()
        pl = pipeline.run(sc, log=log,
                          extra_track_cfgs=[pipeline.TrackConfig(method="lm", lm_iters=10)])
        pl["wall_seconds"] = time.time() - t
        pl["workload"] = ("room256 geometry, 300-frame 640x480 sequence (path_m long), every 10th and the last "
                          "frame mapped into a dynamic 256^3 grid grown from depth, every frame "
                          "tracked (Adam, 200 iterations of 4096 random rays, one CUDA graph; again with "
                          "10 Levenberg-Marquardt iterations on whole frames)")
        pl["scope"] = "one GPU (under torchrun every rank runs it; rank 0's numbers)"
        line["pipeline"] = pl
    if not args.no_cpu and rank == 0:
        line["cpu_baseline"] = cpu_baseline(sc, cams_np, rgb_np, depth_np, opts, args.cpu_seconds)
    if rank == 0:
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()


def run_tracking(args, world, rank, barrier, clk=None):
    """Tracking iterations/s: 100 GN iterations in one CUDA graph (``clk``:
    the clocks sampled during the mapping leg, for the issue roofline)."""
    import torch

    from paper_2307_03404_b300 import plx, scenes
    from paper_2307_03404_b300.trajectory import pose_error

    R, occ, npr, seed = scenes.WORKLOADS[args.tracking_workload]
    t = time.time()
    sc = scenes.workload_scene(args.tracking_workload)
    cam = scenes.room_cameras(sc, 1, seed + 1 + rank)[0]
    log(f"[bench] {args.tracking_workload} tracking scene in {time.time() - t:.1f}s")
    opts = dict(step=0.5 * float(sc.grid.h[0]), lambda_d=1.0, depth_is_z=False)
    o = plx.opts_from_dict(opts)
    T0 = scenes.perturb_pose(cam.T_wc, 0.03, 2.0, np.random.default_rng(seed + 5))
    iters = args.tracking_iters
    out = {"workload": f"{args.tracking_workload}: {R}^3 grid, {sc.grid.n_alloc} allocated, "
                       f"opaque surfaces with a 10 cm texture, one 640x480 frame, {iters} "
                       "Gauss-Newton iterations per CUDA graph, targets rendered at the true "
                       "pose, start perturbed 3 cm / 2 deg",
           "unit": "iters/s"}
    ceil = l2_ceilings()
    o_exact = o
    for storage, method, stop in (("f32", "lm", 0.0), ("bf16", "lm", 0.0), ("f32", "gn", 0.0),
                                  ("f32", "lm", 1e-4)):
        # stop > 0: rays stop once their transmittance falls below it (the
        # targets are rendered the same way); in the opaque room that is just
        # behind the first surface
        o = plx.opts_from_dict(dict(opts, stop_T=stop)) if stop > 0 else o_exact
        grid = plx.Grid.from_scene(sc.grid, storage)
        cams = plx.CameraSet([cam])
        tg = plx.render_forward(grid, cams, o)       # targets at the true pose
        rgb_t, depth_t = tg["rgb"].clone(), tg["depth"].clone()
        if not args.no_tune:
            from paper_2307_03404_b300 import autotune

            cams.poses.copy_(torch.tensor(T0.reshape(1, 12), device="cuda"))
            autotune.tune_tracking(grid, cams, 0, o, rgb_t, depth_t, reps=3,
                                   cache=os.path.join("/tmp", f"plx_tuning_{os.getpid()}.json"))
        cams.poses.copy_(torch.tensor(T0.reshape(1, 12), device="cuda"))
        start = cams.poses.clone()
        H = torch.empty(6, 6, device="cuda", dtype=torch.float64)
        b = torch.empty(6, device="cuda", dtype=torch.float64)
        loss = torch.empty(2, device="cuda", dtype=torch.float64)
        lm = plx.lm_state()
        pose = cams.poses[0]

        def one_iteration():
            plx.render_backward_pose(grid, cams, 0, o, rgb_t, depth_t, out=(H, b, loss))
            if method == "lm":
                plx.pose_step_lm(H, b, loss, lm, pose)
            else:
                plx.pose_step(H, b, pose)

        one_iteration()
        torch.cuda.synchronize()
        s = torch.cuda.Stream()
        s.wait_stream(torch.cuda.current_stream())
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g, stream=s):
            for _ in range(iters):
                one_iteration()
        for _ in range(args.warmup):
            cams.poses.copy_(start)
            lm.zero_()
            g.replay()
        barrier()
        evs = []
        for _ in range(max(1, args.steps // 2)):
            cams.poses.copy_(start)
            lm.zero_()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            g.replay()
            e1.record()
            evs.append((e0, e1))
        barrier()
        ms = [a.elapsed_time(b_) for a, b_ in evs]
        T = pose.cpu().numpy().reshape(3, 4)
        ms_it = sum(ms) / len(ms) / iters
        # the fixed no-reuse model of one iteration at the start pose (untimed):
        # 32 B of links per marched sample, one gather per sample with an
        # allocated corner, 16 B of targets per ray
        pose_now = cams.poses.clone()
        cams.poses.copy_(start)
        cnt = plx.render_forward(grid, cams, o, counts=True)["counts"].cpu().numpy()
        cams.poses.copy_(pose_now)
        rec = 896.0 if storage == "f32" else 448.0
        it_bytes = float((cnt[:, 0] * 32.0 + cnt[:, 1] * rec).sum() + 16.0 * cnt.shape[0])
        # the vertices the frame's rays composite with (untimed: nonzero rows
        # of the grid adjoint at the start pose)
        gfw = plx.render_forward(grid, cams, o)
        gr, _ = plx.render_backward_grid(grid, cams, o, rgb_t, depth_t, gfw["rgb"], gfw["depth"])
        touched = int((gr[:, :28] != 0).any(1).sum())
        del gr, gfw
        compulsory = touched * (rec / 7.0 + 4.0) + 16.0 * cnt.shape[0]
        res = {"value": iters * len(ms) / (sum(ms) / 1e3),
               "ms_per_iter": ms_it,
               "roofline": roofline_block(
                   "backward_pose", args.tracking_workload, storage, cnt.shape[0], ms_it, ceil,
                   compulsory, it_bytes,
                   "compulsory bytes: each vertex the frame's rays composite with read once "
                   "(its 128 B FP32 / 64 B 16-bit record) with its 4 B link, 16 B of targets "
                   "per ray", clk),
               "step": ("Gauss-Newton with Marquardt damping, accept/reject on the loss "
                        "(plx_pose_step_lm)" if method == "lm" else
                        "undamped Gauss-Newton (plx_pose_step)"),
               "launch_config": grid.get_config(),
               "start_err_cm_deg": list(pose_error(T0, cam.T_wc)),
               "final_err_cm_deg": list(pose_error(T, cam.T_wc)),
               "final_loss": float(loss[0].item())}
        if stop > 0:
            res["stop_T"] = stop
            res["note"] = ("rays stop once T < stop_T (targets rendered the same way): every "
                           "rendered value within stop_T x max |colour| of the exact render; "
                           "compare ms_per_iter with f32")
            out["f32_stop_T"] = res
        else:
            out[storage if method == "lm" else "gn_undamped_f32"] = res
        grid.close()
    o = o_exact  # the exact options again (the loop above ended on the early-stop variant)
    # the paper's tracker (Sec. 5.4): Adam on random rays of the frame
    n_rays, lr, aiters = args.adam_rays, args.adam_lr, args.adam_iters
    for storage in ("f32", "bf16"):
        grid = plx.Grid.from_scene(sc.grid, storage)
        cams = plx.CameraSet([cam])
        tg = plx.render_forward(grid, cams, o)
        rgb_t, depth_t = tg["rgb"].clone(), tg["depth"].clone()
        start = torch.tensor(T0.reshape(1, 12), device="cuda")
        cams.poses.copy_(start)
        state = plx.adam_state()
        buf = (torch.empty(6, 6, device="cuda", dtype=torch.float64),
               torch.empty(6, device="cuda", dtype=torch.float64),
               torch.empty(2, device="cuda", dtype=torch.float64))
        plx.track_adam_step(grid, cams, 0, o, n_rays, 3, rgb_t, depth_t, state, lr, out=buf)
        torch.cuda.synchronize()
        s = torch.cuda.Stream()
        s.wait_stream(torch.cuda.current_stream())
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g, stream=s):
            for _ in range(aiters):
                plx.track_adam_step(grid, cams, 0, o, n_rays, 3, rgb_t, depth_t, state, lr, out=buf)
        for _ in range(args.warmup):
            cams.poses.copy_(start)
            state.zero_()
            g.replay()
        barrier()
        evs = []
        for _ in range(max(1, args.steps // 2)):
            cams.poses.copy_(start)
            state.zero_()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            g.replay()
            e1.record()
            evs.append((e0, e1))
        barrier()
        ms = [a.elapsed_time(b_) for a, b_ in evs]
        T = cams.poses[0].cpu().numpy().reshape(3, 4)
        out.setdefault("adam", {"rays_per_iter": n_rays, "lr": lr, "iters_per_frame": aiters,
                                "sampler": "SplitMix64 over the frame's pixels"})
        out["adam"][storage] = {
            "value": aiters * len(ms) / (sum(ms) / 1e3), "unit": "iters/s",
            "ms_per_frame": sum(ms) / len(ms),
            "start_err_cm_deg": list(pose_error(T0, cam.T_wc)),
            "final_err_cm_deg": list(pose_error(T, cam.T_wc)),
            "final_loss": float(buf[2][0].item())}
        grid.close()
    out["value"] = out["f32"]["value"]
    out["roofline"] = out["f32"]["roofline"]
    return out


def run_small_bench(args, barrier):
    """The small plain-FP32 workload: the dense 64^3 sphere grid, one 64x48
    frame (3,072 rays), targets rendered on the GPU from the perturbed copy of
    the grid. One step = forward + RGB-D loss + grid adjoint (re-marching, no
    sample cache) + pose Jacobian with its FP64 reduction, back to back on one
    stream. Its 29 MB grid sits in L2; the step is launch- and latency-bound
    at this size (a few microseconds per kernel)."""
    import torch

    from paper_2307_03404_b300 import plx, scenes

    g, cam, gp = scenes.sphere_scene()
    opts = plx.opts_from_dict(dict(step=0.5 * float(g.h[0]), lambda_d=1.0, depth_is_z=False))
    cams = plx.CameraSet([cam])
    tgrid = plx.Grid.from_scene(gp, "f32")
    tg = plx.render_forward(tgrid, cams, opts)
    rgb_t, depth_t = tg["rgb"].clone(), tg["depth"].clone()
    tgrid.close()
    grid = plx.Grid.from_scene(g, "f32")
    n_rays = cam.width * cam.height
    fw = plx.render_forward(grid, cams, opts)
    grad = torch.zeros(grid.n_alloc, plx.GRAD_STRIDE, device="cuda")
    loss = torch.empty(2, device="cuda", dtype=torch.float64)
    pose_out = (torch.empty(6, 6, device="cuda", dtype=torch.float64),
                torch.empty(6, device="cuda", dtype=torch.float64),
                torch.empty(2, device="cuda", dtype=torch.float64))

    def step():
        grad.zero_()
        plx.render_forward(grid, cams, opts, out=fw)
        plx.render_backward_grid(grid, cams, opts, rgb_t, depth_t, fw["rgb"], fw["depth"],
                                 grad=grad, loss=loss)
        plx.render_backward_pose(grid, cams, 0, opts, rgb_t, depth_t, out=pose_out)

    K = max(20, 10 * args.steps)

    def timed():
        for _ in range(max(3, args.warmup)):
            step()
        barrier()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(K):
            step()
        e1.record()
        barrier()
        return e0.elapsed_time(e1) / K

    ms = timed()  # default launch choices: a warp per ray at this size
    config = grid.get_config()
    grid.set_config(seg_rays=0)  # the same step with one ray per lane
    ms_lane = timed()
    grid.set_config(seg_rays=config["seg_rays"])
    cnt = plx.render_forward(grid, cams, opts, counts=True)["counts"].cpu().numpy()
    grid.close()
    return {"workload": "sphere64: dense 64^3 grid (262,144 vertices, FP32), one 64x48 frame "
                        "(3,072 rays); forward + loss + grid adjoint + pose Jacobian per step",
            "value": n_rays / (ms / 1e3), "unit": "rays/s", "ms_per_step": ms, "steps": K,
            "S_all_mean": float(cnt[:, 0].mean()), "S_occ_mean": float(cnt[:, 1].mean()),
            "loss": loss.cpu().tolist(), "gpu_launches_per_step": 4,
            "launch_config": config,
            "one_ray_per_lane": {"value": n_rays / (ms_lane / 1e3), "ms_per_step": ms_lane,
                                 "launch": "seg_rays = 0: each lane marches a whole ray"},
            "timing": "K steps back to back between two CUDA events; the grid stays in L2"}


def run_batch_bench(args, barrier):
    """64 frames of mixed sizes (32 mapping, 32 tracking) on a 512^3 grid in one
    persistent launch, against the same work through the separate calls."""
    import torch

    from paper_2307_03404_b300 import plx, scenes

    torch.cuda.empty_cache()
    R, occ, npr, seed = scenes.WORKLOADS["room512mix"]
    t = time.time()
    sc = scenes.room_scene(R, occ, npr, seed)
    cams_np = scenes.mixed_resolution_cameras(sc, 64, seed + 1)
    rgb_np, depth_np = scenes.sensor_frames(sc, cams_np, seed + 2)
    log(f"[bench] room512mix scene + 64 frames in {time.time() - t:.1f}s")
    work = [(i, plx.WORK_MAP if i % 2 == 0 else plx.WORK_TRACK) for i in range(64)]
    sizes = [c.width * c.height for c in cams_np]
    offs = np.cumsum([0] + sizes)
    rows = int(offs[-1])
    o = plx.opts_from_dict(dict(step=0.5 * float(sc.grid.h[0]), lambda_d=1.0, depth_is_z=True))
    cams = plx.CameraSet(cams_np)
    rgb_t = torch.from_numpy(rgb_np).cuda()
    depth_t = torch.from_numpy(depth_np).cuda()
    mi = [i for i, (_, m) in enumerate(work) if m == plx.WORK_MAP]
    ti = [i for i, (_, m) in enumerate(work) if m == plx.WORK_TRACK]
    mrows = torch.from_numpy(np.concatenate([np.arange(offs[i], offs[i + 1]) for i in mi])).cuda()
    map_cams = plx.CameraSet([cams_np[i] for i in mi])
    trk_cams = plx.CameraSet([cams_np[i] for i in ti])
    rgb_m, depth_m = rgb_t[mrows].contiguous(), depth_t[mrows].contiguous()
    trk = [(rgb_t[offs[i]:offs[i + 1]], depth_t[offs[i]:offs[i + 1]]) for i in ti]
    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")
    out = {"workload": f"room512mix: 512^3 grid, {sc.grid.n_alloc} allocated, 64 frames drawn "
                       f"from 320x240/640x480/848x480/1200x680 ({rows} rays), 32 mapped "
                       "(forward + adjoint) and 32 tracked (pose Jacobian) in one launch",
           "unit": "rays/s"}

    def timed(fn, K, W):
        for _ in range(W):
            fn()
        barrier()
        ev = []
        for _ in range(K):
            flush.fill_(1)
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record()
            fn()
            b.record()
            ev.append((a, b))
        barrier()
        return sum(x.elapsed_time(y) for x, y in ev) / K

    for storage in ("bf16", "f32"):
        grid = plx.Grid.from_scene(sc.grid, storage)
        # sample caches (untimed set-up): per mapping ray for the separate
        # calls, per thread slot for the batched launch, K from a probe forward
        om = ob = o
        sep_cache = bat_cache = None  # the other storage's caches go first
        torch.cuda.empty_cache()
        cache_note_b = "off"
        if args.sample_cache != "off":
            sep_cache = plx.SampleCache.sized_for(grid, map_cams, o)
            bat_cache = plx.SampleCache.for_batch(sep_cache.cap)
            om, ob = sep_cache.opts(o), bat_cache.opts(o)
            cache_note_b = (f"K = {sep_cache.cap}: the batched launch keeps a ray's samples in its "
                            f"thread's row ({bat_cache.n_rays} rows, "
                            f"{plx.sample_cache_bytes(bat_cache.n_rays, bat_cache.cap) / 1e9:.2f} GB); "
                            f"the separate calls per mapping ray "
                            f"({plx.sample_cache_bytes(sep_cache.n_rays, sep_cache.cap) / 1e9:.1f} GB)")
        if not args.no_tune:
            from paper_2307_03404_b300 import autotune

            autotune.tune_batch(grid, cams, work, ob, rgb_t, depth_t, reps=2,
                                cache=os.path.join("/tmp", f"plx_tuning_{os.getpid()}.json"))
        grad = torch.zeros(grid.n_alloc, plx.GRAD_STRIDE, device="cuda")
        mloss = torch.empty(2, device="cuda", dtype=torch.float64)
        bo = (torch.empty(32, 6, 6, device="cuda", dtype=torch.float64),
              torch.empty(32, 6, device="cuda", dtype=torch.float64),
              torch.empty(32, 2, device="cuda", dtype=torch.float64))

        def batch():
            grad.zero_()
            plx.render_batch(grid, cams, work, ob, rgb_t, depth_t, grad=grad, map_loss=mloss,
                             out=bo)

        fw = plx.render_forward(grid, map_cams, om)
        po = (torch.empty(6, 6, device="cuda", dtype=torch.float64),
              torch.empty(6, device="cuda", dtype=torch.float64),
              torch.empty(2, device="cuda", dtype=torch.float64))

        def separate():
            grad.zero_()
            plx.render_forward(grid, map_cams, om, out=fw)
            plx.render_backward_grid(grid, map_cams, om, rgb_m, depth_m, fw["rgb"], fw["depth"],
                                     grad=grad, loss=mloss)
            for k, (r_, d_) in enumerate(trk):
                plx.render_backward_pose(grid, trk_cams, k, o, r_, d_, out=po)

        ms_b = timed(batch, max(2, args.steps // 2), args.warmup)
        ms_s = timed(separate, max(2, args.steps // 2), args.warmup)
        out[storage] = {"value": rows / (ms_b / 1e3), "ms_per_batch": ms_b,
                        "launch_config": grid.get_config(), "sample_cache": cache_note_b,
                        "separate_calls": {"value": rows / (ms_s / 1e3), "ms": ms_s,
                                           "launches": (4 if om is not o else 3) + 32}}
        # the mapping optimiser on this grid (Sec. 5.4 RMSProp, one pass over
        # all records, gradients and state): a plain streaming kernel, timed
        # against the copy bandwidth
        state = torch.zeros_like(grad)
        n = grid.n_alloc
        rec_r, rec_w = (112, 112) if storage == "f32" else (64, 64)
        per_vertex = 112 + 112 + rec_r + 112 + 112 + rec_w  # grad, state r+w, record, zeroed grad

        def rms():
            plx.grid_rmsprop(grid, grad, state, 1e-3, lr_density=1e-2, zero_grad=True)

        ms_r = timed(rms, max(3, args.steps), args.warmup)
        hbm, peak_kind = peaks()
        gbs = n * per_vertex / (ms_r / 1e3) / 1e9
        out[storage]["rmsprop"] = {
            "vertices": n, "ms": ms_r, "bytes_per_vertex": per_vertex, "achieved_gbs": gbs,
            "peak_gbs": hbm, "frac": gbs / hbm, "peak_kind": f"{peak_kind} copy bandwidth"}
        grid.close()
    out["value"] = out["bf16"]["value"]
    return out


def run_large_bench(args, barrier):
    """The large mapping workload: a 1024^3 multi-room house (~2% allocated),
    BF16 storage, 16 keyframes of 1200x680 (f = 600), step 0.5 voxel, up to
    2048 samples per ray; one step = forward + adjoint over all 13 M rays,
    per-ray transmittance recomputed in the adjoint (only C, D, the final T
    and the compositing range of each ray are kept between the two
    launches)."""
    import torch

    from paper_2307_03404_b300 import plx, scenes

    torch.cuda.empty_cache()  # what earlier legs left cached goes back to the device
    R, occ, npr, seed = scenes.WORKLOADS["house1024"]
    t = time.time()
    sc = scenes.house_scene(R, occ, npr, seed, device="cuda")
    cams_np = scenes.house_cameras(sc, 16, seed + 1, 1200, 680, 600.0)
    rgb_t, depth_t = scenes.sensor_frames_torch(sc, cams_np, seed + 2, device="cuda")
    log(f"[bench] house1024 scene ({sc.grid.n_alloc} allocated) + 16 frames in "
        f"{time.time() - t:.1f}s")
    storage = "bf16"
    o = plx.opts_from_dict(dict(step=0.5 * float(sc.grid.h[0]), lambda_d=1.0, depth_is_z=True,
                                max_samples=2048))
    cams = plx.CameraSet(cams_np)
    n_rays = int(rgb_t.shape[0])
    grid = plx.Grid.from_scene(sc.grid, storage)
    n_alloc = grid.n_alloc
    del sc
    grad = torch.zeros(n_alloc, plx.GRAD_STRIDE, device="cuda")
    loss = torch.empty(2, device="cuda", dtype=torch.float64)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")
    tune_file = os.path.join("/tmp", f"plx_tuning_{os.getpid()}.json")
    K = max(2, args.steps // 2)

    def measure(oo):
        """Autotune (unless off), then K timed forward + adjoint steps."""
        tuned = None
        if not args.no_tune:
            from paper_2307_03404_b300 import autotune

            tuned = autotune.tune_mapping(grid, cams, oo, rgb_t, depth_t, reps=1, cache=tune_file)
        fw = plx.render_forward(grid, cams, oo)

        def step(ev):
            grad.zero_()
            ev[0].record()
            plx.render_forward(grid, cams, oo, out=fw)
            ev[1].record()
            plx.render_backward_grid(grid, cams, oo, rgb_t, depth_t, fw["rgb"], fw["depth"],
                                     grad=grad, loss=loss)
            ev[2].record()

        for _ in range(args.warmup):
            step([torch.cuda.Event(enable_timing=True) for _ in range(3)])
        barrier()
        E = [[torch.cuda.Event(enable_timing=True) for _ in range(3)] for _ in range(K)]
        for e in E:
            flush.fill_(1)
            step(e)
        barrier()
        del fw
        return (statistics.mean(e[0].elapsed_time(e[1]) for e in E),
                statistics.mean(e[1].elapsed_time(e[2]) for e in E), tuned)

    # the workload as defined: the adjoint recomputes every ray (per ray only
    # C, D, the final T and the compositing range are kept between the
    # launches: the gradient checkpointing of per-ray state)
    fwd_ms, bwd_ms, tuned = measure(plx.RayRange(n_rays).opts(o))
    step_ms = fwd_ms + bwd_ms
    loss_main = loss.cpu().tolist()
    config_main = grid.get_config()
    touched = int((grad[:, :28] != 0).any(1).sum())
    counts = plx.render_forward(grid, cams, o, counts=True)["counts"].cpu().numpy()
    d = depth_t.cpu().numpy()
    valid = np.isfinite(d) & (d > 0)
    fwd_b, bwd_b, s_all, s_occ = bytes_model(counts, storage, valid)
    hbm, peak_kind = peaks()
    compulsory = touched * (64 + 2 * 112 + 4) + 32.0 * int(valid.sum())
    roof = roofline_block(
        "backward_grid", "house1024", storage, n_rays, bwd_ms, l2_ceilings(), compulsory, bwd_b,
        "compulsory bytes: per touched vertex its 64 B record once, 2 x 112 B of FP32 gradient "
        "read-modify-write and 4 B of link; 32 B per valid ray")
    roof.update({"step_no_reuse_frac": (fwd_b + bwd_b) / (hbm * 1e9) * 1e3 / step_ms,
                 "S_all_mean": s_all, "S_occ_mean": s_occ, "touched_vertices": touched})
    out = {"workload": f"house1024: 1024^3 grid, {n_alloc} allocated "
                       f"({n_alloc / 1024 ** 3:.2%}), {storage} storage, 16 x 1200x680 keyframes "
                       f"({n_rays} rays), step 0.5 voxel, <= 2048 samples per ray; the adjoint "
                       "recomputes each ray's state over its compositing range (per ray 8 bytes "
                       "kept: first and one past the last sample with sigma > 0; no per-sample "
                       "state)",
           "value": n_rays / (step_ms / 1e3), "unit": "rays/s", "ms_per_step": step_ms,
           "kernels_ms": {"forward": fwd_ms, "backward_grid": bwd_ms},
           "roofline": roof,
           "loss": loss_main, "launch_config": config_main,
           "autotuned": tuned is not None, "steps": K,
           "scope": "one GPU (under torchrun every rank runs it; rank 0's numbers)"}
    # beside it, the full re-march (no per-ray range)
    ff, fb, _ = measure(o)
    out["full_remarch"] = {"value": n_rays / ((ff + fb) / 1e3), "unit": "rays/s",
                           "ms_per_step": ff + fb, "kernels_ms": {"forward": ff, "backward_grid": fb},
                           "note": "the adjoint re-marches every ray from its first sample"}
    if args.sample_cache != "off":
        # beside it, the same steps with the forward's compositing samples kept
        # for the adjoint (tens of GB of per-sample state in HBM)
        scache = (plx.SampleCache.sized_for(grid, cams, o) if args.sample_cache == "fit"
                  else plx.SampleCache(n_rays, int(args.sample_cache)))
        fc, bc, _ = measure(scache.opts(o))
        kept = scache.counts().cpu().numpy().copy()
        cache_res = {"cap": scache.cap, "bytes": plx.sample_cache_bytes(n_rays, scache.cap)}
        del scache
        _, bwd_i, _, _ = bytes_model(counts, storage, valid, kept, cache_res["cap"])
        out["with_sample_cache"] = {
            "value": n_rays / ((fc + bc) / 1e3), "unit": "rays/s", "ms_per_step": fc + bc,
            "kernels_ms": {"forward": fc, "backward_grid": bc},
            "sample_cache": cache_note({"cache": cache_res, "kept": kept}, n_rays),
            "no_reuse_frac": bwd_b / (bc / 1e3) / 1e9 / hbm,
            "as_run_no_reuse_frac": bwd_i / (bc / 1e3) / 1e9 / hbm,
            "launch_config": grid.get_config()}
    grid.close()
    return out


# ---------------------------------------------------------- CPU baselines
def cpu_baseline(sc, cams, rgb_np, depth_np, opts, seconds):
    """The FP64 oracle (as it stands) on seeded chunks of 2048 of the workload's
    rays, repeated until ``seconds`` of wall time have passed."""
    import oracle
    from oracle import build as obuild

    from paper_2307_03404_b300 import scenes

    obuild.build()
    cores = os.cpu_count() or 1
    oracle.set_threads(cores)
    offs = np.cumsum([0] + [c.width * c.height for c in cams])[:-1]
    done, t0, i = 0, time.time(), 0
    while time.time() - t0 < seconds:
        cid, pix = scenes.random_rays(cams, 2048, 12345 + i)
        rows = offs[cid] + pix
        oracle.grad_grid(sc.grid, cams, opts, rgb_np[rows], depth_np[rows], rays=(cid, pix))
        done += 2048
        i += 1
    dt = time.time() - t0
    # one thread, one chunk of 1024 rays
    oracle.set_threads(1)
    cid, pix = scenes.random_rays(cams, 1024, 999)
    rows = offs[cid] + pix
    t1 = time.time()
    oracle.grad_grid(sc.grid, cams, opts, rgb_np[rows], depth_np[rows], rays=(cid, pix))
    dt1 = time.time() - t1
    oracle.set_threads(cores)
    return {"value": done / dt, "unit": "rays/s", "cores": cores, "kind": "oracle",
            "sample": f"{done} seeded random rays of the same 8 keyframes in chunks of 2048 "
                      f"(forward + loss + grid gradient, FP64, OpenMP over rays), {dt:.1f} s",
            "single_thread": {"value": 1024 / dt1, "unit": "rays/s", "cores": 1,
                              "sample": f"1024 seeded random rays, {dt1:.1f} s"}}


def run_reference(args):
    """--impl reference: the oracle timed on the host cores, same metric/config."""
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    import oracle
    from oracle import build as obuild

    from paper_2307_03404_b300 import scenes

    obuild.build()
    sc, cams, rgb_np, depth_np, opts = mapping_workload(1, 0)
    cores = os.cpu_count() or 1
    oracle.set_threads(cores)
    n = args.cpu_rays_per_step
    offs = np.cumsum([0] + [c.width * c.height for c in cams])[:-1]

    def one(i):
        cid, pix = scenes.random_rays(cams, n, 777 + i)
        rows = offs[cid] + pix
        oracle.grad_grid(sc.grid, cams, opts, rgb_np[rows], depth_np[rows], rays=(cid, pix))

    for i in range(args.warmup):
        one(i)
    t = time.time()
    for i in range(args.steps):
        one(100 + i)
    dt = time.time() - t
    value = n * args.steps / dt
    line = {"metric": METRIC, "value": value, "unit": "rays/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": dt / args.steps * 1e3,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "impl": "reference",
            "config": dict(workload_config(sc, cams, "f64"), parallelism="host cores",
                           l2="not applicable (host run)"),
            "cpu_baseline": {"value": value, "unit": "rays/s", "cores": cores, "kind": "oracle",
                             "sample": f"each step {n} seeded random rays of the workload"},
            "e2e": {"value": value, "unit": "rays/s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--storage", default="f32", choices=["f32", "bf16", "f16", "f32_bf16"])
    ap.add_argument("--tracking-workload", default="room512")
    ap.add_argument("--tracking-iters", type=int, default=100)
    ap.add_argument("--adam-rays", type=int, default=1024)
    ap.add_argument("--adam-lr", type=float, default=1e-3)
    ap.add_argument("--adam-iters", type=int, default=200)
    ap.add_argument("--no-tracking", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--no-batch", action="store_true")
    ap.add_argument("--no-tune", action="store_true")
    ap.add_argument("--no-large", action="store_true")
    ap.add_argument("--no-pipeline", action="store_true")
    ap.add_argument("--no-small", action="store_true")
    ap.add_argument("--map-frames", type=int, default=FRAMES_PER_RANK,
                    help="keyframes per rank of the mapping workload (8; fewer only for "
                         "profiler captures)")
    ap.add_argument("--sample-cache", default="fit",
                    help='"fit" (sized so no ray overflows), "off", or samples per ray')
    ap.add_argument("--cpu-seconds", type=float, default=12.0)
    ap.add_argument("--cpu-rays-per-step", type=int, default=4096)
    args = ap.parse_args()
    if args.warmup < 3:
        log("[bench] warmup raised to 3")
        args.warmup = 3
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
