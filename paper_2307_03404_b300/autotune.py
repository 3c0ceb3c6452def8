"""Autotuner of the launch choices of a grid's kernels.

The choices are those of ``plx_grid_set_config``: the granularity of the
empty-space map (blocks of 2^shift cells per axis), per ray kernel the
number of resident 256-thread blocks per SM it is compiled for (1 or 2: a
register budget of 255 or 128 per thread; the forward also 3, 80 registers),
and the rays per warp (one ray per lane, or a warp per ray up to
``seg_rays`` rays). None of them changes a result; they
trade occupancy against spills and skipping granularity against lookup cost,
and the best values depend on the grid and the rays, and on the options: with
options naming a sample cache, tune_mapping times the cached adjoint. The tuner times the
caller's own workload with CUDA events (coordinate descent, a few repetitions
per candidate) and keeps the winner in a JSON cache keyed by device and
workload, so later runs apply it without timing.
"""
from __future__ import annotations

import json
import os

import torch

from . import plx

SHIFTS = (2, 3, 4)
FINE_FORWARD, FINE_ADJOINT, FINE_POSE, FINE_BATCH = 1, 2, 4, 8


def _fine(bit):
    """Candidates of fine_skip that toggle one kernel's bit."""
    return lambda cur: [cur | bit, cur & ~bit]
BLOCKS = (1, 2)
FORWARD_BLOCKS = (1, 2, 3)
# rays per warp (seg_rays): one ray per lane (0), or a warp per ray for calls
# up to the default 16384 ray slots or up to 2^24; tried only for calls of at
# most SEG_TUNE_MAX rays, where a warp per ray can win (above, the 32 lanes of
# a warp splitting one ray cost more than they save)
SEG_RAYS = (0, 16384, 1 << 24)
SEG_TUNE_MAX = 1 << 16


def _cache_path(path=None):
    return path or os.environ.get("PLX_TUNING_CACHE") or os.path.join(
        os.path.expanduser("~"), ".cache", "plx_tuning.json")


def _key(grid, kind, n_rays):
    name = torch.cuda.get_device_name()
    return f"{name}|{kind}|res={'x'.join(map(str, grid.res))}|n={grid.n_alloc}|" \
           f"storage={grid.storage}|rays={n_rays}"


def _time(fn, reps):
    fn()
    torch.cuda.synchronize()
    best = float("inf")
    for _ in range(reps):
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record()
        fn()
        b.record()
        torch.cuda.synchronize()
        best = min(best, a.elapsed_time(b))
    return best


def _descend(grid, fn, fields, reps, log):
    """Coordinate descent over ``fields`` [(name, candidates)] from the
    grid's current choices; returns the best config and its time."""
    best_cfg = grid.get_config()
    best = _time(fn, reps)
    log.append((dict(best_cfg), best))
    for name, cands in fields:
        if callable(cands):
            cands = cands(best_cfg[name])
        for v in cands:
            if v == best_cfg[name]:
                continue
            grid.set_config(**{**best_cfg, name: v})
            t = _time(fn, reps)
            log.append((grid.get_config(), t))
            if t < best:
                best, best_cfg = t, grid.get_config()
        grid.set_config(**best_cfg)
    return best_cfg, best


def _lookup(grid, key, cache):
    p = _cache_path(cache)
    if os.path.exists(p):
        try:
            d = json.load(open(p))
        except (OSError, ValueError):
            d = {}
        if key in d:
            grid.set_config(**d[key]["config"])
            return d[key]
    return None


def _store(key, entry, cache):
    p = _cache_path(cache)
    d = {}
    if os.path.exists(p):
        try:
            d = json.load(open(p))
        except (OSError, ValueError):
            d = {}
    d[key] = entry
    os.makedirs(os.path.dirname(p), exist_ok=True)
    tmp = p + ".tmp"
    with open(tmp, "w") as f:
        json.dump(d, f, indent=1)
    os.replace(tmp, p)


def tune_mapping(grid, cams, opts, rgb_target, depth_target, rays=None, reps=3, cache=None,
                 use_cache=True):
    """Tune block_shift, fine_skip, forward_blocks and adjoint_blocks (and, for
    few rays without a sample cache, seg_rays) on one mapping step (forward +
    adjoint) of these rays. Returns dict(config, ms, trials)."""
    n = cams.n_pixels() if rays is None else int(rays[1].shape[0])
    # with a sample cache another adjoint kernel runs: its own entry
    key = _key(grid, "mapping+cache" if opts.sample_cap > 0 else "mapping", n)
    if use_cache:
        hit = _lookup(grid, key, cache)
        if hit:
            return dict(hit, cached=True)
    grad = torch.zeros(grid.n_alloc, plx.GRAD_STRIDE, device="cuda")
    loss = torch.empty(2, device="cuda", dtype=torch.float64)
    fw = plx.render_forward(grid, cams, opts, rays=rays)

    def step():
        plx.render_forward(grid, cams, opts, rays=rays, out=fw)
        plx.render_backward_grid(grid, cams, opts, rgb_target, depth_target, fw["rgb"],
                                 fw["depth"], rays=rays, grad=grad, loss=loss)

    log = []
    fields = [("block_shift", SHIFTS), ("fine_skip", _fine(FINE_FORWARD)),
              ("fine_skip", _fine(FINE_ADJOINT)), ("adjoint_blocks", BLOCKS),
              ("forward_blocks", FORWARD_BLOCKS)]
    if n <= SEG_TUNE_MAX and opts.sample_cap == 0:
        fields.insert(0, ("seg_rays", SEG_RAYS))
    cfg, ms = _descend(grid, step, fields, reps, log)
    entry = {"config": cfg, "ms": ms, "trials": [[c, t] for c, t in log]}
    _store(key, entry, cache)
    return dict(entry, cached=False)


def tune_tracking(grid, cams, cam, opts, rgb_target, depth_target, reps=3, cache=None,
                  use_cache=True):
    """Tune pose_blocks (and block_shift, fine_skip; seg_rays for few rays) on
    one pose-Jacobian launch."""
    n = cams.n_pixels(cam)
    key = _key(grid, "tracking", n)
    if use_cache:
        hit = _lookup(grid, key, cache)
        if hit:
            return dict(hit, cached=True)
    out = (torch.empty(6, 6, device="cuda", dtype=torch.float64),
           torch.empty(6, device="cuda", dtype=torch.float64),
           torch.empty(2, device="cuda", dtype=torch.float64))

    def step():
        plx.render_backward_pose(grid, cams, cam, opts, rgb_target, depth_target, out=out)

    log = []
    fields = [("pose_blocks", BLOCKS), ("block_shift", SHIFTS), ("fine_skip", _fine(FINE_POSE))]
    if n <= SEG_TUNE_MAX:
        fields.insert(0, ("seg_rays", SEG_RAYS))
    cfg, ms = _descend(grid, step, fields, reps, log)
    entry = {"config": cfg, "ms": ms, "trials": [[c, t] for c, t in log]}
    _store(key, entry, cache)
    return dict(entry, cached=False)


def tune_batch(grid, cams, work, opts, rgb_target, depth_target, reps=2, cache=None,
               use_cache=True):
    """Tune batch_blocks (and block_shift, fine_skip) on one batched launch."""
    n = sum(cams.n_pixels(c) for c, _ in work)
    key = _key(grid, f"batch{len(work)}", n)
    if use_cache:
        hit = _lookup(grid, key, cache)
        if hit:
            return dict(hit, cached=True)
    grad = torch.zeros(grid.n_alloc, plx.GRAD_STRIDE, device="cuda")

    def step():
        plx.render_batch(grid, cams, work, opts, rgb_target, depth_target, grad=grad)

    log = []
    cfg, ms = _descend(grid, step, [("batch_blocks", BLOCKS), ("block_shift", SHIFTS),
                                    ("fine_skip", _fine(FINE_BATCH))], reps, log)
    entry = {"config": cfg, "ms": ms, "trials": [[c, t] for c, t in log]}
    _store(key, entry, cache)
    return dict(entry, cached=False)
