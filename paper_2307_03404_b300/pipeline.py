"""The paper's two-stage method over a sequence (Sec. 5, Sec. 6.1): offline
mapping of every k-th frame with known poses into a dynamic grid, then online
tracking of every frame against the fixed map, with the trajectory metrics of
Sec. 6.1 (ATE, RPE_t, RPE_r over 1 m) and the mapping metrics (L1 depth error
and colour PSNR on random pixels of random frames).

Every rendering, gradient, optimiser and growth step runs in the CUDA library;
this module only sequences the calls, holds the device buffers and draws the
random ray lists of the mapping steps (Sec. 5.4: mapping takes "a random set of
sample rays from all available images").
"""
from __future__ import annotations

import dataclasses
import time

import numpy as np
import torch

from . import plx, trajectory


class DynamicGrid:
    """A sparse grid that grows from observed depth (``plx_grid_grow``). The
    link array stays on the device; after each growth the library grid is
    rebuilt with the current values plus initial values for the new vertices
    (density ``density0`` > 0, where the ReLU passes gradient; SH 0, colour 0.5),
    and the RMSProp state is extended with zeros."""

    def __init__(self, res, lo, hi, storage="f32", density0=0.1):
        self.res = tuple(int(r) for r in res)
        self.lo = np.asarray(lo, np.float64)
        self.hi = np.asarray(hi, np.float64)
        self.storage = storage
        self.density0 = float(density0)
        R = self.res
        self.links = torch.full((R[2], R[1], R[0]), -1, dtype=torch.int32, device="cuda")
        self.n = 0
        self.grid = None
        self.state = torch.zeros(0, plx.GRAD_STRIDE, device="cuda")

    def grow(self, cams: plx.CameraSet, depth: torch.Tensor, band: float, depth_is_z=True) -> int:
        n_new = int(plx.grid_grow(self.res, self.lo, self.hi, self.links, self.n, cams, depth, band,
                                  depth_is_z=depth_is_z).item())
        if n_new < 0:
            raise RuntimeError("grid_grow: vertex count would exceed int32")
        if n_new == 0 and self.grid is not None:
            return 0
        if self.grid is not None:
            dens, sh = self.grid.download()
            self.grid.close()
        else:
            dens = torch.empty(0, device="cuda")
            sh = torch.empty(0, 27, device="cuda")
        dens = torch.cat([dens, torch.full((n_new,), self.density0, device="cuda")])
        sh = torch.cat([sh, torch.zeros(n_new, 27, device="cuda")])
        self.state = torch.cat([self.state, torch.zeros(n_new, plx.GRAD_STRIDE, device="cuda")])
        self.n += n_new
        self.grid = plx.Grid(self.res, self.lo, self.hi, self.links, dens, sh, self.storage)
        return n_new

    def close(self):
        if self.grid is not None:
            self.grid.close()
            self.grid = None


@dataclasses.dataclass
class MapConfig:
    """RMSProp mapping; the rates decay exponentially from lr_* to lr_*_final
    over the steps (the paper gives no schedule). 3000 steps: surfaces that the
    keyframes see only from far away converge last, and until they do the
    map's loss minimum for frames looking at them lies centimetres from the
    true pose (on the 300-frame room256 sequence the last 50 frames' mean
    error after tracking is 7.9 / 1.85 / 0.73 / 0.48 cm after 200 / 1000 /
    3000 / 6000 steps)."""
    iters: int = 3000
    rays_per_step: int = 1 << 18
    lr_density: float = 3.0
    lr_sh: float = 0.02
    lr_density_final: float = 3.0
    lr_sh_final: float = 0.02
    alpha: float = 0.95
    eps: float = 1e-8
    band: float = 2.0
    seed: int = 7
    sort_rays: bool = True      # order each step's random rays for coherence
    sample_cache: bool = True   # forward keeps compositing samples for the adjoint
    cache_check_every: int = 50  # steps between looks at the cache's overflow
    cache_max_overflow: float = 0.01  # re-size when more rays than this re-march


@dataclasses.dataclass
class TrackConfig:
    """Adam tracking per frame; the rate decays exponentially from lr to
    lr_final over the iterations (each captured call carries its own rate)."""
    iters: int = 200
    n_rays: int = 4096
    lr: float = 1e-3
    lr_final: float = 1e-4
    beta1: float = 0.9
    beta2: float = 0.999
    eps: float = 1e-8
    constant_velocity: bool = True
    seed: int = 11
    method: str = "adam"        # "adam": the paper's tracker; "lm": damped Gauss-Newton
    lm_iters: int = 20          # LM iterations per frame (whole-frame Jacobian each)
    lm_lambda: float = 1e-3


def _morton2(x, y):
    """Interleave the bits of two non-negative int64 tensors (< 2^16)."""
    def spread(a):
        a = a & 0xFFFF
        a = (a | (a << 8)) & 0x00FF00FF
        a = (a | (a << 4)) & 0x0F0F0F0F
        a = (a | (a << 2)) & 0x33333333
        a = (a | (a << 1)) & 0x55555555
        return a
    return spread(x) | (spread(y) << 1)


def map_offline(dg: DynamicGrid, cams: plx.CameraSet, rgb: torch.Tensor, depth: torch.Tensor,
                opts, cfg: MapConfig, log=None):
    """Grow the grid from the keyframes' depth, then ``cfg.iters`` RMSProp
    steps, each on ``cfg.rays_per_step`` rays drawn uniformly (with
    replacement) from all keyframe pixels. rgb/depth hold every pixel of every
    keyframe in camera order. Returns per-step losses (device FP64 [iters])
    and a record of the sample cache: its cap, every re-sizing, and the rays
    that overflowed it (re-marched) at each check.

    The cache is sized on the first ray set with headroom. As the grid's
    values change, rays may composite more samples than the cap; those are
    re-marched, correctly but slower. Every ``cache_check_every`` steps the
    overflow of the step just taken is read (one device-to-host copy); above
    ``cache_max_overflow`` of the rays the cache is rebuilt with a cap of
    1.25 x that step's largest count."""
    dg.grow(cams, depth, cfg.band, depth_is_z=bool(opts.depth_is_z))
    sizes = torch.tensor([w * h for w, h in cams.sizes], device="cuda")
    offs = torch.cumsum(sizes, 0) - sizes
    total = int(sizes.sum())
    gen = torch.Generator(device="cuda")
    gen.manual_seed(cfg.seed)
    grad = torch.zeros(dg.n, plx.GRAD_STRIDE, device="cuda")
    losses = torch.zeros(cfg.iters, 2, dtype=torch.float64, device="cuda")
    fw = None
    cache, oc = None, opts
    cache_log = {"cap": [], "overflow": []}
    widths = torch.tensor([w for w, _ in cams.sizes], device="cuda")
    for it in range(cfg.iters):
        rows = torch.randint(0, total, (cfg.rays_per_step,), generator=gen, device="cuda")
        cam_id = torch.searchsorted(offs, rows, right=True) - 1
        pix = rows - offs[cam_id]
        if cfg.sort_rays:
            # the same random set, ordered by camera and then by the Z-order of
            # the pixel, so the rays of a warp are neighbours in the image and
            # share grid lines as dense tiles do
            w = widths[cam_id]
            key = (cam_id << 40) | _morton2(pix % w, pix // w)
            order = torch.argsort(key)
            rows, cam_id, pix = rows[order], cam_id[order], pix[order]
        cam_id, pix = cam_id.to(torch.int32), pix.to(torch.int32)
        rays = (cam_id, pix)
        rgb_t, depth_t = rgb[rows], depth[rows]
        if it == 0 and cfg.sample_cache:
            # sized on the first ray set with headroom; a later ray with more
            # compositing samples than the cap is re-marched by the adjoint
            cache = plx.SampleCache.sized_for(dg.grid, cams, opts, rays=rays, headroom=1.5)
            oc = cache.opts(opts)
            cache_log["cap"].append([0, cache.cap])
        fw = plx.render_forward(dg.grid, cams, oc, rays=rays, out=fw)
        plx.render_backward_grid(dg.grid, cams, oc, rgb_t, depth_t, fw["rgb"], fw["depth"],
                                 rays=rays, grad=grad, loss=losses[it])
        if cache is not None and (it + 1) % cfg.cache_check_every == 0:
            cnt = cache.counts()
            over = int((cnt > cache.cap).sum().item())
            cache_log["overflow"].append([it, over])
            if over > cfg.cache_max_overflow * cnt.shape[0]:
                cap = int(1.25 * int(cnt.max().item()) + 7) // 8 * 8
                del oc, cache
                cache = plx.SampleCache(cfg.rays_per_step, cap)
                oc = cache.opts(opts)
                cache_log["cap"].append([it + 1, cap])
                if log:
                    log(f"[map] step {it}: {over} rays overflowed the sample cache; cap -> {cap}")
        f = it / max(1, cfg.iters - 1)
        lr_d = cfg.lr_density * (cfg.lr_density_final / cfg.lr_density) ** f
        lr_s = cfg.lr_sh * (cfg.lr_sh_final / cfg.lr_sh) ** f
        plx.grid_rmsprop(dg.grid, grad, dg.state, lr_s, cfg.alpha, cfg.eps, zero_grad=True,
                         lr_density=lr_d)
        if log and (it % 250 == 0 or it == cfg.iters - 1):
            log(f"[map] step {it} loss {float(losses[it, 0]):.5f}")
    return losses[:, 0], cache_log


def mapping_metrics(grid: plx.Grid, cam_list, rgb_frames, depth_frames, opts, n_rays=100_000,
                    n_frames=32, seed=3):
    """L1 depth error (metres, over pixels with valid depth) and colour PSNR
    (dB, peak 1) on random pixels of ``n_frames`` random frames (Sec. 6.1's
    mapping metrics). The rendered depth is a ray distance; sensor z-depths
    are compared after turning them into ray distances. rgb_frames /
    depth_frames: [n, W*H, 3] / [n, W*H], one camera size."""
    rng = np.random.default_rng(seed)
    pick = np.sort(rng.choice(len(cam_list), size=min(n_frames, len(cam_list)), replace=False))
    cam_list = [cam_list[k] for k in pick]
    cams = plx.CameraSet(cam_list)
    npx = int(cam_list[0].width) * int(cam_list[0].height)
    gen = torch.Generator(device="cuda")
    gen.manual_seed(seed)
    cam_id = torch.randint(0, len(cam_list), (n_rays,), generator=gen, device="cuda",
                           dtype=torch.int32)
    pix = torch.randint(0, npx, (n_rays,), generator=gen, device="cuda", dtype=torch.int32)
    frame = torch.from_numpy(pick).cuda()[cam_id.long()]
    rgb_t = rgb_frames[frame, pix.long()]
    d = depth_frames[frame, pix.long()].double()
    out = plx.render_forward(grid, cams, opts, rays=(cam_id, pix), state=False)
    mse = torch.mean((out["rgb"].double() - rgb_t.double()) ** 2)
    psnr = float(-10.0 * torch.log10(mse))
    ok = torch.isfinite(d) & (d > 0)
    if opts.depth_is_z:
        par = torch.tensor([[c.fx, c.fy, c.cx, c.cy, c.width] for c in cam_list],
                           dtype=torch.float64, device="cuda")[cam_id.long()]
        p = pix.double()
        u = torch.remainder(p, par[:, 4]) + 0.5
        v = torch.div(p, par[:, 4], rounding_mode="floor") + 0.5
        d = d * torch.sqrt(((u - par[:, 2]) / par[:, 0]) ** 2 + ((v - par[:, 3]) / par[:, 1]) ** 2
                           + 1.0)
    l1 = float(torch.mean(torch.abs(out["depth"].double()[ok] - d[ok])))
    return {"l1_depth_m": l1, "psnr_db": psnr, "rays": n_rays}


def track_sequence(grid: plx.Grid, cam_list, rgb_frames, depth_frames, opts, cfg: TrackConfig,
                   init_pose=None, log=None):
    """Track every frame against the fixed map: Adam on random rays of the
    current frame (``plx_track_adam_step``), ``cfg.iters`` iterations per
    frame captured in one CUDA graph. Frame k starts from frame k-1's estimate
    (times the last inter-frame motion when ``constant_velocity``); frame 0
    starts at ``init_pose`` (default: its given pose). Returns the estimated
    poses [n, 3, 4] (FP64, numpy) and the mean milliseconds per frame."""
    intr = cam_list[0]
    one = plx.CameraSet([intr])
    W, H = int(intr.width), int(intr.height)
    rgb_buf = torch.empty(W * H, 3, device="cuda")
    depth_buf = torch.empty(W * H, device="cuda")
    state = plx.adam_state()
    outs = (torch.empty(6, 6, device="cuda", dtype=torch.float64),
            torch.empty(6, device="cuda", dtype=torch.float64),
            torch.empty(2, device="cuda", dtype=torch.float64))

    if cfg.method == "lm":
        state = plx.lm_state()

    def iterations():
        if cfg.method == "lm":
            for _ in range(cfg.lm_iters):
                plx.render_backward_pose(grid, one, 0, opts, rgb_buf, depth_buf, out=outs)
                plx.pose_step_lm(outs[0], outs[1], outs[2], state, one.poses[0], cfg.lm_lambda)
            return
        for k in range(cfg.iters):
            lr = cfg.lr * (cfg.lr_final / cfg.lr) ** (k / max(1, cfg.iters - 1))
            plx.track_adam_step(grid, one, 0, opts, cfg.n_rays, cfg.seed, rgb_buf, depth_buf, state,
                                lr, cfg.beta1, cfg.beta2, cfg.eps, out=outs)

    # capture once (warm-up on a side stream first, as CUDA graphs require)
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(s):
        state.zero_()
        if cfg.method == "lm":
            plx.render_backward_pose(grid, one, 0, opts, rgb_buf, depth_buf, out=outs)
        else:
            plx.track_adam_step(grid, one, 0, opts, cfg.n_rays, cfg.seed, rgb_buf, depth_buf,
                                state, cfg.lr, cfg.beta1, cfg.beta2, cfg.eps, out=outs)
    torch.cuda.current_stream().wait_stream(s)
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph):
        iterations()

    n = len(cam_list)
    est = np.zeros((n, 3, 4))
    est_h = np.tile(np.eye(4), (n, 1, 1))
    first = np.asarray(cam_list[0].T_wc if init_pose is None else init_pose, np.float64)
    start, end = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ms = 0.0
    for k in range(n):
        if k == 0:
            pred = first.reshape(3, 4)
        elif cfg.constant_velocity and k >= 2:
            motion = est_h[k - 1] @ np.linalg.inv(est_h[k - 2])
            pred = (motion @ est_h[k - 1])[:3]
        else:
            pred = est[k - 1]
        one.poses.copy_(torch.from_numpy(pred.reshape(1, 12)))
        rgb_buf.copy_(rgb_frames[k])
        depth_buf.copy_(depth_frames[k])
        state.zero_()
        start.record()
        graph.replay()
        end.record()
        end.synchronize()
        ms += start.elapsed_time(end)
        est[k] = one.poses.reshape(3, 4).cpu().numpy()
        est_h[k, :3] = est[k]
        if log and k % 50 == 0:
            log(f"[track] frame {k}")
    return est, ms / n


def run(scene, n_frames=300, span=0.3, map_every=10, res=None, storage="f32", depth_noise=0.0025,
        map_cfg=None, track_cfg=None, extra_track_cfgs=(), seed=21, log=None, map_last=True,
        per_frame=False, keep=None):
    """Whole pipeline on a synthetic room: a smooth sequence of ``n_frames``
    640x480 RGB-D frames along the first ``span`` of a spline path (depth
    noise N(0, (depth_noise z^2)^2), 2% of depths missing), every
    ``map_every``-th frame mapped with its true pose into a ``res``^3 dynamic
    grid over the scene's box, every frame tracked from the first true pose
    with ``track_cfg`` (and again with each of ``extra_track_cfgs``, on the
    same map). With ``map_last`` the last frame is a keyframe too, so that no
    tracked frame looks past the mapped end of the sequence (without it the
    frames after the last keyframe see space the map has never observed,
    which renders empty, and tracking there drifts). ``per_frame`` adds each
    frame's camera-centre error. With a dict ``keep`` the map stays open and
    the dict receives it ("grid", "opts", "close") with the sequence ("cams",
    "rgb", "depth" per frame, true poses "gt"), so a caller can track more on
    it; the caller then calls ``keep["close"]()``. Returns a dict of metrics
    and timings."""
    from . import scenes

    map_cfg = map_cfg or MapConfig()
    track_cfg = track_cfg or TrackConfig()
    cams_np = scenes.sequence_cameras(scene, n_frames, seed, span=span)
    rgb, depth = scenes.sensor_frames_torch(scene, cams_np, seed + 1, device="cuda",
                                            depth_noise=depth_noise)
    npx = cams_np[0].width * cams_np[0].height
    rgb = rgb.reshape(n_frames, npx, 3)
    depth = depth.reshape(n_frames, npx)
    g = scene.grid
    R = res or g.res[0]
    opts = plx.opts_from_dict(dict(step=0.5 * float((g.hi[0] - g.lo[0]) / (R - 1)), lambda_d=1.0,
                                   depth_is_z=True))
    keys = list(range(0, n_frames, map_every))
    if map_last and keys[-1] != n_frames - 1:
        keys.append(n_frames - 1)
    kcams = plx.CameraSet([cams_np[k] for k in keys])
    krgb = rgb[keys].reshape(-1, 3).contiguous()
    kdepth = depth[keys].reshape(-1).contiguous()
    dg = DynamicGrid((R, R, R), g.lo, g.hi, storage)
    torch.cuda.synchronize()
    t0 = time.time()
    losses, cache_log = map_offline(dg, kcams, krgb, kdepth, opts, map_cfg, log=log)
    torch.cuda.synchronize()
    t_map = time.time() - t0
    mm = mapping_metrics(dg.grid, cams_np, rgb, depth, opts)
    gt = np.array([np.asarray(c.T_wc, np.float64).reshape(3, 4) for c in cams_np])

    def tracked(cfg):
        est, ms_frame = track_sequence(dg.grid, cams_np, rgb, depth, opts, cfg, log=log)
        t_rpe, r_rpe = trajectory.rpe(est, gt)
        err = np.linalg.norm(est[:, :, 3] - gt[:, :, 3], axis=1)
        desc = (f"Adam, {cfg.iters} iterations of {cfg.n_rays} random rays" if cfg.method == "adam"
                else f"Levenberg-Marquardt, {cfg.lm_iters} whole-frame Jacobians")
        res = {"tracker": desc, "track_ms_per_frame": ms_frame,
               "ate_m": trajectory.ate(est, gt), "rpe_t_m": t_rpe, "rpe_r_deg": r_rpe,
               "median_err_m": float(np.median(err)), "max_err_m": float(err.max())}
        if per_frame:
            res["err_m"] = err.tolist()
        return res

    out = {"frames": n_frames, "keyframes": len(keys), "grid": f"{R}^3 dynamic, {storage}",
           "allocated": dg.n, "map_seconds": t_map, "map_steps": map_cfg.iters,
           "map_rays_per_step": map_cfg.rays_per_step,
           "map_loss_first_last": [float(losses[0]), float(losses[-1])],
           "sample_cache": cache_log,
           "mapping": mm,
           "path_m": float(np.sum(np.linalg.norm(np.diff(gt[:, :, 3], axis=0), axis=1)))}
    out.update(tracked(track_cfg))
    out["other_trackers"] = [tracked(c) for c in extra_track_cfgs]
    if keep is None:
        dg.close()
    else:
        keep.update(grid=dg.grid, opts=opts, close=dg.close, cams=cams_np, rgb=rgb, depth=depth,
                    gt=gt)
    return out


def main(argv=None):
    """Command line: run the pipeline on the seeded 256^3 room and print the
    metrics as one JSON line (python -m paper_2307_03404_b300.pipeline)."""
    import argparse
    import json
    import sys

    from . import scenes

    ap = argparse.ArgumentParser(description=main.__doc__)
    ap.add_argument("--frames", type=int, default=300)
    ap.add_argument("--span", type=float, default=0.3)
    ap.add_argument("--map-every", type=int, default=10)
    ap.add_argument("--map-steps", type=int, default=1000)
    ap.add_argument("--tracker", choices=["adam", "lm"], default="adam")
    ap.add_argument("--storage", default="f32", choices=["f32", "bf16", "f16", "f32_bf16"])
    a = ap.parse_args(argv)
    R, occ, npr, seed = scenes.WORKLOADS["room256"]
    sc = scenes.room_scene(R, occ, npr, seed)
    out = run(sc, n_frames=a.frames, span=a.span, map_every=a.map_every, storage=a.storage,
              map_cfg=MapConfig(iters=a.map_steps), track_cfg=TrackConfig(method=a.tracker),
              log=lambda *m: print(*m, file=sys.stderr, flush=True))
    print(json.dumps(out))


if __name__ == "__main__":
    main()
