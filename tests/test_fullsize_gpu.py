"""Full-size launches against the FP64 oracle, element by element.

The mapping adjoint the benchmark times (dense launch, one whole 640x480
keyframe of the 256^3 room with sensor targets: 307,200 rays) is compared
with the oracle's gradient of every grid value (Sec. 5.2, Eq. 6-10), without
a sample cache and with a fitted one. The FP32 set-up
of a ray may round its sample count (floor((t_max - t_min) / delta)) the other
way from the FP64 oracle; the rate of such flips is bounded and, because the
room keeps an empty border, a flipped sample adds nothing: colour and depth of
the flipped rays stay within the FP32 bound.

The batched persistent launch (Sec. 5.2 + 5.3) on the 512^3 mixed-resolution
room: frames of all four sizes, mapping and tracking mixed, against the
separate calls; its smallest mapping and tracking frames again alone against
the oracle.
"""
import os

import numpy as np
import pytest
import torch

import oracle
from gpu_helpers import dev, norm_err, rel_err
from paper_2307_03404_b300 import plx, scenes

pytestmark = pytest.mark.gpu

TOL_FWD = 1e-5
TOL_GRAD = 1e-4


@pytest.fixture(scope="module")
def keyframe():
    oracle.set_threads(os.cpu_count() or 1)
    R, occ, npr, seed = scenes.WORKLOADS["room256"]
    sc = scenes.room_scene(R, occ, npr, seed)
    cam = scenes.room_cameras(sc, 8, seed + 1)[0]
    rgb_t, depth_t = scenes.sensor_frames(sc, [cam], seed + 2)
    opts = dict(step=0.5 * float(sc.grid.h[0]), lambda_d=1.0, depth_is_z=True)
    ref = oracle.grad_grid(sc.grid, [cam], opts, rgb_t, depth_t)
    return sc.grid, cam, rgb_t, depth_t, opts, ref


@pytest.mark.parametrize("cache", [None, "fit", "range", "range+small"])
def test_dense_keyframe_adjoint_against_oracle(keyframe, cache):
    """cache None: the re-marching adjoint; "fit": a sample cache that holds
    every ray; "range": the re-march over each ray's compositing range;
    "range+small": a cache of 8 samples per ray, most rays overflowing it
    and re-marching over their range."""
    g, cam, rgb_t, depth_t, opts, ref = keyframe
    grid = plx.Grid.from_scene(g, "f32")
    cams = plx.CameraSet([cam])
    o = plx.opts_from_dict(opts)
    if cache == "fit":
        sc_ = plx.SampleCache.sized_for(grid, cams, o)
        o = sc_.opts(o)
    if cache in ("range", "range+small"):
        o = plx.RayRange(cams.n_pixels()).opts(o)
    if cache == "range+small":
        o = plx.SampleCache(cams.n_pixels(), 8).opts(o)
    fw = plx.render_forward(grid, cams, o)
    grad, loss = plx.render_backward_grid(grid, cams, o, dev(rgb_t), dev(depth_t), fw["rgb"],
                                          fw["depth"])
    torch.cuda.synchronize()
    grid.check()
    if cache == "fit":
        assert int(sc_.counts().max().item()) <= sc_.cap  # every ray through the cache
    grid.close()
    gn = grad.cpu().numpy()
    l = loss.cpu().numpy()
    assert l[1] == ref.M and ref.M > 0.95 * cam.width * cam.height
    assert abs(l[0] - ref.loss) <= 1e-5 * ref.loss
    assert norm_err(gn[:, 0], ref.grad_density) <= TOL_GRAD
    assert norm_err(gn[:, 1:28], ref.grad_sh) <= TOL_GRAD
    assert np.all(gn[:, 28:] == 0)
    assert (np.abs(ref.grad_density) > 0).sum() > 50_000   # a real full-frame scatter


def test_sample_count_flips_are_rare_and_harmless(keyframe):
    """20,000 seeded rays of the keyframe: marched / allocated sample counts
    against the oracle's, and the outputs of the rays whose counts differ."""
    g, cam, _, _, opts, _ = keyframe
    pix = np.random.default_rng(11).permutation(cam.width * cam.height)[:20000].astype(np.int32)
    rays = (np.zeros(pix.shape[0], np.int32), pix)
    ref = oracle.render(g, [cam], opts, rays)
    grid = plx.Grid.from_scene(g, "f32")
    cams = plx.CameraSet([cam])
    out = plx.render_forward(grid, cams, plx.opts_from_dict(opts), counts=True)
    torch.cuda.synchronize()
    grid.close()
    cnt = out["counts"].cpu().numpy()[pix]
    flip = (cnt[:, 0] != ref.n_marched) | (cnt[:, 1] != ref.n_alloc)
    assert flip.mean() <= 0.003, flip.mean()
    # a count differs by one sample, at the box exit inside the empty border
    assert np.all(np.abs(cnt[flip, 0] - ref.n_marched[flip]) <= 1)
    assert np.all(cnt[flip, 1] == ref.n_alloc[flip])
    rgb = out["rgb"].cpu().numpy()[pix]
    depth = out["depth"].cpu().numpy()[pix]
    assert rel_err(rgb, ref.rgb) <= TOL_FWD and rel_err(depth, ref.depth) <= TOL_FWD
    if flip.any():
        assert rel_err(rgb[flip], ref.rgb[flip]) <= TOL_FWD
        assert rel_err(depth[flip], ref.depth[flip]) <= TOL_FWD


# --------------------------------------------------------------- batched
@pytest.fixture(scope="module")
def mixroom():
    oracle.set_threads(os.cpu_count() or 1)
    R, occ, npr, seed = scenes.WORKLOADS["room512mix"]
    sc = scenes.room_scene(R, occ, npr, seed)
    base = scenes.room_cameras(sc, 8, seed + 8)
    sizes = [(320, 240), (640, 480), (848, 480), (1200, 680)]
    cams_np = []
    for i, c in enumerate(base):      # each size twice, in mixed order
        W, H = sizes[(3 * i) % 4]
        f = 525.0 * W / 640.0
        cams_np.append(scenes.Camera(f, f, W / 2.0 - 0.5, H / 2.0 - 0.5, W, H, c.T_wc))
    rgb_t, depth_t = scenes.sensor_frames(sc, cams_np, seed + 2)
    opts = dict(step=0.5 * float(sc.grid.h[0]), lambda_d=1.0, depth_is_z=True)
    return sc.grid, cams_np, rgb_t, depth_t, opts


def _separate(grid, cams_np, work, o, rgb_t, depth_t, offs):
    """The batch's work through plx_render_forward / plx_render_backward_grid
    (all mapping items in one list-mode call: the same M) and
    plx_render_backward_pose per tracking item."""
    cams = plx.CameraSet(cams_np)
    mi = [i for i, (_, m) in enumerate(work) if m == plx.WORK_MAP]
    mcid = np.concatenate([np.full(offs[i + 1] - offs[i], work[i][0], np.int32) for i in mi])
    mpix = np.concatenate([np.arange(offs[i + 1] - offs[i], dtype=np.int32) for i in mi])
    mr = np.concatenate([np.arange(offs[i], offs[i + 1]) for i in mi])
    rr = (dev(mcid, torch.int32), dev(mpix, torch.int32))
    f = plx.render_forward(grid, cams, o, rays=rr)
    g2, l2 = plx.render_backward_grid(grid, cams, o, dev(rgb_t[mr]), dev(depth_t[mr]), f["rgb"],
                                      f["depth"], rays=rr)
    poses = []
    for i, (c, m) in enumerate(work):
        if m == plx.WORK_TRACK:
            sl = slice(offs[i], offs[i + 1])
            H, b, l = plx.render_backward_pose(grid, cams, c, o, dev(rgb_t[sl]), dev(depth_t[sl]))
            poses.append((H.cpu().numpy(), b.cpu().numpy(), l.cpu().numpy()))
    torch.cuda.synchronize()
    return g2.cpu().numpy(), l2.cpu().numpy(), poses


@pytest.mark.parametrize("storage,cache", [("bf16", True), ("f32", False)])
def test_batched_mixed_frames_match_separate_calls(mixroom, storage, cache):
    g, cams_np, rgb_t, depth_t, opts = mixroom
    work = [(i, plx.WORK_MAP if i % 2 == 0 else plx.WORK_TRACK) for i in range(len(cams_np))]
    sizes = [c.width * c.height for c in cams_np]
    offs = np.cumsum([0] + sizes)
    assert len({(c.width, c.height) for c in cams_np}) == 4
    grid = plx.Grid.from_scene(g, storage)
    cams = plx.CameraSet(cams_np)
    o = plx.opts_from_dict(opts)
    ob = plx.SampleCache.for_batch(256).opts(o) if cache else o
    grad, mloss, H, b, tloss = plx.render_batch(grid, cams, work, ob, dev(rgb_t), dev(depth_t))
    torch.cuda.synchronize()
    grid.check()
    g2, l2, poses = _separate(grid, cams_np, work, o, rgb_t, depth_t, offs)
    grid.close()
    gb = grad.cpu().numpy()
    assert mloss[1].item() == l2[1]
    assert abs(mloss[0].item() - l2[0]) <= 1e-6 * l2[0]
    assert norm_err(gb[:, :28], g2[:, :28]) <= 1e-5
    for s, (Hs, bs, ls) in enumerate(poses):
        assert tloss[s, 1].item() == ls[1]
        assert abs(tloss[s, 0].item() - ls[0]) <= 1e-6 * ls[0]
        assert norm_err(H[s].cpu().numpy(), Hs) <= 1e-5
        assert norm_err(b[s].cpu().numpy(), bs) <= 1e-5


def test_batched_smallest_frames_against_oracle(mixroom):
    """One 320x240 frame mapped and another tracked, in one batched launch
    with a sample cache, against the oracle's gradient and pose system."""
    g, cams_np, rgb_t, depth_t, opts = mixroom
    small = [i for i, c in enumerate(cams_np) if c.width == 320][:2]
    sub = [cams_np[i] for i in small]
    sizes = [c.width * c.height for c in cams_np]
    offs = np.cumsum([0] + sizes)
    rows = np.concatenate([np.arange(offs[i], offs[i + 1]) for i in small])
    rgb_s, depth_s = rgb_t[rows], depth_t[rows]
    work = [(0, plx.WORK_MAP), (1, plx.WORK_TRACK)]
    grid = plx.Grid.from_scene(g, "f32")
    cams = plx.CameraSet(sub)
    o = plx.opts_from_dict(opts)
    ob = plx.SampleCache.for_batch(256).opts(o)
    grad, mloss, H, b, tloss = plx.render_batch(grid, cams, work, ob, dev(rgb_s), dev(depth_s))
    torch.cuda.synchronize()
    grid.check()
    grid.close()
    n = sub[0].width * sub[0].height
    ref = oracle.grad_grid(g, [sub[0]], opts, rgb_s[:n], depth_s[:n])
    gb = grad.cpu().numpy()
    assert mloss[1].item() == ref.M
    assert abs(mloss[0].item() - ref.loss) <= 1e-5 * ref.loss
    assert norm_err(gb[:, 0], ref.grad_density) <= TOL_GRAD
    assert norm_err(gb[:, 1:28], ref.grad_sh) <= TOL_GRAD
    rp = oracle.pose_jacobian(g, [sub[1]], opts, rgb_s[n:], depth_s[n:])
    assert tloss[0, 1].item() == rp.M
    assert abs(tloss[0, 0].item() - rp.loss) <= 1e-5 * rp.loss
    assert norm_err(H[0].cpu().numpy(), rp.H) <= TOL_GRAD
    assert norm_err(b[0].cpu().numpy(), rp.b) <= TOL_GRAD
