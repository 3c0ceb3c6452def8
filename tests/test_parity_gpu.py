"""CUDA path vs FP64 oracle, element by element, through the C ABI.

Tolerances: FP32 colour/depth 1e-5 relative (|d| / max(|ref|, 1e-3)),
gradients and pose systems 1e-4 norm-wise, BF16-stored colour 2e-3
relative; integer sample counts bit-exact.
"""
import math

import numpy as np
import pytest
import torch

import oracle
from gpu_helpers import GpuCase, dev, norm_err, rel_err
from paper_2307_03404_b300 import plx, scenes

pytestmark = pytest.mark.gpu

TOL_FWD = 1e-5
TOL_GRAD = 1e-4


@pytest.fixture(scope="module")
def sphere():
    g, cam, gp = scenes.sphere_scene()
    opts = dict(step=0.5 * g.h[0], lambda_d=1.0)
    return g, cam, gp, opts


def tiny_cams():
    T1 = scenes.look_at((2.2, 1.4, -2.6), (0, 0.1, 0))
    T2 = scenes.look_at((-2.0, 0.8, 2.4), (0.1, 0, 0))
    T3 = scenes.look_at((0.3, 2.9, 0.2), (0, 0, 0), up=(0, 0, 1))
    return [scenes.Camera(7.0, 6.5, 6.3, 3.4, 13, 7, T1),
            scenes.Camera(5.0, 5.0, 4.0, 2.0, 8, 4, T2),
            scenes.Camera(3.0, 3.0, 0.5, 0.5, 1, 1, T3)]


# ------------------------------------------------------------------ forward
def test_forward_sphere_scene(sphere):
    g, cam, _, opts = sphere
    case = GpuCase(g, [cam])
    got = case.forward(opts)
    ref = oracle.render(g, [cam], opts)
    assert rel_err(got["rgb"], ref.rgb) <= TOL_FWD
    assert rel_err(got["depth"], ref.depth) <= TOL_FWD
    assert np.abs(got["state"] - ref.T_final).max() <= 1e-6
    np.testing.assert_array_equal(got["counts"][:, 0], ref.n_marched)
    np.testing.assert_array_equal(got["counts"][:, 1], ref.n_alloc)
    assert (ref.n_alloc > 0).mean() > 0.3


@pytest.mark.parametrize("alloc,act,bg,max_samples,near", [
    (1.0, "sigmoid", (0, 0, 0), 1 << 30, 0.0),
    (0.6, "sigmoid", (0.2, 0.4, 0.9), 1 << 30, 0.0),
    (0.8, "identity", (0.5, 0.5, 0.5), 7, 0.0),
    (0.7, "sigmoid", (0.1, 0.0, 0.3), 1 << 30, 2.9),
])
def test_forward_tiny_grids_several_cameras(alloc, act, bg, max_samples, near):
    g = scenes.tiny_grid(7, seed=21, alloc_frac=alloc, sigma_mean=2.0, sigma_std=2.0)
    cams = tiny_cams()
    opts = dict(step=0.11, bg=bg, color_act=act, max_samples=max_samples, near=near)
    case = GpuCase(g, cams)
    got = case.forward(opts)
    ref = oracle.render(g, cams, opts)
    assert got["rgb"].shape == (13 * 7 + 8 * 4 + 1, 3)
    assert rel_err(got["rgb"], ref.rgb) <= TOL_FWD
    assert rel_err(got["depth"], ref.depth) <= TOL_FWD
    np.testing.assert_array_equal(got["counts"][:, 0], ref.n_marched)
    np.testing.assert_array_equal(got["counts"][:, 1], ref.n_alloc)
    # list mode: a shuffled subset with repeats, rows follow the list
    rng = np.random.default_rng(3)
    cid, pix = scenes.dense_rays(cams)
    sel = rng.integers(0, cid.shape[0], 77)
    rays = (cid[sel], pix[sel])
    got_l = case.forward(opts, rays=rays)
    np.testing.assert_array_equal(got_l["rgb"], got["rgb"][sel])
    np.testing.assert_array_equal(got_l["depth"], got["depth"][sel])


def test_forward_edge_cases():
    cams = tiny_cams()
    opts = dict(step=0.1, bg=(0.3, 0.6, 0.9))
    # zero density everywhere: background, depth 0
    g0 = scenes.constant_grid(5, 0.0, (1.0, 1.0, 1.0))
    got = GpuCase(g0, cams).forward(opts)
    np.testing.assert_allclose(got["rgb"], np.tile([0.3, 0.6, 0.9], (got["rgb"].shape[0], 1)),
                               rtol=1e-7)
    assert np.all(got["depth"] == 0)
    # nothing allocated at all
    ge = scenes.Grid((4, 4, 4), np.full(3, -1.0), np.full(3, 1.0),
                     np.full((4, 4, 4), -1, np.int32), np.zeros(0, np.float32),
                     np.zeros((0, 27), np.float32))
    got = GpuCase(ge, cams).forward(opts)
    assert np.all(got["counts"][:, 1] == 0) and np.all(got["depth"] == 0)
    # empty ray list
    case = GpuCase(scenes.tiny_grid(5, seed=2), cams)
    got = case.forward(opts, rays=(np.zeros(0, np.int32), np.zeros(0, np.int32)))
    assert got["rgb"].shape == (0, 3)
    # rays that miss the box
    away = scenes.Camera(4.0, 4.0, 2.0, 2.0, 4, 4, scenes.look_at((0, 0, 3), (0, 0, 6)))
    got = GpuCase(scenes.tiny_grid(5, seed=2), [away]).forward(opts)
    assert np.all(got["counts"][:, 0] == 0)
    np.testing.assert_allclose(got["rgb"][:, 2], 0.9, rtol=1e-7)


def test_axis_aligned_rays_on_grid_planes():
    """Rays exactly along the grid axes, starting on vertex planes (direction
    components exactly 0, sample positions exactly on cell faces): forward,
    adjoint and pose system against the oracle, sample counts bit-exact."""
    g = scenes.tiny_grid(9, seed=4, alloc_frac=0.8)
    h = (g.hi - g.lo) / (np.array(g.res) - 1)
    cams = []
    for R_ in (np.eye(3), np.array([[0.0, 0, 1], [0, 1, 0], [-1, 0, 0]]),
               np.array([[1.0, 0, 0], [0, 0, -1], [0, 1, 0]])):
        T = np.zeros((3, 4))
        T[:, :3] = R_
        T[:, 3] = g.lo + h * np.array([4.0, 3.0, 2.0]) - 3.0 * R_[:, 2]   # a vertex, 3 back
        # 5x5 pixels with the centre pixel's ray exactly on the optical axis
        cams.append(scenes.Camera(6.0, 6.0, 2.5, 2.5, 5, 5, T))
    opts = dict(step=0.5 * h[0], lambda_d=0.6, depth_is_z=False, bg=(0.2, 0.1, 0.3))
    case = GpuCase(g, cams)
    got = case.forward(opts)
    ref = oracle.render(g, cams, opts)
    assert rel_err(got["rgb"], ref.rgb) <= TOL_FWD
    assert rel_err(got["depth"], ref.depth) <= TOL_FWD
    np.testing.assert_array_equal(got["counts"][:, 0], ref.n_marched)
    np.testing.assert_array_equal(got["counts"][:, 1], ref.n_alloc)
    rgb_t = np.clip(ref.rgb + 0.05, 0, 1).astype(np.float32)
    depth_t = (ref.depth * 1.02 + 0.01).astype(np.float32)
    gd, gs, _, loss = case.backward_grid(opts, rgb_t, depth_t)
    rg = oracle.grad_grid(g, cams, opts, rgb_t, depth_t)
    assert norm_err(gd, rg.grad_density) <= TOL_GRAD and norm_err(gs, rg.grad_sh) <= TOL_GRAD
    H, b, _ = case.backward_pose(opts, 1, rgb_t[25:50], depth_t[25:50])
    rp = oracle.pose_jacobian(g, [cams[1]], opts, rgb_t[25:50], depth_t[25:50])
    assert norm_err(H, rp.H) <= TOL_GRAD and norm_err(b, rp.b) <= TOL_GRAD


def test_bad_ray_list_sets_the_device_error_word():
    cams = tiny_cams()
    case = GpuCase(scenes.tiny_grid(5, seed=2), cams)
    o = plx.opts_from_dict(dict(step=0.1))
    out = plx.render_forward(case.grid, case.cams, o,
                             rays=(dev([0, 5], torch.int32), dev([3, 10 ** 6], torch.int32)))
    torch.cuda.synchronize()
    with pytest.raises(plx.PlxError) as e:
        case.grid.check()
    assert e.value.status == 4
    assert np.isnan(out["rgb"][1].cpu().numpy()).all()
    case.grid.check()  # the word is cleared by the read


# ------------------------------------------------------------------ adjoint
def sphere_targets(sphere, depth_is_z):
    g, cam, gp, opts = sphere
    tg = oracle.render(gp, [cam], dict(opts, depth_is_z=False))
    rng = np.random.default_rng(77)
    rgb_t = tg.rgb.astype(np.float32)
    if depth_is_z:
        depth_t = rng.uniform(1.5, 3.5, tg.depth.shape).astype(np.float32)
        depth_t[rng.random(depth_t.shape) < 0.05] = 0.0
        depth_t[7] = np.nan
    else:
        depth_t = tg.depth.astype(np.float32)
    return rgb_t, depth_t


@pytest.mark.parametrize("cache_cap", [None, 256, 3])
@pytest.mark.parametrize("depth_is_z,act,bg", [(False, "sigmoid", (0, 0, 0)),
                                                (True, "sigmoid", (0.3, 0.2, 0.1)),
                                                (True, "identity", (0.0, 0.5, 0.0))])
def test_backward_grid_sphere_scene(sphere, depth_is_z, act, bg, cache_cap):
    """Without a sample cache, with one that holds every ray, and with one so
    small that most rays overflow it and re-march (both paths in one call)."""
    g, cam, _, opts = sphere
    opts = dict(opts, depth_is_z=depth_is_z, color_act=act, bg=bg, lambda_d=0.7)
    rgb_t, depth_t = sphere_targets(sphere, depth_is_z)
    case = GpuCase(g, [cam])
    gd, gs, gpad, loss = case.backward_grid(opts, rgb_t, depth_t, cache_cap=cache_cap)
    if cache_cap is not None:
        kept = case.cache.counts().cpu().numpy()
        fwd = case.forward(opts)
        assert np.all(kept >= 0) and np.all(kept <= fwd["counts"][:, 1])
        if cache_cap == 256:
            assert kept.max() <= 256
        else:
            assert (kept > cache_cap).mean() > 0.2 and (kept[kept > 0] <= cache_cap).any()
    ref = oracle.grad_grid(g, [cam], opts, rgb_t, depth_t)
    assert loss[1] == ref.M
    assert abs(loss[0] - ref.loss) <= 1e-5 * ref.loss
    assert norm_err(gd, ref.grad_density) <= TOL_GRAD
    assert norm_err(gs, ref.grad_sh) <= TOL_GRAD
    assert np.all(gpad == 0)


@pytest.mark.parametrize("cache_cap", [None, 3])
@pytest.mark.parametrize("stop_T", [0.0, 1e-2])
def test_backward_grid_over_the_compositing_range(sphere, cache_cap, stop_T):
    """The forward writes each ray's compositing range (first sample with
    sigma > 0, one past the last) and the re-marching adjoint marches only
    that: the oracle's gradients (which come from the full march), with and
    without early stopping and with a cache so small that most rays
    overflow it and re-march over their range. The ranges are the first
    and last kept samples of a cached forward on the same rays."""
    g, cam, _, opts = sphere
    opts = dict(opts, depth_is_z=True, bg=(0.3, 0.2, 0.1), lambda_d=0.7, stop_T=stop_T)
    rgb_t, depth_t = sphere_targets(sphere, True)
    case = GpuCase(g, [cam])
    gd, gs, gpad, loss = case.backward_grid(opts, rgb_t, depth_t, cache_cap=cache_cap,
                                            ray_range=True)
    ref = oracle.grad_grid(g, [cam], opts, rgb_t, depth_t)
    assert loss[1] == ref.M and abs(loss[0] - ref.loss) <= 1e-5 * ref.loss
    assert norm_err(gd, ref.grad_density) <= TOL_GRAD
    assert norm_err(gs, ref.grad_sh) <= TOL_GRAD
    assert np.all(gpad == 0)
    rng = case.range.ranges().cpu().numpy()
    n = rng.shape[0]
    full = plx.SampleCache(n, 512)
    plx.render_forward(case.grid, case.cams, full.opts(plx.opts_from_dict(opts)), state=False)
    kept = full.counts().cpu().numpy()
    ck = full.buf[4 * 512 * n: 5 * 512 * n].view(torch.int32).view(512, n).cpu().numpy()
    assert kept.max() <= 512 and (kept == 0).any() and (kept > 0).any()
    has = kept > 0
    np.testing.assert_array_equal(rng[has, 0], ck[0, has])
    np.testing.assert_array_equal(rng[has, 1], ck[kept[has] - 1, np.nonzero(has)[0]] + 1)
    assert np.all(rng[~has] == 0)
    assert np.all(rng[has, 1] - rng[has, 0] >= kept[has])


@pytest.mark.parametrize("cache_cap", [None, 8])
def test_backward_grid_sparse_list_mode_accumulates(cache_cap):
    g = scenes.tiny_grid(7, seed=31, alloc_frac=0.6, sigma_mean=2.0, sigma_std=2.0)
    cams = tiny_cams()
    opts = dict(step=0.11, bg=(0.2, 0.1, 0.0), lambda_d=0.4)
    rng = np.random.default_rng(5)
    cid, pix = scenes.dense_rays(cams)
    sel = rng.permutation(cid.shape[0])[:100]
    rays = (cid[sel], pix[sel])
    rgb_t = rng.uniform(0, 1, (100, 3)).astype(np.float32)
    depth_t = rng.uniform(0.5, 4, 100).astype(np.float32)
    depth_t[::9] = -1.0
    case = GpuCase(g, cams)
    gd, gs, _, loss = case.backward_grid(opts, rgb_t, depth_t, rays=rays, cache_cap=cache_cap)
    ref = oracle.grad_grid(g, cams, opts, rgb_t, depth_t, rays=rays)
    assert loss[1] == ref.M
    assert abs(loss[0] - ref.loss) <= 1e-5 * ref.loss
    assert norm_err(gd, ref.grad_density) <= TOL_GRAD
    assert norm_err(gs, ref.grad_sh) <= TOL_GRAD
    # a second call adds into the same buffer
    o = plx.opts_from_dict(opts)
    rr = (dev(rays[0], torch.int32), dev(rays[1], torch.int32))
    out = plx.render_forward(case.grid, case.cams, o, rays=rr)
    grad, _ = plx.render_backward_grid(case.grid, case.cams, o, dev(rgb_t), dev(depth_t),
                                       out["rgb"], out["depth"], rays=rr)
    plx.render_backward_grid(case.grid, case.cams, o, dev(rgb_t), dev(depth_t), out["rgb"],
                             out["depth"], rays=rr, grad=grad)
    g2 = grad.cpu().numpy()
    assert norm_err(g2[:, 0], 2 * ref.grad_density) <= TOL_GRAD


# -------------------------------------------------------------------- pose
def test_backward_pose_matches_oracle(sphere):
    g, cam, _, opts = sphere
    opts = dict(opts, depth_is_z=False, lambda_d=0.8, bg=(0.1, 0.1, 0.2))
    ref_t = oracle.render(g, [cam], opts)
    T0 = scenes.perturb_pose(cam.T_wc, 0.03, 2.0, np.random.default_rng(9))
    cam0 = cam.with_pose(T0)
    rgb_t = ref_t.rgb.astype(np.float32)
    depth_t = ref_t.depth.astype(np.float32)
    case = GpuCase(g, [cam0])
    H, b, loss = case.backward_pose(opts, 0, rgb_t, depth_t)
    ref = oracle.pose_jacobian(g, [cam0], opts, rgb_t, depth_t)
    assert loss[1] == ref.M
    assert abs(loss[0] - ref.loss) <= 1e-5 * ref.loss
    assert norm_err(H, ref.H) <= TOL_GRAD
    assert norm_err(b, ref.b) <= TOL_GRAD
    np.testing.assert_array_equal(H, H.T)
    # pixel-list mode over a subset, with the camera among others
    pix = np.random.default_rng(1).permutation(cam.width * cam.height)[:500].astype(np.int32)
    other = scenes.Camera(10.0, 10.0, 2.0, 2.0, 4, 4, cam.T_wc)
    case2 = GpuCase(g, [other, cam0])
    H2, b2, l2 = case2.backward_pose(opts, 1, rgb_t[pix], depth_t[pix], pixels=pix)
    ref2 = oracle.pose_jacobian(g, [cam0], opts, rgb_t[pix], depth_t[pix],
                                rays=(np.zeros(500, np.int32), pix))
    assert l2[1] == ref2.M
    assert norm_err(H2, ref2.H) <= TOL_GRAD
    assert norm_err(b2, ref2.b) <= TOL_GRAD
    # deterministic reduction
    H3, b3, l3 = case2.backward_pose(opts, 1, rgb_t[pix], depth_t[pix], pixels=pix)
    np.testing.assert_array_equal(H2, H3)
    np.testing.assert_array_equal(b2, b3)


@pytest.mark.parametrize("storage", ["f32", "bf16"])
def test_backward_pose_view_direction_variant(sphere, storage):
    """PLX_POSE_VIEW_DIR (the SH colour also turns with the ray): the pose
    system against the oracle's variant, on dense and list rays and in the
    batched launch; it differs from the paper's system. Colour
    only (lambda_d = 0), identity activation and 4x SH, so the term is large
    enough to tell the two systems apart at the tolerance."""
    g0, cam, _, opts = sphere
    g = g0.with_values(g0.density, 4.0 * g0.sh)
    opts = dict(opts, depth_is_z=False, lambda_d=0.0, bg=(0.1, 0.1, 0.2), color_act="identity")
    ref_t = oracle.render(g, [cam], opts)
    T0 = scenes.perturb_pose(cam.T_wc, 0.03, 2.0, np.random.default_rng(9))
    cam0 = cam.with_pose(T0)
    rgb_t = ref_t.rgb.astype(np.float32)
    depth_t = ref_t.depth.astype(np.float32)
    gr = g
    if storage == "bf16":
        gr = g.with_values(torch.from_numpy(g.density).bfloat16().float().numpy(),
                           torch.from_numpy(g.sh).bfloat16().float().numpy())
    case = GpuCase(g, [cam0], storage=storage)
    ov = dict(opts, dir_term=True)
    H, b, loss = case.backward_pose(ov, 0, rgb_t, depth_t)
    ref = oracle.pose_jacobian(gr, [cam0], ov, rgb_t, depth_t)
    base = oracle.pose_jacobian(gr, [cam0], opts, rgb_t, depth_t)
    assert loss[1] == ref.M
    assert abs(loss[0] - ref.loss) <= 1e-5 * ref.loss
    assert norm_err(H, ref.H) <= TOL_GRAD
    assert norm_err(b, ref.b) <= TOL_GRAD
    assert norm_err(base.b, ref.b) > 10 * TOL_GRAD       # the term matters here
    pix = np.random.default_rng(2).permutation(cam.width * cam.height)[:700].astype(np.int32)
    H2, b2, _ = case.backward_pose(ov, 0, rgb_t[pix], depth_t[pix], pixels=pix)
    ref2 = oracle.pose_jacobian(gr, [cam0], ov, rgb_t[pix], depth_t[pix],
                                rays=(np.zeros(700, np.int32), pix))
    assert norm_err(H2, ref2.H) <= TOL_GRAD
    assert norm_err(b2, ref2.b) <= TOL_GRAD
    # the batched launch's tracking items honour the flag too
    _, _, Hb, bb, lb = plx.render_batch(case.grid, case.cams, [(0, plx.WORK_TRACK)],
                                        plx.opts_from_dict(ov), dev(rgb_t), dev(depth_t))
    assert lb[0, 1].item() == ref.M
    assert norm_err(Hb[0].cpu().numpy(), ref.H) <= TOL_GRAD
    assert norm_err(bb[0].cpu().numpy(), ref.b) <= TOL_GRAD


def test_pose_step_matches_oracle():
    rng = np.random.default_rng(12)
    A = rng.standard_normal((9, 6))
    H = A.T @ A + 0.05 * np.eye(6)
    b = 0.1 * rng.standard_normal(6)
    T0 = scenes.look_at((1.0, 0.4, -2.0), (0, 0, 0))
    ref_T, ref_xi, ok = oracle.pose_step(H, b, T0, damping=0.01)
    pose = dev(T0.reshape(12), torch.float64)
    xi = torch.empty(6, device="cuda", dtype=torch.float64)
    st = torch.full((1,), 7, device="cuda", dtype=torch.int32)
    plx.pose_step(dev(H, torch.float64), dev(b, torch.float64), pose, damping=0.01,
                  xi_out=xi, status=st)
    torch.cuda.synchronize()
    assert st.item() == 0
    np.testing.assert_allclose(xi.cpu().numpy(), ref_xi, rtol=1e-12, atol=1e-15)
    np.testing.assert_allclose(pose.cpu().numpy().reshape(3, 4), ref_T, atol=1e-13)
    # not positive definite: status 1, pose untouched
    pose2 = dev(T0.reshape(12), torch.float64)
    plx.pose_step(dev(-np.eye(6), torch.float64), dev(b, torch.float64), pose2, status=st)
    torch.cuda.synchronize()
    assert st.item() == 1
    np.testing.assert_array_equal(pose2.cpu().numpy().reshape(3, 4), T0)


def test_pose_step_lm_matches_oracle_sequence():
    """A sequence of Levenberg-Marquardt calls with losses going down and up
    (accept, reject and restore, accept) against the oracle's, call by call."""
    rng = np.random.default_rng(21)
    T = scenes.look_at((1.0, 0.4, -2.0), (0, 0, 0))
    st_ref = np.zeros(64)
    st = torch.zeros(64, device="cuda", dtype=torch.float64)
    pose = dev(T.reshape(12), torch.float64)
    xi = torch.empty(6, device="cuda", dtype=torch.float64)
    status = torch.empty(1, device="cuda", dtype=torch.int32)
    T_ref = T.copy()
    statuses = []
    for k, L in enumerate([1.0, 0.8, 0.9, 0.95, 0.5, 0.5, 0.7, 0.2]):
        A = rng.standard_normal((9, 6))
        H = A.T @ A + 0.05 * np.eye(6)
        b = 0.1 * rng.standard_normal(6)
        T_ref, xi_ref, s_ref = oracle.pose_step_lm(H, b, L, st_ref, T_ref, 1e-2, 4.0)
        plx.pose_step_lm(dev(H, torch.float64), dev(b, torch.float64),
                         dev(np.array([L, 10.0]), torch.float64), st, pose, 1e-2, 4.0,
                         xi_out=xi, status=status)
        torch.cuda.synchronize()
        assert status.item() == s_ref
        statuses.append(s_ref)
        np.testing.assert_allclose(xi.cpu().numpy(), xi_ref, rtol=1e-11, atol=1e-15)
        np.testing.assert_allclose(pose.cpu().numpy().reshape(3, 4), T_ref, atol=1e-13)
        np.testing.assert_allclose(st.cpu().numpy(), st_ref, rtol=1e-11, atol=1e-15)
    assert 0 in statuses and 2 in statuses


def test_lm_tracking_loop_in_a_cuda_graph_converges(sphere):
    """The damped loop (pose Jacobian + LM step) in one CUDA graph."""
    g, cam, _, opts = sphere
    opts = dict(opts, depth_is_z=False)
    ref_t = oracle.render(g, [cam], opts)
    T0 = scenes.perturb_pose(cam.T_wc, 0.03, 2.0, np.random.default_rng(9))
    case = GpuCase(g, [cam.with_pose(T0)])
    o = plx.opts_from_dict(opts)
    rgb_t, depth_t = dev(ref_t.rgb), dev(ref_t.depth)
    H = torch.empty(6, 6, device="cuda", dtype=torch.float64)
    b = torch.empty(6, device="cuda", dtype=torch.float64)
    loss = torch.empty(2, device="cuda", dtype=torch.float64)
    st = plx.lm_state()
    pose = case.cams.poses[0]
    plx.render_backward_pose(case.grid, case.cams, 0, o, rgb_t, depth_t, out=(H, b, loss))
    plx.pose_step_lm(H, b, loss, st, pose)
    torch.cuda.synchronize()
    pose.copy_(dev(T0.reshape(12), torch.float64))
    st.zero_()
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph, stream=s):
        for _ in range(60):
            plx.render_backward_pose(case.grid, case.cams, 0, o, rgb_t, depth_t, out=(H, b, loss))
            plx.pose_step_lm(H, b, loss, st, pose)
    graph.replay()
    torch.cuda.synchronize()
    T = pose.cpu().numpy().reshape(3, 4)
    assert np.abs(T - cam.T_wc).max() < 1e-4 * np.abs(T0 - cam.T_wc).max()


def test_tracking_loop_in_a_cuda_graph_converges(sphere):
    """100 GN iterations (pose Jacobian + step) captured in one CUDA graph
    bring a 3 cm / 2 deg perturbed pose back to the rendering pose."""
    g, cam, _, opts = sphere
    opts = dict(opts, depth_is_z=False)
    ref_t = oracle.render(g, [cam], opts)
    T0 = scenes.perturb_pose(cam.T_wc, 0.03, 2.0, np.random.default_rng(9))
    case = GpuCase(g, [cam.with_pose(T0)])
    o = plx.opts_from_dict(opts)
    rgb_t, depth_t = dev(ref_t.rgb), dev(ref_t.depth)
    H = torch.empty(6, 6, device="cuda", dtype=torch.float64)
    b = torch.empty(6, device="cuda", dtype=torch.float64)
    loss = torch.empty(2, device="cuda", dtype=torch.float64)
    pose = case.cams.poses[0]
    # warm-up outside capture (loads the kernels), then restore the pose
    plx.render_backward_pose(case.grid, case.cams, 0, o, rgb_t, depth_t, out=(H, b, loss))
    plx.pose_step(H, b, pose)
    torch.cuda.synchronize()
    pose.copy_(dev(T0.reshape(12), torch.float64))
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph, stream=s):
        for _ in range(100):
            plx.render_backward_pose(case.grid, case.cams, 0, o, rgb_t, depth_t, out=(H, b, loss))
            plx.pose_step(H, b, pose)
    graph.replay()
    torch.cuda.synchronize()
    T = pose.cpu().numpy().reshape(3, 4)
    err0 = np.abs(T0 - cam.T_wc).max()
    assert np.abs(T - cam.T_wc).max() < 1e-4 * err0
    assert loss[0].item() < 1e-10


# ------------------------------------------------------------ 16-bit storage
@pytest.mark.parametrize("storage", ["bf16", "f16", "f32_bf16"])
def test_16bit_storage_error(sphere, storage):
    g, cam, _, opts = sphere
    case = GpuCase(g, [cam], storage=storage)
    got = case.forward(opts, counts=False)
    ref = oracle.render(g, [cam], opts)
    assert rel_err(got["rgb"], ref.rgb) <= 2e-3
    # against the oracle on the same rounded values the kernel error is FP32-level
    tdt = {"bf16": torch.bfloat16, "f16": torch.float16, "f32_bf16": torch.bfloat16}[storage]
    dens = torch.from_numpy(g.density)
    if storage != "f32_bf16":
        dens = dens.to(tdt).float()
    sh = torch.from_numpy(g.sh).to(tdt).float()
    gr = g.with_values(dens.numpy(), sh.numpy())
    ref_r = oracle.render(gr, [cam], opts)
    assert rel_err(got["rgb"], ref_r.rgb) <= TOL_FWD
    assert rel_err(got["depth"], ref_r.depth) <= TOL_FWD
    d2, s2 = case.grid.download()
    np.testing.assert_array_equal(d2.cpu().numpy(), gr.density)
    np.testing.assert_array_equal(s2.cpu().numpy(), gr.sh)


@pytest.mark.parametrize("cache_cap", [None, 256])
@pytest.mark.parametrize("storage", ["bf16", "f16", "f32_bf16"])
def test_16bit_storage_adjoint_and_pose(sphere, storage, cache_cap):
    """Grid adjoint and pose system with 16-bit storage against the oracle on
    the same rounded values: FP32-level agreement (the kernels decode the
    records exactly; only the rounding of the stored values differs from
    FP32 storage)."""
    g, cam, gp, opts = sphere
    opts = dict(opts, depth_is_z=False, lambda_d=0.7)
    tdt = {"bf16": torch.bfloat16, "f16": torch.float16, "f32_bf16": torch.bfloat16}[storage]
    dens = torch.from_numpy(g.density)
    if storage != "f32_bf16":
        dens = dens.to(tdt).float()
    gr = g.with_values(dens.numpy(), torch.from_numpy(g.sh).to(tdt).float().numpy())
    tg = oracle.render(gp, [cam], opts)
    rgb_t, depth_t = tg.rgb.astype(np.float32), tg.depth.astype(np.float32)
    case = GpuCase(g, [cam], storage=storage)
    gd, gs, _, loss = case.backward_grid(opts, rgb_t, depth_t, cache_cap=cache_cap)
    ref = oracle.grad_grid(gr, [cam], opts, rgb_t, depth_t)
    assert loss[1] == ref.M and abs(loss[0] - ref.loss) <= 1e-5 * ref.loss
    assert norm_err(gd, ref.grad_density) <= TOL_GRAD
    assert norm_err(gs, ref.grad_sh) <= TOL_GRAD
    T0 = scenes.perturb_pose(cam.T_wc, 0.02, 1.0, np.random.default_rng(3))
    case.cams.poses.copy_(torch.tensor(T0.reshape(1, 12), device="cuda"))
    H, b, _ = case.backward_pose(opts, 0, rgb_t, depth_t)
    rp = oracle.pose_jacobian(gr, [cam.with_pose(T0)], opts, rgb_t, depth_t)
    assert norm_err(H, rp.H) <= TOL_GRAD and norm_err(b, rp.b) <= TOL_GRAD


@pytest.mark.parametrize("cache_cap", [None, 256])
def test_stop_T_forward_adjoint_and_pose(sphere, cache_cap):
    """Early termination (stop_T > 0): every kernel ends a ray after the
    sample that takes T below stop_T, as the oracle does; the grid adjoint
    with and without a sample cache, and the pose Jacobian (which then takes
    its thread-per-ray form)."""
    g, cam, gp, opts = sphere
    opts = dict(opts, depth_is_z=False, lambda_d=0.7, stop_T=0.02)
    case = GpuCase(g, [cam])
    got = case.forward(opts)
    ref = oracle.render(g, [cam], opts)
    full = oracle.render(g, [cam], dict(opts, stop_T=0.0))
    assert (ref.n_marched < full.n_marched).mean() > 0.2   # the stop does bite
    np.testing.assert_array_equal(got["counts"][:, 0], ref.n_marched)
    assert rel_err(got["rgb"], ref.rgb) <= TOL_FWD
    assert rel_err(got["depth"], ref.depth) <= TOL_FWD
    tg = oracle.render(gp, [cam], opts)
    rgb_t, depth_t = tg.rgb.astype(np.float32), tg.depth.astype(np.float32)
    gd, gs, _, loss = case.backward_grid(opts, rgb_t, depth_t, cache_cap=cache_cap)
    rg = oracle.grad_grid(g, [cam], opts, rgb_t, depth_t)
    assert loss[1] == rg.M and abs(loss[0] - rg.loss) <= 1e-5 * rg.loss
    assert norm_err(gd, rg.grad_density) <= TOL_GRAD
    assert norm_err(gs, rg.grad_sh) <= TOL_GRAD
    T0 = scenes.perturb_pose(cam.T_wc, 0.02, 1.0, np.random.default_rng(4))
    case.cams.poses.copy_(torch.tensor(T0.reshape(1, 12), device="cuda"))
    H, b, _ = case.backward_pose(opts, 0, rgb_t, depth_t)
    rp = oracle.pose_jacobian(g, [cam.with_pose(T0)], opts, rgb_t, depth_t)
    assert norm_err(H, rp.H) <= TOL_GRAD and norm_err(b, rp.b) <= TOL_GRAD


def test_upload_replaces_values(sphere):
    g, cam, gp, opts = sphere
    case = GpuCase(g, [cam])
    case.grid.upload(dev(gp.density), dev(gp.sh))
    got = case.forward(opts, counts=False)
    ref = oracle.render(gp, [cam], opts)
    assert rel_err(got["rgb"], ref.rgb) <= TOL_FWD


@pytest.mark.parametrize("width,height", [(128, 128), (128, 130)])
def test_warp_per_ray_threshold(width, height):
    """16,384 rays take the warp-per-ray forward and adjoint (a warp marches
    segments of one ray and composes them by a scan), 16,640 the
    one-ray-per-thread kernels: both against the oracle, FP32 bounds."""
    g, cam0, gp = scenes.sphere_scene(width=width, height=height, f=120.0)
    opts = dict(step=0.5 * g.h[0], lambda_d=0.7, bg=(0.1, 0.2, 0.3), depth_is_z=False)
    tg = oracle.render(gp, [cam0], opts)
    rgb_t, depth_t = tg.rgb.astype(np.float32), tg.depth.astype(np.float32)
    case = GpuCase(g, [cam0])
    got = case.forward(opts)
    ref = oracle.render(g, [cam0], opts)
    assert rel_err(got["rgb"], ref.rgb) <= TOL_FWD
    assert rel_err(got["depth"], ref.depth) <= TOL_FWD
    np.testing.assert_array_equal(got["counts"][:, 0], ref.n_marched)
    np.testing.assert_array_equal(got["counts"][:, 1], ref.n_alloc)
    gd, gs, _, loss = case.backward_grid(opts, rgb_t, depth_t)
    rg = oracle.grad_grid(g, [cam0], opts, rgb_t, depth_t)
    assert loss[1] == rg.M and abs(loss[0] - rg.loss) <= 1e-5 * rg.loss
    assert norm_err(gd, rg.grad_density) <= TOL_GRAD
    assert norm_err(gs, rg.grad_sh) <= TOL_GRAD
    case.close()


# ------------------------------------------------ full-size room, sampled
@pytest.fixture(scope="module")
def room256():
    R, occ, npr, seed = scenes.WORKLOADS["room256"]
    sc = scenes.room_scene(R, occ, npr, seed)
    cams = scenes.room_cameras(sc, 8, seed + 1)
    rgb_t, depth_t = scenes.sensor_frames(sc, cams, seed + 2)
    opts = dict(step=0.5 * sc.grid.h[0], lambda_d=1.0, depth_is_z=True)
    return sc.grid, cams, rgb_t, depth_t, opts


def test_room256_dense_forward_sampled_against_oracle(room256):
    """The bench's launch configuration (dense, 8 x 640x480, FP32 storage):
    1024 sampled rays against the oracle."""
    g, cams, _, _, opts = room256
    case = GpuCase(g, cams)
    got = case.forward(opts)
    cid, pix = scenes.random_rays(cams, 1024, 99)
    rows = np.array([sum(c.width * c.height for c in cams[:k]) for k in range(len(cams))])[cid] + pix
    ref = oracle.render(g, cams, opts, rays=(cid, pix))
    assert rel_err(got["rgb"][rows], ref.rgb) <= TOL_FWD
    assert rel_err(got["depth"][rows], ref.depth) <= TOL_FWD
    assert np.mean(got["counts"][rows, 0] == ref.n_marched) >= 0.999
    assert np.mean(got["counts"][rows, 1] == ref.n_alloc) >= 0.999
    assert ref.n_alloc.mean() > 5


def test_room256_backward_sampled_and_partition(room256):
    g, cams, rgb_t, depth_t, opts = room256
    case = GpuCase(g, cams)
    cid, pix = scenes.random_rays(cams, 384, 7)
    rows = np.array([sum(c.width * c.height for c in cams[:k]) for k in range(len(cams))])[cid] + pix
    gd, gs, _, loss = case.backward_grid(opts, rgb_t[rows], depth_t[rows], rays=(cid, pix))
    ref = oracle.grad_grid(g, cams, opts, rgb_t[rows], depth_t[rows], rays=(cid, pix))
    assert loss[1] == ref.M
    assert abs(loss[0] - ref.loss) <= 1e-5 * ref.loss
    assert norm_err(gd, ref.grad_density) <= TOL_GRAD
    assert norm_err(gs, ref.grad_sh) <= TOL_GRAD
    # dense launch over all 2.46M rays = the sum over a partition in two lists
    gdd, gsd, _, ld = case.backward_grid(opts, rgb_t, depth_t)
    allc, allp = scenes.dense_rays(cams)
    half = allc.shape[0] // 2
    parts = []
    for sl in (slice(0, half), slice(half, None)):
        parts.append(case.backward_grid(opts, rgb_t[sl], depth_t[sl], rays=(allc[sl], allp[sl])))
    comb = sum(p[0] * p[3][1] for p in parts) / ld[1]
    assert ld[1] == parts[0][3][1] + parts[1][3][1]
    assert norm_err(gdd, comb) <= 1e-5
    assert abs(ld[0] * ld[1] - sum(p[3][0] * p[3][1] for p in parts)) <= 1e-9 * ld[0] * ld[1]


@pytest.fixture(scope="module")
def room512():
    R, occ, npr, seed = scenes.WORKLOADS["room512"]
    sc = scenes.workload_scene("room512")
    cam = scenes.room_cameras(sc, 1, seed + 1)[0]
    rgb_t, depth_t = scenes.sensor_frames(sc, [cam], seed + 2)
    opts = dict(step=0.5 * sc.grid.h[0], lambda_d=1.0, depth_is_z=True)
    return sc.grid, cam, rgb_t, depth_t, opts


def test_room512_forward_and_pose_sampled_against_oracle(room512):
    """512^3 grid, one 640x480 frame: the dense launch's sampled outputs and
    the pose system of 512 sampled pixels against the oracle."""
    g, cam, rgb_t, depth_t, opts = room512
    case = GpuCase(g, [cam])
    got = case.forward(opts)
    pix = np.random.default_rng(4).permutation(cam.width * cam.height)[:512].astype(np.int32)
    ref = oracle.render(g, [cam], opts, rays=(np.zeros(512, np.int32), pix))
    assert rel_err(got["rgb"][pix], ref.rgb) <= TOL_FWD
    assert rel_err(got["depth"][pix], ref.depth) <= TOL_FWD
    H, b, loss = case.backward_pose(opts, 0, rgb_t[pix], depth_t[pix], pixels=pix)
    rp = oracle.pose_jacobian(g, [cam], opts, rgb_t[pix], depth_t[pix],
                              rays=(np.zeros(512, np.int32), pix))
    assert loss[1] == rp.M
    assert abs(loss[0] - rp.loss) <= 1e-5 * rp.loss
    assert norm_err(H, rp.H) <= TOL_GRAD
    assert norm_err(b, rp.b) <= TOL_GRAD
    # dense launch over the whole frame = M-weighted sum over a pixel partition
    Hd, bd, ld = case.backward_pose(opts, 0, rgb_t, depth_t)
    allp = np.arange(cam.width * cam.height, dtype=np.int32)
    acc_H, acc_b, acc_M = 0.0, 0.0, 0.0
    for part in np.array_split(allp, 3):
        Hp, bp, lp = case.backward_pose(opts, 0, rgb_t[part], depth_t[part], pixels=part)
        acc_H, acc_b, acc_M = acc_H + Hp * lp[1], acc_b + bp * lp[1], acc_M + lp[1]
    assert ld[1] == acc_M
    assert norm_err(Hd * ld[1], acc_H) <= 1e-9
    assert norm_err(bd * ld[1], acc_b) <= 1e-9


@pytest.mark.parametrize("cache_cap", [None, 64])
def test_no_valid_target_depth(cache_cap):
    """Degenerate targets: every depth missing (0, NaN or negative), so M = 0
    rays enter the loss (Eq. 4-5, 11). The oracle then gives loss 0 and zero
    gradients; the grid adjoint, the pose system and the batched launch must
    agree (no division by M = 0), and a Gauss-Newton step on the zero system
    reports it as not positive definite and leaves the pose alone."""
    g = scenes.tiny_grid(7, seed=5, alloc_frac=0.7, sigma_mean=2.0, sigma_std=2.0)
    cams = tiny_cams()
    opts = dict(step=0.1, bg=(0.2, 0.1, 0.3), lambda_d=0.5)
    case = GpuCase(g, cams)
    n = case.cams.n_pixels()
    rng = np.random.default_rng(3)
    rgb_t = rng.uniform(0, 1, (n, 3)).astype(np.float32)
    depth_t = np.zeros(n, np.float32)
    depth_t[1::3] = np.nan
    depth_t[2::3] = -1.0
    ref = oracle.grad_grid(g, cams, opts, rgb_t, depth_t)
    assert ref.M == 0 and ref.loss == 0.0
    gd, gs, gpad, loss = case.backward_grid(opts, rgb_t, depth_t, cache_cap=cache_cap)
    assert loss[0] == 0.0 and loss[1] == 0.0
    assert not gd.any() and not gs.any() and not gpad.any()
    w0 = cams[0].width * cams[0].height
    H, b, ploss = case.backward_pose(opts, 0, rgb_t[:w0], depth_t[:w0])
    rp = oracle.pose_jacobian(g, [cams[0]], opts, rgb_t[:w0], depth_t[:w0])
    assert rp.M == 0 and not rp.H.any() and not rp.b.any()
    assert not H.any() and not b.any() and ploss[0] == 0.0 and ploss[1] == 0.0
    pose = case.cams.poses[0].clone()
    st = torch.full((1,), 7, device="cuda", dtype=torch.int32)
    plx.pose_step(dev(H, torch.float64), dev(b, torch.float64), pose, status=st)
    torch.cuda.synchronize()
    assert st.item() == 1
    assert torch.equal(pose, case.cams.poses[0])
    o = plx.opts_from_dict(opts)
    if cache_cap is not None:
        o = plx.SampleCache.for_batch(cache_cap).opts(o)
    work = [(0, plx.WORK_MAP), (1, plx.WORK_TRACK), (1, plx.WORK_MAP)]
    sizes = [cams[c].width * cams[c].height for c, _ in work]
    rows = int(sum(sizes))
    bt_rgb = rng.uniform(0, 1, (rows, 3)).astype(np.float32)
    bt_depth = np.zeros(rows, np.float32)
    grad, mloss, Hb, bb, tloss = plx.render_batch(case.grid, case.cams, work, o, dev(bt_rgb),
                                                  dev(bt_depth))
    torch.cuda.synchronize()
    case.grid.check()
    assert mloss.cpu().tolist() == [0.0, 0.0]
    assert not grad.any().item()
    assert not Hb.any().item() and not bb.any().item()
    assert tloss.cpu().tolist() == [[0.0, 0.0]]
