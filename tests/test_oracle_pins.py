"""Pins of the FP64 oracle against what the paper and mathematics fix.

None of these compares the oracle with itself: each checks it against a closed
form, an invariant, a library routine on an independent formulation, or finite
differences of its own forward (which the closed forms pin in turn).
Arithmetic cited: arXiv 2307.03404, Sec. 4 Eq. 1-3, Sec. 5.2 Eq. 4-11,
Sec. 5.3 Eq. 12-14, Appendix A Eq. 15-16.
"""
import math

import numpy as np
import pytest
import scipy.linalg

import oracle
from paper_2307_03404_b300 import scenes

Y00 = 0.28209479177387814  # 1 / (2 sqrt(pi)), the constant real SH of degree 0


def axis_camera(ox=0.1, oy=0.2, oz=-3.0):
    """1x1-pixel camera at (ox, oy, oz) whose only ray points along +z."""
    T = np.array([[1.0, 0, 0, ox], [0, 1.0, 0, oy], [0, 0, 1.0, oz]])
    return scenes.Camera(1.0, 1.0, 0.5, 0.5, 1, 1, T)


# ------------------------------------------------------- compositing, Eq. 1-3
def slab_expected(sigma, c, bg, t_min, step, n):
    q = math.exp(-sigma * step)
    L = n * step
    C = (1 - math.exp(-sigma * L)) * np.asarray(c) + math.exp(-sigma * L) * np.asarray(bg)
    t0 = t_min + 0.5 * step
    s1 = q * (1 - n * q ** (n - 1) + (n - 1) * q ** n) / (1 - q) ** 2
    D = t0 * (1 - q ** n) + step * (1 - q) * s1
    return C, D


@pytest.mark.parametrize("sigma", [0.3, 2.0, 7.5])
def test_constant_slab_closed_form(sigma):
    """A ray through a constant-density cube: C = (1-e^{-sigma L}) c + e^{-sigma L} bg
    and D = a geometric series (Eq. 1-3 telescoped)."""
    k = np.array([0.7, -0.4, 1.3])
    g = scenes.constant_grid(8, sigma, k)
    bg = (0.2, 0.5, 0.9)
    opts = dict(step=0.15, bg=bg, color_act="identity")
    r = oracle.render(g, [axis_camera()], opts)
    n = math.floor(2.0 / 0.15)
    assert r.n_marched[0] == n
    sigma = float(g.density[0])                       # the stored (float32) values
    k = g.sh[0, [0, 9, 18]].astype(np.float64)
    C, D = slab_expected(sigma, Y00 * k, bg, 2.0, 0.15, n)
    np.testing.assert_allclose(r.rgb[0], C, rtol=1e-12, atol=1e-14)
    np.testing.assert_allclose(r.depth[0], D, rtol=1e-12)
    np.testing.assert_allclose(r.T_final[0], math.exp(-sigma * n * 0.15), rtol=1e-12)


def test_slab_sigmoid_and_caps():
    """Sigmoid colour; max_samples caps N; stop_T ends the march after the
    first sample whose T_{i+1} falls below it."""
    k = np.array([0.7, -0.4, 1.3])
    sig = 2.0
    g = scenes.constant_grid(8, sig, k)
    k = g.sh[0, [0, 9, 18]].astype(np.float64)
    c = 1 / (1 + np.exp(-Y00 * k))
    r = oracle.render(g, [axis_camera()], dict(step=0.15, max_samples=5))
    C, D = slab_expected(sig, c, (0, 0, 0), 2.0, 0.15, 5)
    np.testing.assert_allclose(r.rgb[0], C, rtol=1e-12)
    np.testing.assert_allclose(r.depth[0], D, rtol=1e-12)
    stop = 0.37
    q = math.exp(-sig * 0.15)
    n_stop = math.floor(math.log(stop) / math.log(q)) + 1
    r = oracle.render(g, [axis_camera()], dict(step=0.15, stop_T=stop))
    assert r.n_marched[0] == n_stop
    C, D = slab_expected(sig, c, (0, 0, 0), 2.0, 0.15, n_stop)
    np.testing.assert_allclose(r.rgb[0], C, rtol=1e-12)


def test_opaque_layer_depth_is_first_hit():
    """Huge density from one vertex layer on: all weight falls on the first
    sample with sigma > 0, so D is that sample's t."""
    R = 9
    g = scenes.constant_grid(R, 0.0, (1.0, 1.0, 1.0))
    dens = np.zeros((R, R, R), np.float32)
    dens[5:] = 1e5                    # z index >= 5, i.e. z >= 0.25
    g = g.with_values(dens.reshape(-1), g.sh)
    r = oracle.render(g, [axis_camera()], dict(step=0.15, color_act="identity"))
    # samples z_k = -1 + (k + 1/2) 0.15; the first with z > 0 is k = 7
    np.testing.assert_allclose(r.depth[0], 2.0 + 7.5 * 0.15, rtol=1e-12)
    np.testing.assert_allclose(r.rgb[0], Y00 * np.ones(3), rtol=1e-12)


def test_zero_density_and_miss_give_background():
    g = scenes.constant_grid(6, 0.0, (0.3, 0.3, 0.3))
    bg = (0.25, 0.5, 0.75)
    r = oracle.render(g, [axis_camera()], dict(step=0.1, bg=bg))
    np.testing.assert_array_equal(r.rgb[0], bg)
    assert r.depth[0] == 0.0
    g2 = scenes.constant_grid(6, 5.0, (0.3, 0.3, 0.3))
    away = axis_camera(0.0, 0.0, 3.0)  # in front of the box, looking away from it
    r = oracle.render(g2, [away], dict(step=0.1, bg=bg))
    assert r.n_marched[0] == 0
    np.testing.assert_array_equal(r.rgb[0], bg)
    beside = axis_camera(1.5, 0.0, -3.0)  # parallel to the box, outside it
    r = oracle.render(g2, [beside], dict(step=0.1, bg=bg))
    assert r.n_marched[0] == 0


def test_weights_sum_to_one_minus_final_transmittance():
    """With c = 1 and bg = 0, C = sum_i w_i = 1 - T_{N+1} <= 1 (Eq. 1-2)."""
    g, cam, _ = scenes.sphere_scene()
    sh = np.zeros_like(g.sh)
    sh[:, [0, 9, 18]] = 1.0 / Y00
    g1 = g.with_values(g.density, sh)
    r = oracle.render(g1, [cam], dict(step=0.5 * g.h[0], color_act="identity"))
    c = Y00 * float(sh[0, 0])         # 1 up to the float32 rounding of 1 / Y00
    assert np.all((r.T_final >= 0) & (r.T_final <= 1))
    np.testing.assert_allclose(r.rgb, c * np.repeat(1 - r.T_final[:, None], 3, 1), atol=1e-12)
    assert r.rgb.max() <= c * (1 + 1e-12)
    assert (r.T_final < 0.01).any() and (r.T_final == 1).any()


def test_link_relabelling_leaves_render_unchanged():
    g = scenes.tiny_grid(6, seed=3, alloc_frac=0.7)
    cam = scenes.Camera(6.0, 6.0, 4.0, 3.0, 8, 6, scenes.look_at((2.0, 1.5, -2.5), (0, 0, 0)))
    opts = dict(step=0.2)
    r0 = oracle.render(g, [cam], opts)
    perm = np.random.default_rng(0).permutation(g.n_alloc)
    inv = np.empty_like(perm)
    inv[perm] = np.arange(g.n_alloc)
    links = np.where(g.links >= 0, inv[np.maximum(g.links, 0)], -1).astype(np.int32)
    g2 = scenes.Grid(g.res, g.lo, g.hi, links, g.density[perm], g.sh[perm])
    r1 = oracle.render(g2, [cam], opts)
    np.testing.assert_array_equal(r0.rgb, r1.rgb)
    np.testing.assert_array_equal(r0.depth, r1.depth)


# --------------------------------------------------------------- SH, Sec. 5.2
def test_sh_basis_orthonormal_by_quadrature():
    mu, wmu = np.polynomial.legendre.leggauss(12)
    nphi = 24
    G = np.zeros((9, 9))
    for m, wm in zip(mu, wmu):
        s = math.sqrt(1 - m * m)
        for j in range(nphi):
            ph = 2 * math.pi * j / nphi
            Y = oracle.sh_basis([s * math.cos(ph), s * math.sin(ph), m])
            G += wm * (2 * math.pi / nphi) * np.outer(Y, Y)
    np.testing.assert_allclose(G, np.eye(9), atol=1e-13)


def test_sh_basis_order_and_parity():
    """Order (1; y, z, x; xy, yz, 3z^2-1, xz, x^2-y^2): the degree-1 terms are
    the coordinates, the degree-2 terms even."""
    d = np.array([0.36, -0.48, 0.8])
    Y = oracle.sh_basis(d)
    Yn = oracle.sh_basis(-d)
    np.testing.assert_allclose(Y[1:4], -Yn[1:4])
    np.testing.assert_allclose(Y[[0, 4, 5, 6, 7, 8]], Yn[[0, 4, 5, 6, 7, 8]])
    k1 = math.sqrt(3 / (4 * math.pi))
    np.testing.assert_allclose(Y[1:4], k1 * d[[1, 2, 0]], rtol=1e-14)
    assert Y[0] == pytest.approx(Y00, rel=1e-15)


# ----------------------------------------------------- trilinear, App. A
def test_trilerp_matches_appendix_A_linear_system():
    """Solve the 8x8 system of Eq. 15 at arbitrary lattice points with numpy,
    evaluate the polynomial and its Eq. 16 derivatives, compare."""
    rng = np.random.default_rng(7)
    for _ in range(20):
        p0 = rng.uniform(-2, 2, 3)
        p1 = p0 + rng.uniform(0.2, 1.5, 3)
        V = rng.standard_normal(8)
        rows = []
        for c in range(8):
            x, y, z = [(p1 if (c >> a) & 1 else p0)[a] for a in range(3)]
            rows.append([1, x, y, z, x * y, x * z, y * z, x * y * z])
        a = np.linalg.solve(np.array(rows), V)
        q = p0 + rng.uniform(0, 1, 3) * (p1 - p0)
        x, y, z = q
        f_ref = a @ [1, x, y, z, x * y, x * z, y * z, x * y * z]
        g_ref = np.array([a[1] + a[4] * y + a[5] * z + a[7] * y * z,
                          a[2] + a[4] * x + a[6] * z + a[7] * x * z,
                          a[3] + a[5] * x + a[6] * y + a[7] * x * y])
        loc = (q - p0) / (p1 - p0)
        f, g = oracle.trilerp(V, *loc)
        assert f == pytest.approx(f_ref, rel=1e-10, abs=1e-10)
        np.testing.assert_allclose(g / (p1 - p0), g_ref, rtol=1e-9, atol=1e-9)


def test_trilerp_reproduces_affine_fields_and_corners():
    rng = np.random.default_rng(8)
    a0, b = rng.standard_normal(), rng.standard_normal(3)
    V = [a0 + b @ [c & 1, (c >> 1) & 1, (c >> 2) & 1] for c in range(8)]
    for _ in range(10):
        x = rng.uniform(0, 1, 3)
        f, g = oracle.trilerp(V, *x)
        assert f == pytest.approx(a0 + b @ x, abs=1e-14)
        np.testing.assert_allclose(g, b, atol=1e-14)
    W = rng.standard_normal(8)
    for c in range(8):
        f, _ = oracle.trilerp(W, c & 1, (c >> 1) & 1, (c >> 2) & 1)
        assert f == pytest.approx(W[c], abs=1e-14)


# ------------------------------------------------------------ camera rays
def test_pixel_ray_reprojects_to_pixel_centre():
    g = scenes.constant_grid(4, 0.0, (0, 0, 0))
    T = scenes.perturb_pose(scenes.look_at((0.3, 0.4, -2.5), (0.1, 0, 0)), 0.2, 15.0,
                            np.random.default_rng(1))
    cam = scenes.Camera(50.0, 47.0, 15.3, 11.1, 32, 24, T)
    R, o_ref = T[:, :3], T[:, 3]
    for pix in [0, 31, 32 * 5 + 7, 32 * 24 - 1]:
        u, v = pix % 32, pix // 32
        o, d, dcn, tr, hit = oracle.pixel_ray(g, cam, pix)
        np.testing.assert_allclose(o, o_ref)
        assert np.linalg.norm(d) == pytest.approx(1.0, abs=1e-15)
        q = R.T @ (o + 2.7 * d - o)
        assert cam.fx * q[0] / q[2] + cam.cx == pytest.approx(u + 0.5, abs=1e-12)
        assert cam.fy * q[1] / q[2] + cam.cy == pytest.approx(v + 0.5, abs=1e-12)
        assert q[2] * dcn == pytest.approx(2.7, abs=1e-12)  # z-depth * |d_c| = t
        if hit:
            eps = 1e-9
            assert np.all(np.abs(o + (tr[0] + eps) * d) <= 1 + 1e-12)
            assert np.all(np.abs(o + (tr[1] - eps) * d) <= 1 + 1e-12)
            assert np.any(np.abs(o + (tr[0] - 1e-6) * d) > 1)
            assert np.any(np.abs(o + (tr[1] + 1e-6) * d) > 1)


# --------------------------------------------- losses and grid adjoint, Eq. 4-11
def fd_setup(seed=5, alloc_frac=0.8):
    g = scenes.tiny_grid(5, seed=seed, alloc_frac=alloc_frac, sigma_mean=3.0, sigma_std=0.5)
    g = g.with_values(np.abs(g.density).astype(np.float64), g.sh.astype(np.float64))
    cam = scenes.Camera(6.0, 6.0, 4.0, 3.0, 8, 6, scenes.look_at((2.2, 1.4, -2.6), (0, 0.1, 0)))
    rng = np.random.default_rng(seed + 100)
    n = 48
    rgb_t = rng.uniform(0, 1, (n, 3))
    depth_t = rng.uniform(1.5, 3.5, n)
    depth_t[5] = 0.0
    depth_t[17] = np.nan
    return g, cam, rgb_t, depth_t


def ray_dc_norm(cam, pix):
    u, v = pix % cam.width, pix // cam.width
    return math.sqrt(((u + 0.5 - cam.cx) / cam.fx) ** 2 + ((v + 0.5 - cam.cy) / cam.fy) ** 2 + 1)


def brute_loss(cam, r, rgb_t, depth_t, lam, depth_is_z=True):
    tot, M = 0.0, 0
    for i in range(len(depth_t)):
        dz = depth_t[i]
        if not (np.isfinite(dz) and dz > 0):
            continue
        M += 1
        Dt = dz * ray_dc_norm(cam, i) if depth_is_z else dz
        tot += sum((r.rgb[i, ch] - rgb_t[i, ch]) ** 2 for ch in range(3))
        tot += lam * (r.depth[i] - Dt) ** 2
    return tot / M, M


@pytest.mark.parametrize("act,depth_is_z", [("sigmoid", True), ("identity", False)])
def test_loss_matches_brute_force(act, depth_is_z):
    g, cam, rgb_t, depth_t = fd_setup()
    opts = dict(step=0.25, bg=(0.1, 0.2, 0.3), lambda_d=0.7, color_act=act,
                depth_is_z=depth_is_z)
    r = oracle.render(g, [cam], opts)
    ref, M = brute_loss(cam, r, rgb_t, depth_t, 0.7, depth_is_z)
    gg = oracle.grad_grid(g, [cam], opts, rgb_t, depth_t)
    pj = oracle.pose_jacobian(g, [cam], opts, rgb_t, depth_t)
    assert gg.M == M == pj.M == 46
    assert gg.loss == pytest.approx(ref, rel=1e-12)
    assert pj.loss == pytest.approx(ref, rel=1e-12)


@pytest.mark.parametrize("act,alloc,bg", [("sigmoid", 0.8, (0.1, 0.2, 0.3)),
                                          ("identity", 1.0, (0.0, 0.0, 0.0)),
                                          ("sigmoid", 0.6, (0.9, 0.1, 0.5))])
def test_grid_gradient_matches_finite_differences(act, alloc, bg):
    """Eq. 8-10 (with the inclusive prefix and the background term) chained
    through activation, SH and trilinear weights equal central differences of
    the loss computed from the forward."""
    g, cam, rgb_t, depth_t = fd_setup(alloc_frac=alloc)
    opts = dict(step=0.25, bg=bg, lambda_d=0.7, color_act=act)
    gg = oracle.grad_grid(g, [cam], opts, rgb_t, depth_t)

    def loss(dens, sh):
        return brute_loss(cam, oracle.render(g.with_values(dens, sh), [cam], opts),
                          rgb_t, depth_t, 0.7)[0]

    rng = np.random.default_rng(11)
    eps = 1e-6
    idx_d = rng.choice(g.n_alloc, 12, replace=False)
    fd, an = [], []
    for i in idx_d:
        dp, dm = g.density.copy(), g.density.copy()
        dp[i] += eps
        dm[i] -= eps
        fd.append((loss(dp, g.sh) - loss(dm, g.sh)) / (2 * eps))
        an.append(gg.grad_density[i])
    for _ in range(24):
        i, j = rng.integers(g.n_alloc), rng.integers(27)
        sp, sm = g.sh.copy(), g.sh.copy()
        sp[i, j] += eps
        sm[i, j] -= eps
        fd.append((loss(g.density, sp) - loss(g.density, sm)) / (2 * eps))
        an.append(gg.grad_sh[i, j])
    fd, an = np.array(fd), np.array(an)
    assert np.abs(an).max() > 1e-4
    assert np.abs(fd - an).max() <= 1e-6 * np.abs(an).max()


def test_grid_gradient_of_relu_clipped_density_is_zero():
    """Vertices whose every sample has f_sigma <= 0 receive no density gradient."""
    g, cam, rgb_t, depth_t = fd_setup()
    dens = -np.abs(g.density)
    gg = oracle.grad_grid(g.with_values(dens, g.sh), [cam], dict(step=0.25), rgb_t, depth_t)
    assert np.all(gg.grad_density == 0) and np.all(gg.grad_sh == 0)
    assert gg.loss > 0


# ---------------------------------------------------- pose Jacobian, Eq. 12-16
def pose_setup():
    g, cam, rgb_t, depth_t = fd_setup(seed=9, alloc_frac=0.9)
    opts = dict(step=0.25, bg=(0.1, 0.2, 0.3), lambda_d=0.7)
    return g, cam, rgb_t, depth_t, opts


def test_pose_jacobian_matches_frozen_sample_differences():
    g, cam, rgb_t, depth_t, opts = pose_setup()
    pj = oracle.pose_jacobian(g, [cam], opts, rgb_t, depth_t)
    eps = 1e-6
    fd = np.zeros_like(pj.J)
    for j in range(6):
        xi = np.zeros(6)
        xi[j] = eps
        fp = oracle.render_frozen(g, [cam], opts, xi)
        fm = oracle.render_frozen(g, [cam], opts, -xi)
        fd[:, :3, j] = (fp.rgb - fm.rgb) / (2 * eps)
        fd[:, 3, j] = (fp.depth - fm.depth) / (2 * eps)
    valid = np.isfinite(depth_t) & (depth_t > 0)
    fd[~valid] = 0
    scale = np.abs(pj.J).max()
    assert scale > 1e-3
    assert np.abs(fd - pj.J).max() <= 1e-5 * scale
    # frozen forward at xi = 0 is the forward itself
    f0 = oracle.render_frozen(g, [cam], opts, np.zeros(6))
    r0 = oracle.render(g, [cam], opts)
    np.testing.assert_array_equal(f0.rgb, r0.rgb)


def test_sh_basis_gradient_matches_differences():
    rng = np.random.default_rng(12)
    for _ in range(5):
        d = rng.standard_normal(3)
        G = oracle.sh_basis_grad(d)
        eps = 1e-6
        for a in range(3):
            e = np.zeros(3)
            e[a] = eps
            fd = (oracle.sh_basis(d + e) - oracle.sh_basis(d - e)) / (2 * eps)
            np.testing.assert_allclose(G[:, a], fd, atol=1e-9)


def test_pose_jacobian_view_direction_variant_matches_differences():
    """Variant (Sec. 5.3 omits it): the SH colour also turns with the ray
    direction. Its Jacobian matches differences of the frozen forward whose SH
    direction follows the pose, and differs from the paper's Jacobian only in
    the colour rows' rotation columns."""
    g, cam, rgb_t, depth_t, opts = pose_setup()
    ov = dict(opts, dir_term=True)
    pj = oracle.pose_jacobian(g, [cam], ov, rgb_t, depth_t)
    eps = 1e-6
    fd = np.zeros_like(pj.J)
    for j in range(6):
        xi = np.zeros(6)
        xi[j] = eps
        fp = oracle.render_frozen(g, [cam], ov, xi)
        fm = oracle.render_frozen(g, [cam], ov, -xi)
        fd[:, :3, j] = (fp.rgb - fm.rgb) / (2 * eps)
        fd[:, 3, j] = (fp.depth - fm.depth) / (2 * eps)
    valid = np.isfinite(depth_t) & (depth_t > 0)
    fd[~valid] = 0
    scale = np.abs(pj.J).max()
    assert np.abs(fd - pj.J).max() <= 1e-5 * scale
    base = oracle.pose_jacobian(g, [cam], opts, rgb_t, depth_t)
    diff = pj.J - base.J
    assert np.abs(diff[:, :3, 3:]).max() > 1e-3 * scale
    assert np.abs(diff[:, :3, :3]).max() <= 1e-12 * scale
    assert np.abs(diff[:, 3, :]).max() <= 1e-12 * scale


def test_pose_gradient_b_is_half_loss_gradient():
    """b = sum J^T W r, so d loss / d xi = 2 b (Eq. 4, 5, 11 chained with Eq. 12-14)."""
    g, cam, rgb_t, depth_t, opts = pose_setup()
    pj = oracle.pose_jacobian(g, [cam], opts, rgb_t, depth_t)
    eps = 1e-6
    grad = np.zeros(6)
    for j in range(6):
        xi = np.zeros(6)
        xi[j] = eps
        lp = brute_loss(cam, oracle.render_frozen(g, [cam], opts, xi), rgb_t, depth_t, 0.7)[0]
        lm = brute_loss(cam, oracle.render_frozen(g, [cam], opts, -xi), rgb_t, depth_t, 0.7)[0]
        grad[j] = (lp - lm) / (2 * eps)
    np.testing.assert_allclose(grad, 2 * pj.b, rtol=1e-6, atol=1e-9 * np.abs(pj.b).max())


def test_pose_hessian_is_curvature_at_zero_residual():
    """With targets rendered at the pose itself, r = 0 and the loss along a
    direction v is xi^T H xi to second order: (L(ev) + L(-ev)) / e^2 = 2 v^T H v."""
    g, cam, _, _, opts = pose_setup()
    opts = dict(opts, depth_is_z=False)
    r0 = oracle.render(g, [cam], opts)
    depth_t = r0.depth.copy()
    pj = oracle.pose_jacobian(g, [cam], opts, r0.rgb, depth_t)
    assert pj.loss == pytest.approx(0.0, abs=1e-28)
    np.testing.assert_allclose(pj.b, 0.0, atol=1e-15)
    rng = np.random.default_rng(4)
    for _ in range(4):
        v = rng.standard_normal(6)
        eps = 1e-4
        lp = brute_loss(cam, oracle.render_frozen(g, [cam], opts, eps * v), r0.rgb, depth_t,
                        0.7, depth_is_z=False)[0]
        lm = brute_loss(cam, oracle.render_frozen(g, [cam], opts, -eps * v), r0.rgb, depth_t,
                        0.7, depth_is_z=False)[0]
        assert (lp + lm) / eps ** 2 == pytest.approx(2 * v @ pj.H @ v, rel=2e-5)


# ------------------------------------------------------------ SE(3), GN step
def twist_matrix(xi):
    rho, phi = xi[:3], xi[3:]
    X = np.zeros((4, 4))
    X[:3, :3] = [[0, -phi[2], phi[1]], [phi[2], 0, -phi[0]], [-phi[1], phi[0], 0]]
    X[:3, 3] = rho
    return X


@pytest.mark.parametrize("scale", [0.0, 1e-9, 1e-7, 1e-3, 0.3, 2.5])
def test_se3_exp_matches_matrix_exponential(scale):
    rng = np.random.default_rng(int(scale * 1e9) % 1000)
    xi = np.concatenate([rng.standard_normal(3), scale * rng.standard_normal(3)])
    T = oracle.se3_exp(xi)
    ref = scipy.linalg.expm(twist_matrix(xi))[:3]
    np.testing.assert_allclose(T, ref, atol=1e-13)
    R = T[:, :3]
    np.testing.assert_allclose(R.T @ R, np.eye(3), atol=1e-13)
    assert np.linalg.det(R) == pytest.approx(1.0, abs=1e-13)


def test_pose_step_solves_and_composes_on_the_left():
    rng = np.random.default_rng(2)
    A = rng.standard_normal((10, 6))
    H = A.T @ A + 0.1 * np.eye(6)
    b = rng.standard_normal(6)
    T0 = scenes.look_at((1.0, 0.5, -2.0), (0, 0, 0))
    T1, xi, ok = oracle.pose_step(H, b, T0, damping=0.05)
    assert ok
    np.testing.assert_allclose(xi, -np.linalg.solve(H + 0.05 * np.eye(6), b), rtol=1e-12)
    T0h = np.vstack([T0, [0, 0, 0, 1]])
    np.testing.assert_allclose(T1, (scipy.linalg.expm(twist_matrix(xi)) @ T0h)[:3], atol=1e-12)
    T2, _, ok = oracle.pose_step(-np.eye(6), b, T0)
    assert not ok
    np.testing.assert_array_equal(T2, T0)


def test_gauss_newton_recovers_the_rendering_pose():
    """Targets rendered at T*; GN with the paper's Jacobian from a 3 cm / 2 deg
    perturbation converges back to T* (the 64^3 sphere scene)."""
    g, cam, _ = scenes.sphere_scene()
    opts = dict(step=0.5 * g.h[0], lambda_d=1.0, depth_is_z=False)
    ref = oracle.render(g, [cam], opts)
    T = scenes.perturb_pose(cam.T_wc, 0.03, 2.0, np.random.default_rng(5))
    err0 = np.abs(T - cam.T_wc).max()
    for _ in range(12):
        pj = oracle.pose_jacobian(g, [cam.with_pose(T)], opts, ref.rgb, ref.depth)
        T, xi, ok = oracle.pose_step(pj.H, pj.b, T)
        assert ok
    err = np.abs(T - cam.T_wc).max()
    assert err < 1e-3 * err0, (err0, err)
