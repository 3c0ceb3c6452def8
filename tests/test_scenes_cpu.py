"""The synthetic workload generators (host side): the allocated fraction, the
unallocated border, cameras in free space, and the torch sensor model against
the numpy one."""
import numpy as np
import pytest
import torch

from paper_2307_03404_b300 import scenes


@pytest.fixture(scope="module")
def small_house():
    return scenes.house_scene(R=96, occupancy=0.02, n_prims=20, seed=11, device="cpu")


def test_house_scene_fraction_and_border(small_house):
    g = small_house.grid
    R = g.res[0]
    assert abs(g.n_alloc / R ** 3 - 0.02) <= 0.002
    for a in range(3):
        sl = [slice(None)] * 3
        for b in (slice(0, 2), slice(R - 2, R)):
            sl[a] = b
            assert (g.links[tuple(sl)] < 0).all()
    # links number the allocated vertices 0..n-1 in raster order
    lk = g.links.reshape(-1)
    np.testing.assert_array_equal(lk[lk >= 0], np.arange(g.n_alloc))
    assert g.density.shape == (g.n_alloc,) and g.sh.shape == (g.n_alloc, 27)


def test_house_cameras_in_free_space(small_house):
    cams = scenes.house_cameras(small_house, 5, 12, 40, 30, 20.0)
    for c in cams:
        o = np.asarray(c.T_wc).reshape(3, 4)[:, 3]
        assert scenes._free_space(small_house, o)[0] > 0.5
        R_ = np.asarray(c.T_wc).reshape(3, 4)[:, :3]
        np.testing.assert_allclose(R_.T @ R_, np.eye(3), atol=1e-12)


def test_torch_sensor_model_matches_numpy(small_house):
    cams = scenes.house_cameras(small_house, 3, 13, 40, 30, 20.0)
    _, dz_np = scenes.sensor_frames(small_house, cams, 1, depth_noise=0.0, missing=0.0)
    rgb_t, dz_t = scenes.sensor_frames_torch(small_house, cams, 1, device="cpu",
                                             depth_noise=0.0, missing=0.0)
    np.testing.assert_allclose(dz_t.numpy(), dz_np, rtol=1e-6)
    assert rgb_t.shape == (dz_np.shape[0], 3)
    assert float(rgb_t.min()) >= 0.0 and float(rgb_t.max()) <= 1.0
    _, dz_m = scenes.sensor_frames_torch(small_house, cams, 1, device="cpu")
    assert 0.005 <= float((dz_m == 0).float().mean()) <= 0.04


def test_room_variants_scale_density_and_add_a_smooth_texture():
    """The tracking room's variant: the same links, densities scaled, and a
    texture interpolated from a 10 cm lattice: strongly correlated between
    neighbouring vertices (h = 6.7 cm here), unlike per-vertex noise."""
    kw = dict(R=96, occupancy=0.1, n_prims=4, seed=21)
    base = scenes.room_scene(**kw)
    flat = scenes.room_scene(**kw, vertex_noise=0.0)
    var = scenes.room_scene(**kw, density_scale=8.0, vertex_noise=0.0, smooth_texture=0.2,
                            texture_cell=0.1)
    np.testing.assert_array_equal(base.grid.links, var.grid.links)
    np.testing.assert_allclose(var.grid.density, 8.0 * base.grid.density, rtol=1e-6)
    tex = var.grid.sh - flat.grid.sh          # the smooth field alone
    noise = base.grid.sh - flat.grid.sh       # the default per-vertex noise alone
    lk = var.grid.links
    a, b = lk[:, :, :-1].reshape(-1), lk[:, :, 1:].reshape(-1)
    both = (a >= 0) & (b >= 0)

    def corr(f):
        x, y = f[a[both]].reshape(-1), f[b[both]].reshape(-1)
        return float(np.corrcoef(x, y)[0, 1])

    assert corr(tex) > 0.5 and abs(corr(noise)) < 0.05
    assert 0.05 < float(tex.std()) < 0.2 and abs(float(noise.std()) - 0.1) < 0.005
