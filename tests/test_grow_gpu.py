"""Grid growth from observed depth on the GPU against the oracle: the grown
link arrays are compared bit for bit (index work)."""
import numpy as np
import pytest
import torch

import oracle
from paper_2307_03404_b300 import plx, scenes

pytestmark = pytest.mark.gpu


def gpu_grow(res, lo, hi, links, n_alloc, cams, depth, band, depth_is_z=True):
    lk = torch.from_numpy(np.ascontiguousarray(links, np.int32)).cuda()
    n = plx.grid_grow(res, lo, hi, lk, n_alloc, plx.CameraSet(cams),
                      torch.from_numpy(np.ascontiguousarray(depth, np.float32)).cuda(), band,
                      depth_is_z=depth_is_z)
    return lk.cpu().numpy(), int(n.item())


def one_pixel_cam(o):
    T = np.zeros((3, 4))
    T[:, :3], T[:, 3] = np.eye(3), o
    return scenes.Camera(10.0, 10.0, 0.5, 0.5, 1, 1, T)


def test_single_point_and_overflow():
    links = -np.ones((8, 8, 8), np.int32)
    args = ((8, 8, 8), (0, 0, 0), (7, 7, 7))
    cam = [one_pixel_cam((2.5, 3.25, 0.0))]
    d = np.array([4.0], np.float32)
    got, k = gpu_grow(*args, links, 0, cam, d, 1.0)
    ref, kr = oracle.grow(*args, links, 0, cam, d, 1.0)
    assert k == kr == 12
    np.testing.assert_array_equal(got, ref)
    # numbers past INT32_MAX: nothing changes, the count reads -1
    got, k = gpu_grow(*args, links, 2 ** 31 - 5, cam, d, 1.0)
    assert k == -1
    np.testing.assert_array_equal(got, links)


@pytest.fixture(scope="module")
def room():
    R, occ, npr, seed = scenes.WORKLOADS["room256"]
    sc = scenes.room_scene(R, occ, npr, seed)
    cams = scenes.room_cameras(sc, 8, seed + 1)
    _, depth = scenes.sensor_frames(sc, cams, seed + 2)
    return sc.grid, cams, depth


@pytest.mark.parametrize("band", [0.0, 1.5, 2.0])
def test_room_frames_grow_bit_exact(room, band):
    g, cams, depth = room
    empty = -np.ones(g.links.shape, np.int32)
    got, k = gpu_grow(g.res, g.lo, g.hi, empty, 0, cams, depth, band)
    ref, kr = oracle.grow(g.res, g.lo, g.hi, empty, 0, cams, depth, band)
    assert k == kr
    assert k > 0 or band == 0.0  # band 0 needs a point exactly on a vertex
    np.testing.assert_array_equal(got, ref)


def test_incremental_growth_and_ray_distance(room):
    g, cams, depth = room
    n0 = 640 * 480 * 4
    empty = -np.ones(g.links.shape, np.int32)
    a_got, ka = gpu_grow(g.res, g.lo, g.hi, empty, 0, cams[:4], depth[:n0], 2.0)
    a_ref, _ = oracle.grow(g.res, g.lo, g.hi, empty, 0, cams[:4], depth[:n0], 2.0)
    np.testing.assert_array_equal(a_got, a_ref)
    b_got, kb = gpu_grow(g.res, g.lo, g.hi, a_got, ka, cams[4:], depth[n0:], 2.0)
    b_ref, kbr = oracle.grow(g.res, g.lo, g.hi, a_ref, ka, cams[4:], depth[n0:], 2.0)
    assert kb == kbr
    np.testing.assert_array_equal(b_got, b_ref)
    # the same depths read as ray distances
    c_got, kc = gpu_grow(g.res, g.lo, g.hi, empty, 0, cams[:2], depth[:640 * 480 * 2], 1.0,
                         depth_is_z=False)
    c_ref, kcr = oracle.grow(g.res, g.lo, g.hi, empty, 0, cams[:2], depth[:640 * 480 * 2], 1.0,
                             depth_is_z=False)
    assert kc == kcr
    np.testing.assert_array_equal(c_got, c_ref)


def test_mixed_sizes_grid_not_cubic():
    rng = np.random.default_rng(5)
    res, lo, hi = (37, 21, 30), (-1.0, -0.6, -0.9), (1.1, 0.7, 1.0)
    cams = [scenes.Camera(9.0, 8.0, 6.1, 3.3, 13, 7, scenes.look_at((0.3, 0.2, -2.2), (0, 0, 0))),
            scenes.Camera(4.0, 4.0, 2.5, 1.5, 5, 3, scenes.look_at((-2.0, 0.5, 0.4), (0, 0.1, 0)))]
    depth = rng.uniform(1.0, 3.0, 13 * 7 + 5 * 3).astype(np.float32)
    depth[rng.random(depth.shape) < 0.1] = 0.0
    depth[7] = np.nan
    links = -np.ones((30, 21, 37), np.int32)
    links[rng.random(links.shape) < 0.02] = 0
    n0 = int((links >= 0).sum())
    links[links >= 0] = rng.permutation(n0)
    got, k = gpu_grow(res, lo, hi, links, n0, cams, depth, 2.5)
    ref, kr = oracle.grow(res, lo, hi, links, n0, cams, depth, 2.5)
    assert k == kr > 0
    np.testing.assert_array_equal(got, ref)
