"""Pins of the oracle's grid growth from observed depth (Sec. 6.1's dynamic
grid, read as: allocate every vertex within `band` grid units, per axis, of a
back-projected depth point; number new vertices in link order)."""
import numpy as np
import pytest

import oracle
from paper_2307_03404_b300 import scenes


def one_pixel_cam(o, R=np.eye(3)):
    T = np.zeros((3, 4))
    T[:, :3], T[:, 3] = R, o
    return scenes.Camera(10.0, 10.0, 0.5, 0.5, 1, 1, T)  # pixel centre on the axis


def test_single_point_by_hand():
    # camera at (2.5, 3.25, 0) looking along +z, z-depth 4: X = (2.5, 3.25, 4),
    # unit spacing; band 1 gives x in {2, 3}, y in {3, 4}, z in {3, 4, 5}
    links = -np.ones((8, 8, 8), np.int32)
    nl, k = oracle.grow((8, 8, 8), (0, 0, 0), (7, 7, 7), links, 0,
                        [one_pixel_cam((2.5, 3.25, 0.0))], np.array([4.0], np.float32), 1.0)
    assert k == 12
    got = {tuple(v) for v in np.argwhere(nl >= 0)}  # (z, y, x)
    want = {(z, y, x) for z in (3, 4, 5) for y in (3, 4) for x in (2, 3)}
    assert got == want
    # numbered 0..11 in link order (x fastest)
    flat = nl.reshape(-1)
    np.testing.assert_array_equal(flat[flat >= 0], np.arange(12))


def test_ray_distance_and_rotated_camera():
    # camera turned 90 degrees about y (its z axis along world +x); ray-distance
    # depth 3 from (1, 4, 4): X = (4, 4, 4) exactly on a vertex; band 0 allocates it alone
    Ry = np.array([[0.0, 0.0, 1.0], [0.0, 1.0, 0.0], [-1.0, 0.0, 0.0]])
    links = -np.ones((8, 8, 8), np.int32)
    nl, k = oracle.grow((8, 8, 8), (0, 0, 0), (7, 7, 7), links, 0,
                        [one_pixel_cam((1.0, 4.0, 4.0), Ry)], np.array([3.0], np.float32), 0.0,
                        depth_is_z=False)
    assert k == 1 and nl[4, 4, 4] == 0


def test_existing_vertices_keep_numbers_and_regrowth_is_idempotent():
    links = -np.ones((8, 8, 8), np.int32)
    links[4, 3, 2] = 0
    links[0, 0, 0] = 1
    cam = one_pixel_cam((2.5, 3.25, 0.0))
    d = np.array([4.0], np.float32)
    nl, k = oracle.grow((8, 8, 8), (0, 0, 0), (7, 7, 7), links, 2, [cam], d, 1.0)
    assert k == 11
    assert nl[4, 3, 2] == 0 and nl[0, 0, 0] == 1
    new = nl[(nl >= 2)]
    assert sorted(new.tolist()) == list(range(2, 13))
    nl2, k2 = oracle.grow((8, 8, 8), (0, 0, 0), (7, 7, 7), nl, 13, [cam], d, 1.0)
    assert k2 == 0
    np.testing.assert_array_equal(nl2, nl)


@pytest.mark.parametrize("bad", [0.0, -1.0, np.nan, np.inf])
def test_invalid_depth_adds_nothing(bad):
    links = -np.ones((6, 6, 6), np.int32)
    _, k = oracle.grow((6, 6, 6), (0, 0, 0), (5, 5, 5), links, 0,
                       [one_pixel_cam((2.0, 2.0, 0.0))], np.array([bad], np.float32), 2.0)
    assert k == 0


def test_point_outside_the_box_beyond_the_band_adds_nothing():
    links = -np.ones((6, 6, 6), np.int32)
    _, k = oracle.grow((6, 6, 6), (0, 0, 0), (5, 5, 5), links, 0,
                       [one_pixel_cam((2.0, 2.0, 0.0))], np.array([7.5], np.float32), 2.0)
    assert k == 0  # X at z = 7.5, box ends at 5: 2.5 > band
    _, k = oracle.grow((6, 6, 6), (0, 0, 0), (5, 5, 5), links, 0,
                       [one_pixel_cam((2.0, 2.0, 0.0))], np.array([6.5], np.float32), 2.0)
    assert k == 5 * 5  # X at z = 6.5: only the last layer z = 5, x, y in 0..4


def test_brute_force_distance_rule_on_a_frame():
    """Every allocated vertex lies within the band of some surface point and
    every vertex strictly inside the band of one is allocated; the points come
    from the oracle's own ray (unit direction times ray distance), a different
    route from the growth rule's."""
    rng = np.random.default_rng(3)
    R = 12
    lo, hi = np.array([-1.0, -1.0, -1.0]), np.array([1.0, 1.2, 0.9])
    cam = scenes.Camera(6.0, 5.0, 3.7, 2.2, 7, 5, scenes.look_at((0.2, 0.1, -2.5), (0, 0, 0)))
    z = rng.uniform(1.5, 3.2, 35).astype(np.float32)
    z[[3, 17]] = 0.0
    band = 1.3
    links = -np.ones((R, R, R), np.int32)
    nl, k = oracle.grow((R, R, R), lo, hi, links, 0, [cam], z, band)
    h = (hi - lo) / (R - 1)
    grid = scenes.Grid((R, R, R), lo, hi, links, np.zeros(0), np.zeros((0, 27)))
    pts = []
    for p in range(35):
        if z[p] <= 0:
            continue
        o, d, n, _, _ = oracle.pixel_ray(grid, cam, p)
        pts.append(o + d * (float(z[p]) * n))
    pts = (np.array(pts) - lo) / h                 # grid coordinates
    iz, iy, ix = np.meshgrid(np.arange(R), np.arange(R), np.arange(R), indexing="ij")
    V = np.stack([ix, iy, iz], -1).reshape(-1, 1, 3).astype(np.float64)
    cheb = np.abs(V - pts[None]).max(-1).min(-1).reshape(R, R, R)
    alloc = nl >= 0
    assert k == alloc.sum() > 0
    assert (cheb[alloc] <= band + 1e-9).all()
    assert alloc[cheb < band - 1e-9].all()
