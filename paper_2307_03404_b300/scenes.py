"""Seeded synthetic inputs: sparse voxel grids, cameras and RGB-D sensor frames.

This module is shared by the CUDA path's tests and benchmark and by the CPU
oracle's tests. It holds none of the rendering method's arithmetic (no
compositing, no SH, no interpolation, no pose algebra beyond building camera
frames): it only builds the grid arrays of an analytic scene, places cameras,
and simulates an RGB-D sensor by intersecting pixel rays with the analytic
primitives. The paper measures on Replica and ScanNet, which are not
available; these scenes stand in for them at the paper's camera model
(640x480, f = 525) and its grid form (28 values per allocated vertex, a dense
int32 link array, Sec. 5.2, Sec. 6.1).

Everything is drawn from ``numpy.random.default_rng(seed)``.
"""
from __future__ import annotations

import dataclasses
from typing import List, Sequence

import numpy as np

N_VALUES = 28          # 1 density + 3 x 9 SH coefficients per vertex (Sec. 5.2)
N_SH = 27


@dataclasses.dataclass
class Grid:
    """Sparse voxel grid in the canonical caller layout.

    ``links[z, y, x]`` is the row of vertex (x, y, z) in ``density`` / ``sh``,
    or -1 where the vertex is not allocated. ``sh[i]`` is channel-major
    (R0..R8, G0..G8, B0..B8). Vertex (x, y, z) sits at lo + (x, y, z) * h with
    h = (hi - lo) / (res - 1).
    """

    res: tuple
    lo: np.ndarray
    hi: np.ndarray
    links: np.ndarray      # int32 [Rz, Ry, Rx]
    density: np.ndarray    # float32 [n]
    sh: np.ndarray         # float32 [n, 27]

    @property
    def n_alloc(self) -> int:
        return int(self.density.shape[0])

    @property
    def h(self) -> np.ndarray:
        return (np.asarray(self.hi, np.float64) - np.asarray(self.lo, np.float64)) / (
            np.asarray(self.res, np.float64) - 1.0)

    def with_values(self, density, sh) -> "Grid":
        return Grid(self.res, self.lo, self.hi, self.links, density, sh)


@dataclasses.dataclass
class Camera:
    """Pinhole camera: intrinsics in pixels, camera-to-world pose [R | o]
    (x right, y down, z forward in the camera frame)."""

    fx: float
    fy: float
    cx: float
    cy: float
    width: int
    height: int
    T_wc: np.ndarray       # float64 [3, 4]

    def with_pose(self, T_wc) -> "Camera":
        return Camera(self.fx, self.fy, self.cx, self.cy, self.width, self.height,
                      np.asarray(T_wc, np.float64).reshape(3, 4).copy())


@dataclasses.dataclass
class Scene:
    """A grid with the analytic primitives it was built from."""

    grid: Grid
    prims: list
    room_lo: np.ndarray | None = None
    room_hi: np.ndarray | None = None


# ------------------------------------------------------------------ cameras
def look_at(eye, target, up=(0.0, 1.0, 0.0)) -> np.ndarray:
    """Camera-to-world [R | eye] for a camera at ``eye`` looking at ``target``."""
    eye = np.asarray(eye, np.float64)
    z = np.asarray(target, np.float64) - eye
    z /= np.linalg.norm(z)
    x = np.cross(z, np.asarray(up, np.float64))
    x /= np.linalg.norm(x)
    y = np.cross(z, x)
    T = np.zeros((3, 4))
    T[:, 0], T[:, 1], T[:, 2], T[:, 3] = x, y, z, eye
    return T


def perturb_pose(T_wc, trans_m: float, rot_deg: float, rng) -> np.ndarray:
    """Move a camera by ``trans_m`` along a random unit axis and turn it by
    ``rot_deg`` about a random axis through its own centre."""
    from scipy.spatial.transform import Rotation

    T = np.asarray(T_wc, np.float64).reshape(3, 4)
    u = rng.standard_normal(3)
    u /= np.linalg.norm(u)
    a = rng.standard_normal(3)
    a /= np.linalg.norm(a)
    Rp = Rotation.from_rotvec(np.deg2rad(rot_deg) * a).as_matrix()
    out = np.zeros((3, 4))
    out[:, :3] = Rp @ T[:, :3]
    out[:, 3] = T[:, 3] + trans_m * u
    return out


def dense_rays(cams: Sequence[Camera]):
    """(cam_id, pixel) of every pixel of every camera, camera by camera."""
    cid, pix = [], []
    for i, c in enumerate(cams):
        n = int(c.width) * int(c.height)
        cid.append(np.full(n, i, np.int32))
        pix.append(np.arange(n, dtype=np.int32))
    return np.concatenate(cid), np.concatenate(pix)


def random_rays(cams: Sequence[Camera], n: int, seed: int):
    """``n`` distinct rays drawn uniformly from all pixels of all cameras."""
    cid, pix = dense_rays(cams)
    rng = np.random.default_rng(seed)
    sel = np.sort(rng.choice(cid.shape[0], size=min(n, cid.shape[0]), replace=False))
    return cid[sel], pix[sel]


# ------------------------------------------------------------ tiny grids
def tiny_grid(R: int = 6, seed: int = 0, alloc_frac: float = 1.0, half: float = 1.0,
              sigma_mean: float = 3.0, sigma_std: float = 1.0, sh_std: float = 0.3,
              border: int = 0) -> Grid:
    """Small random grid for finite differences and closed forms.

    ``alloc_frac`` < 1 leaves a random subset of vertices unallocated;
    ``border`` layers of vertices at the box faces are left unallocated.
    """
    rng = np.random.default_rng(seed)
    alloc = rng.random((R, R, R)) < alloc_frac
    if border > 0:
        b = border
        inner = np.zeros((R, R, R), bool)
        inner[b:R - b, b:R - b, b:R - b] = True
        alloc &= inner
    links = np.full((R, R, R), -1, np.int32)
    n = int(alloc.sum())
    order = rng.permutation(n).astype(np.int32)
    links[alloc] = order
    density = (sigma_mean + sigma_std * rng.standard_normal(n)).astype(np.float32)
    sh = (sh_std * rng.standard_normal((n, N_SH))).astype(np.float32)
    lo = np.full(3, -half)
    hi = np.full(3, half)
    return Grid((R, R, R), lo, hi, links, density, sh)


def constant_grid(R: int, sigma: float, sh_dc: Sequence[float], half: float = 1.0) -> Grid:
    """Every vertex allocated with the same density and only the degree-0 SH
    coefficient set (``sh_dc`` per channel)."""
    n = R ** 3
    links = np.arange(n, dtype=np.int32).reshape(R, R, R)
    density = np.full(n, sigma, np.float32)
    sh = np.zeros((n, N_SH), np.float32)
    for ch in range(3):
        sh[:, 9 * ch] = sh_dc[ch]
    return Grid((R, R, R), np.full(3, -half), np.full(3, half), links, density, sh)


# ------------------------------------------------- dense 64^3 sphere scene
def sphere_scene(R: int = 64, seed: int = 1001, width: int = 64, height: int = 48,
                 f: float = 60.0):
    """Dense R^3 grid over [-1,1]^3: density 40 inside three random spheres
    (centres in [-0.5,0.5]^3, radius 0.15-0.35) and in the floor slab
    y <= -0.8, 0 elsewhere; the two outermost vertex layers are 0; SH ~ N(0,0.3).
    One camera on the radius-2.5 sphere (elevation 10-60 deg) looking at the
    origin. Also returns a perturbed copy of the grid (density * (1 + 0.1 N),
    SH + N(0, 0.05)) from which targets are rendered.
    """
    rng = np.random.default_rng(seed)
    xs = np.linspace(-1.0, 1.0, R)
    Z, Y, X = np.meshgrid(xs, xs, xs, indexing="ij")
    occ = Y <= -0.8
    for _ in range(3):
        c = rng.uniform(-0.5, 0.5, 3)
        r = rng.uniform(0.15, 0.35)
        occ |= (X - c[0]) ** 2 + (Y - c[1]) ** 2 + (Z - c[2]) ** 2 <= r * r
    dens = np.where(occ, 40.0, 0.0)
    dens[:2], dens[-2:] = 0.0, 0.0
    dens[:, :2], dens[:, -2:] = 0.0, 0.0
    dens[:, :, :2], dens[:, :, -2:] = 0.0, 0.0
    n = R ** 3
    links = np.arange(n, dtype=np.int32).reshape(R, R, R)
    density = dens.reshape(-1).astype(np.float32)
    sh = (0.3 * rng.standard_normal((n, N_SH))).astype(np.float32)
    grid = Grid((R, R, R), np.full(3, -1.0), np.full(3, 1.0), links, density, sh)
    az = rng.uniform(0, 2 * np.pi)
    el = np.deg2rad(rng.uniform(10, 60))
    eye = 2.5 * np.array([np.cos(el) * np.cos(az), np.sin(el), np.cos(el) * np.sin(az)])
    cam = Camera(f, f, width / 2.0, height / 2.0, width, height, look_at(eye, (0, 0, 0)))
    pd = (density * (1.0 + 0.1 * rng.standard_normal(n))).astype(np.float32)
    ps = (sh + 0.05 * rng.standard_normal((n, N_SH))).astype(np.float32)
    return grid, cam, grid.with_values(pd, ps)


# ------------------------------------------------------------- room scenes
def _box_sdf(P, c, half):
    q = np.abs(P - c) - half
    outside = np.linalg.norm(np.maximum(q, 0.0), axis=-1)
    inside = np.minimum(q.max(axis=-1), 0.0)
    return outside + inside


def _prim_sdf(P, prim):
    if prim["kind"] == "sphere":
        return np.linalg.norm(P - prim["c"], axis=-1) - prim["r"]
    return _box_sdf(P, prim["c"], prim["half"])


def _prim_sdf_sep(xs, ys, zs, prim):
    """Same distance as _prim_sdf on the grid zs x ys x xs, from 1-D axes."""
    c = prim["c"].astype(np.float32)
    if prim["kind"] == "sphere":
        d2 = ((zs - c[2]) ** 2)[:, None, None] + ((ys - c[1]) ** 2)[None, :, None] \
            + ((xs - c[0]) ** 2)[None, None, :]
        return np.sqrt(d2) - np.float32(prim["r"])
    hf = prim["half"].astype(np.float32)
    qx, qy, qz = np.abs(xs - c[0]) - hf[0], np.abs(ys - c[1]) - hf[1], np.abs(zs - c[2]) - hf[2]
    out2 = (np.maximum(qz, 0) ** 2)[:, None, None] + (np.maximum(qy, 0) ** 2)[None, :, None] \
        + (np.maximum(qx, 0) ** 2)[None, None, :]
    inside = np.minimum(np.maximum(np.maximum(qz[:, None, None], qy[None, :, None]),
                                   qx[None, None, :]), 0)
    return np.sqrt(out2) + inside


def _prim_extent(prim):
    return np.full(3, prim["r"]) if prim["kind"] == "sphere" else prim["half"]


def _random_prims(rng, room_lo, room_hi, n):
    prims = []
    span = room_hi - room_lo
    for i in range(n):
        rgb = rng.uniform(0.1, 0.9, 3)
        if i % 2 == 0:
            r = rng.uniform(0.04, 0.12) * span.min()
            c = rng.uniform(room_lo + r, room_hi - r)
            prims.append({"kind": "sphere", "c": c, "r": r, "rgb": rgb})
        else:
            half = rng.uniform(0.03, 0.12, 3) * span.min()
            c = rng.uniform(room_lo + half, room_hi - half)
            c[1] = room_lo[1] + half[1] if rng.random() < 0.5 else c[1]  # some on the floor
            prims.append({"kind": "box", "c": c, "half": half, "rgb": rgb})
    return prims


def _scene_sdf_grid(R, lo, hi, room_lo, room_hi, prims, margin_vox=12):
    """Signed distance (positive in free space) at every vertex, and the id of
    the nearest surface (0..5 the walls -x, +x, -y, +y, -z, +z; 6 + i primitive
    i). Walls are the faces of the room box (solid outside it). Each primitive
    is evaluated only within ``margin_vox`` voxels of its extent; farther away
    its distance exceeds any band width used here, so the band is unchanged."""
    xs = np.linspace(lo[0], hi[0], R).astype(np.float32)
    ys = np.linspace(lo[1], hi[1], R).astype(np.float32)
    zs = np.linspace(lo[2], hi[2], R).astype(np.float32)

    def wall(v, a):
        lo_d, hi_d = v - room_lo[a], room_hi[a] - v
        return np.minimum(lo_d, hi_d).astype(np.float32), (hi_d < lo_d).astype(np.uint8)

    (wx, sx), (wy, sy), (wz, sz) = wall(xs, 0), wall(ys, 1), wall(zs, 2)
    s = np.empty((R, R, R), np.float32)
    ids = np.empty((R, R, R), np.uint8)
    for k in range(R):          # slab by slab keeps the temporaries small
        sl = np.minimum(wy[:, None], wx[None, :])
        idl = np.where(wy[:, None] <= wx[None, :], 2 + sy[:, None], 0 + sx[None, :])
        zsel = wz[k] <= sl
        s[k] = np.where(zsel, wz[k], sl)
        ids[k] = np.where(zsel, 4 + sz[k], idl)
    h = (hi - lo) / (R - 1)
    for i, p in enumerate(prims):
        ext = _prim_extent(p) + margin_vox * h
        i0 = np.clip(np.floor((p["c"] - ext - lo) / h).astype(int), 0, R - 1)
        i1 = np.clip(np.ceil((p["c"] + ext - lo) / h).astype(int) + 1, 0, R)
        sub = s[i0[2]:i1[2], i0[1]:i1[1], i0[0]:i1[0]]
        isub = ids[i0[2]:i1[2], i0[1]:i1[1], i0[0]:i1[0]]
        d = _prim_sdf_sep(xs[i0[0]:i1[0]], ys[i0[1]:i1[1]], zs[i0[2]:i1[2]], p)
        closer = d < sub
        sub[closer] = d[closer]
        isub[closer] = 6 + i
    return s, ids


def _add_smooth_texture(sh, sel, R, h, amp, cell, rng, chunk=1 << 20):
    """Adds to ``sh`` [n, 27] a smooth random field: N(0, amp) values on a
    lattice of spacing ``cell`` covering the grid box, interpolated
    trilinearly at the positions of the allocated vertices ``sel`` (flat
    indices into the R^3 vertex lattice)."""
    span = (R - 1) * h
    m = np.ceil(span / cell).astype(int) + 2
    lat = (amp * rng.standard_normal((m[2], m[1], m[0], sh.shape[1]))).astype(np.float32)
    for a in range(0, sel.shape[0], chunk):
        idx = sel[a:a + chunk]
        iz, rem = np.divmod(idx, R * R)
        iy, ix = np.divmod(rem, R)
        q = [(ix * h[0]) / cell, (iy * h[1]) / cell, (iz * h[2]) / cell]
        i0 = [np.minimum(np.floor(v).astype(np.int64), m[k] - 2) for k, v in enumerate(q)]
        f = [(v - i0[k]).astype(np.float32)[:, None] for k, v in enumerate(q)]
        acc = np.zeros((idx.shape[0], sh.shape[1]), np.float32)
        for dz in (0, 1):
            wz = f[2] if dz else 1 - f[2]
            for dy in (0, 1):
                wy = f[1] if dy else 1 - f[1]
                for dx in (0, 1):
                    wx = f[0] if dx else 1 - f[0]
                    acc += (wx * wy * wz) * lat[i0[2] + dz, i0[1] + dy, i0[0] + dx]
        sh[a:a + chunk] += acc


def room_scene(R: int, occupancy: float, n_prims: int, seed: int, half: float = 3.2,
               wall_inset_vox: float = 4.0, border: int = 2, density_scale: float = 1.0,
               vertex_noise: float = 0.1, smooth_texture: float = 0.0,
               texture_cell: float = 0.1) -> Scene:
    """Analytic room: the six faces of a box inset by ``wall_inset_vox`` voxels
    from the grid box, plus ``n_prims`` random spheres and boxes. The vertices
    closest to the surfaces are allocated, as many as the fraction
    ``occupancy`` of all vertices (distance ties broken by a seeded jitter of
    +-0.05 voxel); the ``border`` outermost vertex layers are never allocated.
    Allocated density rises across the band into the solid, about 0.6 / h at
    the inner band edge and slightly negative at the outer one. SH: each
    surface (wall or primitive) has its own N(0, 0.28) coefficients, and each
    vertex adds N(0, 0.1) to those of its nearest surface (about N(0, 0.3)
    overall): surfaces carry a colour with texture, as scanned rooms do.

    Variants (defaults give the scene above): ``density_scale`` multiplies
    every density (8 makes the surfaces opaque: a ray keeps about 1e-4 of its
    transmittance after the room); ``vertex_noise`` is the per-vertex SH noise;
    ``smooth_texture`` > 0 adds a spatially smooth texture of that standard
    deviation: N(0, 1) values on a lattice of ``texture_cell`` metres, drawn
    after everything else, interpolated trilinearly at each vertex.
    """
    rng = np.random.default_rng(seed)
    lo = np.full(3, -half)
    hi = np.full(3, half)
    h = (hi - lo) / (R - 1)
    hm = float(h.min())
    room_lo = lo + wall_inset_vox * h
    room_hi = hi - wall_inset_vox * h
    prims = _random_prims(rng, room_lo, room_hi, n_prims)
    s, ids = _scene_sdf_grid(R, lo, hi, room_lo, room_hi, prims)
    b = border
    key = np.abs(s)
    key += (rng.random(key.shape, dtype=np.float32) - np.float32(0.5)) * np.float32(0.1 * hm)
    key[:b], key[R - b:] = np.inf, np.inf
    key[:, :b], key[:, R - b:] = np.inf, np.inf
    key[:, :, :b], key[:, :, R - b:] = np.inf, np.inf
    n = int(round(occupancy * R ** 3))
    flat = key.reshape(-1)
    sel = np.argpartition(flat, n - 1)[:n] if n > 0 else np.zeros(0, np.int64)
    sel.sort()
    del key, flat
    links = np.full(R ** 3, -1, np.int32)
    links[sel] = np.arange(n, dtype=np.int32)
    links = links.reshape(R, R, R)
    sv = s.reshape(-1)[sel].astype(np.float64)
    surf = ids.reshape(-1)[sel]
    del s, ids
    w = max(float(np.abs(sv).max()), hm)
    density = ((0.6 / hm) * (0.5 - 0.6 * sv / w)
               + (0.05 / hm) * rng.standard_normal(n)).astype(np.float32)
    if density_scale != 1.0:
        density *= np.float32(density_scale)
    base = (0.28 * rng.standard_normal((6 + len(prims), N_SH))).astype(np.float32)
    sh = rng.standard_normal((n, N_SH), dtype=np.float32)
    sh *= np.float32(vertex_noise)
    sh += base[surf]
    if smooth_texture > 0.0:
        _add_smooth_texture(sh, sel, R, h, smooth_texture, texture_cell, rng)
    grid = Grid((R, R, R), lo, hi, links, density, sh)
    return Scene(grid, prims, room_lo, room_hi)


def _house_prims(rng, room_lo, room_hi, n):
    """Two partition walls (x = 0 and z = 0, 0.12 m thick) with a door each,
    as boxes, then ``n`` random spheres and boxes of 0.1-0.4 m half-size."""
    prims = []
    floor, ceil = room_lo[1], room_hi[1]
    door_h, door_w, t = 2.1, 1.0, 0.06
    grey = np.array([0.7, 0.7, 0.68])
    for axis in (0, 2):  # wall normal along x, then along z
        other = 2 - axis
        lo_o, hi_o = room_lo[other], room_hi[other]
        d = rng.uniform(lo_o + 1.5, hi_o - 1.5)  # door centre along the wall
        pieces = [(lo_o, d - door_w / 2, floor, ceil), (d + door_w / 2, hi_o, floor, ceil),
                  (d - door_w / 2, d + door_w / 2, floor + door_h, ceil)]
        for a0, a1, y0, y1 in pieces:
            c = np.zeros(3)
            half = np.zeros(3)
            c[axis], half[axis] = 0.0, t
            c[other], half[other] = 0.5 * (a0 + a1), 0.5 * (a1 - a0)
            c[1], half[1] = 0.5 * (y0 + y1), 0.5 * (y1 - y0)
            prims.append({"kind": "box", "c": c, "half": half, "rgb": grey})
    for i in range(n):
        rgb = rng.uniform(0.1, 0.9, 3)
        if i % 2 == 0:
            r = rng.uniform(0.1, 0.4)
            c = rng.uniform(room_lo + r, room_hi - r)
            prims.append({"kind": "sphere", "c": c, "r": r, "rgb": rgb})
        else:
            half = rng.uniform(0.1, 0.4, 3)
            c = rng.uniform(room_lo + half, room_hi - half)
            c[1] = room_lo[1] + half[1] if rng.random() < 0.5 else c[1]
            prims.append({"kind": "box", "c": c, "half": half, "rgb": rgb})
    return prims


def house_scene(R: int = 1024, occupancy: float = 0.02, n_prims: int = 200, seed: int = 1005,
                half: float = 6.4, wall_inset_vox: float = 4.0, border: int = 2,
                device: str = "cuda") -> Scene:
    """Multi-room house for large grids, built with torch on ``device`` (a
    1024^3 grid has 1.07 G vertices): the room box split into four rooms by two
    partition walls with doors, plus ``n_prims`` random primitives. The same
    recipe as ``room_scene`` otherwise: the vertices nearest to the surfaces
    are allocated (threshold = the ``occupancy`` quantile of |sdf| + a seeded
    +-0.05-voxel jitter, estimated on 16 M random vertices, so the fraction is
    approximate), two border layers never allocated, density rising into the
    solid, per-surface SH plus per-vertex noise.
    """
    import torch

    rng = np.random.default_rng(seed)
    gen = torch.Generator(device=device)
    gen.manual_seed(seed)
    lo = np.full(3, -half)
    hi = np.full(3, half)
    h = (hi - lo) / (R - 1)
    hm = float(h.min())
    room_lo = lo + wall_inset_vox * h
    room_hi = hi - wall_inset_vox * h
    prims = _house_prims(rng, room_lo, room_hi, n_prims)
    f32 = torch.float32
    ax = [torch.linspace(lo[a], hi[a], R, device=device, dtype=torch.float64).to(f32)
          for a in range(3)]
    walls = []
    for a in range(3):
        lo_d, hi_d = ax[a] - float(room_lo[a]), float(room_hi[a]) - ax[a]
        walls.append((torch.minimum(lo_d, hi_d), (hi_d < lo_d).to(torch.uint8)))
    (wx, sx), (wy, sy), (wz, sz) = walls
    s = torch.empty((R, R, R), dtype=f32, device=device)
    ids = torch.empty((R, R, R), dtype=torch.uint8, device=device)
    for z0 in range(0, R, 64):
        z1 = min(R, z0 + 64)
        sl = torch.minimum(wy[:, None], wx[None, :])
        idl = torch.where(wy[:, None] <= wx[None, :], 2 + sy[:, None], 0 + sx[None, :])
        zs = wz[z0:z1, None, None]
        zsel = zs <= sl[None]
        s[z0:z1] = torch.where(zsel, zs, sl[None])
        ids[z0:z1] = torch.where(zsel, (4 + sz[z0:z1])[:, None, None], idl[None])
    for i, p in enumerate(prims):
        ext = _prim_extent(p) + 12 * h
        i0 = np.clip(np.floor((p["c"] - ext - lo) / h).astype(int), 0, R - 1)
        i1 = np.clip(np.ceil((p["c"] + ext - lo) / h).astype(int) + 1, 0, R)
        X, Yv, Z = ax[0][i0[0]:i1[0]], ax[1][i0[1]:i1[1]], ax[2][i0[2]:i1[2]]
        c = [float(v) for v in p["c"]]
        if p["kind"] == "sphere":
            d = torch.sqrt((Z - c[2])[:, None, None] ** 2 + (Yv - c[1])[None, :, None] ** 2
                           + (X - c[0])[None, None, :] ** 2) - float(p["r"])
        else:
            hf = [float(v) for v in p["half"]]
            qx, qy, qz = (X - c[0]).abs() - hf[0], (Yv - c[1]).abs() - hf[1], (Z - c[2]).abs() - hf[2]
            out = torch.sqrt(qz.clamp(min=0)[:, None, None] ** 2 + qy.clamp(min=0)[None, :, None] ** 2
                             + qx.clamp(min=0)[None, None, :] ** 2)
            inside = torch.maximum(torch.maximum(qz[:, None, None], qy[None, :, None]),
                                   qx[None, None, :]).clamp(max=0)
            d = out + inside
        sub = s[i0[2]:i1[2], i0[1]:i1[1], i0[0]:i1[0]]
        isub = ids[i0[2]:i1[2], i0[1]:i1[1], i0[0]:i1[0]]
        closer = d < sub
        sub[closer] = d[closer]
        isub[closer] = 6 + i
    key = s.abs()
    key += (torch.rand((R, R, R), generator=gen, device=device, dtype=f32) - 0.5) * (0.1 * hm)
    b = border
    for sl_ in (np.s_[:b], np.s_[R - b:]):
        key[sl_] = float("inf")
        key[:, sl_] = float("inf")
        key[:, :, sl_] = float("inf")
    pick = torch.randint(0, R ** 3, (min(R ** 3, 1 << 24),), generator=gen, device=device)
    sample = key.reshape(-1)[pick]
    k = max(1, int(round(occupancy * sample.numel())))
    w = float(torch.kthvalue(sample, k).values)
    mask = (key <= w).reshape(-1)
    del key
    n = int(mask.sum())
    links = torch.full((R ** 3,), -1, dtype=torch.int32, device=device)
    links[mask] = torch.arange(n, dtype=torch.int32, device=device)
    sv = s.reshape(-1)[mask].double()
    surf = ids.reshape(-1)[mask].long()
    del s, ids
    wmax = max(float(sv.abs().max()), hm)
    density = ((0.6 / hm) * (0.5 - 0.6 * sv / wmax)
               + (0.05 / hm) * torch.randn(n, generator=gen, device=device, dtype=torch.float64))
    base = torch.from_numpy((0.28 * rng.standard_normal((6 + len(prims), N_SH))).astype(np.float32))
    sh = torch.randn((n, N_SH), generator=gen, device=device, dtype=f32) * 0.1 + base.to(device)[surf]
    grid = Grid((R, R, R), lo, hi, links.reshape(R, R, R).cpu().numpy(),
                density.float().cpu().numpy(), sh.cpu().numpy())
    return Scene(grid, prims, room_lo, room_hi)


def _free_space(scene: Scene, P):
    P = np.atleast_2d(P)
    d = np.minimum((P - scene.room_lo).min(axis=-1), (scene.room_hi - P).min(axis=-1))
    for p in scene.prims:
        d = np.minimum(d, _prim_sdf(P, p))
    return d


def house_cameras(scene: Scene, n: int, seed: int, width: int = 1200, height: int = 680,
                  f: float = 600.0, clearance: float = 0.5) -> List[Camera]:
    """``n`` keyframes spread over the rooms of a house: each at a random
    free-space point of the lower half, looking horizontally in a random
    direction with a slight downward pitch."""
    rng = np.random.default_rng(seed)
    span = scene.room_hi - scene.room_lo
    cams = []
    while len(cams) < n:
        p = rng.uniform(scene.room_lo + 0.1 * span, scene.room_hi - 0.1 * span)
        p[1] = rng.uniform(scene.room_lo[1] + 0.1 * span[1], scene.room_lo[1] + 0.5 * span[1])
        if _free_space(scene, p)[0] <= clearance:
            continue
        yaw = rng.uniform(0.0, 2.0 * np.pi)
        pitch = np.deg2rad(rng.uniform(-20, 0))
        look = np.array([np.cos(pitch) * np.cos(yaw), np.sin(pitch), np.cos(pitch) * np.sin(yaw)])
        cams.append(Camera(f, f, width / 2.0 - 0.5, height / 2.0 - 0.5, width, height,
                           look_at(p, p + look)))
    return cams


def _spline_path(scene: Scene, rng, clearance: float):
    """Catmull-Rom spline through six random free-space points of the room
    (drawn from ``rng``): returns (spline(u) -> (position, tangent), segments)."""
    span = scene.room_hi - scene.room_lo
    pts = []
    while len(pts) < 6:
        p = rng.uniform(scene.room_lo + 0.2 * span, scene.room_hi - 0.2 * span)
        if _free_space(scene, p)[0] > clearance:
            pts.append(p)
    pts = np.array(pts)
    ctrl = np.vstack([pts[:1], pts, pts[-1:]])

    def spline(u):
        seg = min(int(u), len(pts) - 2)
        t = u - seg
        p0, p1, p2, p3 = ctrl[seg], ctrl[seg + 1], ctrl[seg + 2], ctrl[seg + 3]
        pos = 0.5 * ((2 * p1) + (-p0 + p2) * t + (2 * p0 - 5 * p1 + 4 * p2 - p3) * t * t
                     + (-p0 + 3 * p1 - 3 * p2 + p3) * t ** 3)
        tan = 0.5 * ((-p0 + p2) + 2 * (2 * p0 - 5 * p1 + 4 * p2 - p3) * t
                     + 3 * (-p0 + 3 * p1 - 3 * p2 + p3) * t * t)
        return pos, tan

    return spline, len(pts) - 1


def _heading(tan, yaw, pitch):
    fwd = np.array([tan[0], 0.0, tan[2]])
    if np.linalg.norm(fwd) < 1e-6:
        fwd = np.array([1.0, 0.0, 0.0])
    fwd /= np.linalg.norm(fwd)
    cy_, sy_ = np.cos(yaw), np.sin(yaw)
    fwd = np.array([cy_ * fwd[0] - sy_ * fwd[2], 0.0, sy_ * fwd[0] + cy_ * fwd[2]])
    return np.cos(pitch) * fwd + np.array([0.0, np.sin(pitch), 0.0])


def room_cameras(scene: Scene, n: int, seed: int, width: int = 640, height: int = 480,
                 f: float = 525.0, clearance: float = 0.5) -> List[Camera]:
    """``n`` keyframes on a Catmull-Rom spline through six random free-space
    points of the room, each looking along the path with a small random yaw
    and a slight downward pitch."""
    rng = np.random.default_rng(seed)
    spline, segs = _spline_path(scene, rng, clearance)
    cams = []
    for i in range(n):
        u = segs * (i + 0.5) / n
        pos, tan = spline(u)
        yaw = np.deg2rad(rng.uniform(-10, 10))
        pitch = np.deg2rad(rng.uniform(-15, 0))
        look = _heading(tan, yaw, pitch)
        cams.append(Camera(f, f, width / 2.0 - 0.5, height / 2.0 - 0.5, width, height,
                           look_at(pos, pos + look)))
    return cams


def sequence_cameras(scene: Scene, n: int, seed: int, width: int = 640, height: int = 480,
                     f: float = 525.0, clearance: float = 0.5, span: float = 1.0,
                     smooth: float = 0.1) -> List[Camera]:
    """A smooth camera sequence of ``n`` frames along the same kind of spline
    (the first ``span`` of it). The heading follows the path direction,
    low-passed (Gaussian over ``smooth`` of the sequence) so sharp bends of the
    path turn the camera gradually, plus a slowly oscillating yaw (+-10
    degrees) and pitch (-12..-4 degrees): consecutive frames are close in
    pose."""
    rng = np.random.default_rng(seed)
    spline, segs = _spline_path(scene, rng, clearance)
    ph = rng.uniform(0, 2 * np.pi, 2)
    us = segs * span * np.arange(n) / max(1, n - 1) * 0.999
    pos, yaw = [], []
    for u in us:
        p, tan = spline(u)
        pos.append(p)
        yaw.append(np.arctan2(tan[2], tan[0]) if np.hypot(tan[0], tan[2]) > 1e-6 else 0.0)
    yaw = np.unwrap(np.array(yaw))
    sig = max(1e-9, smooth * n)
    k = np.arange(-int(3 * sig) - 1, int(3 * sig) + 2)
    w = np.exp(-0.5 * (k / sig) ** 2)
    pad = np.concatenate([np.full(len(k) // 2, yaw[0]), yaw, np.full(len(k) // 2, yaw[-1])])
    yaw = np.convolve(pad, w / w.sum(), mode="valid")[:n]
    cams = []
    for i, u in enumerate(us):
        a = yaw[i] + np.deg2rad(10.0 * np.sin(2 * np.pi * u / 3.0 + ph[0]))
        pitch = np.deg2rad(-8.0 + 4.0 * np.sin(2 * np.pi * u / 2.0 + ph[1]))
        look = np.array([np.cos(pitch) * np.cos(a), np.sin(pitch), np.cos(pitch) * np.sin(a)])
        cams.append(Camera(f, f, width / 2.0 - 0.5, height / 2.0 - 0.5, width, height,
                           look_at(pos[i], pos[i] + look)))
    return cams


def sensor_frames(scene: Scene, cams: Sequence[Camera], seed: int, depth_noise: float = 0.01,
                  missing: float = 0.02):
    """Simulated RGB-D frames: per pixel, the first analytic surface hit along
    the pinhole ray gives the z-depth (noise N(0, (depth_noise z^2)^2), a
    fraction ``missing`` of pixels set to 0 = invalid) and a colour (the
    primitive's base colour with a smooth pattern, clipped to [0, 1]).
    Returns (rgb [n,3] float32, depth_z [n] float32) for ``dense_rays(cams)``.
    """
    rng = np.random.default_rng(seed)
    rgbs, depths = [], []
    wall_rgb = np.array([[0.8, 0.75, 0.7], [0.6, 0.65, 0.7], [0.5, 0.5, 0.45]])
    for cam in cams:
        W, H = int(cam.width), int(cam.height)
        u, v = np.meshgrid(np.arange(W) + 0.5, np.arange(H) + 0.5)
        dc = np.stack([(u - cam.cx) / cam.fx, (v - cam.cy) / cam.fy, np.ones_like(u)], -1)
        dc = dc.reshape(-1, 3)
        zlen = np.linalg.norm(dc, axis=-1)
        T = np.asarray(cam.T_wc, np.float64).reshape(3, 4)
        d = (dc @ T[:, :3].T) / zlen[:, None]
        o = T[:, 3]
        # walls: exit of the room box
        with np.errstate(divide="ignore", invalid="ignore"):
            ta = (scene.room_lo - o) / d
            tb = (scene.room_hi - o) / d
        tfar = np.maximum(ta, tb)
        tfar = np.where(np.isfinite(tfar), tfar, np.inf)
        axis = np.argmin(tfar, axis=-1)
        t_best = np.min(tfar, axis=-1)
        col = wall_rgb[axis]
        for p in scene.prims:
            if p["kind"] == "sphere":
                oc = o - p["c"]
                bq = d @ oc
                cq = oc @ oc - p["r"] ** 2
                disc = bq * bq - cq
                th = -bq - np.sqrt(np.maximum(disc, 0.0))
                hit = (disc > 0) & (th > 1e-6)
            else:
                with np.errstate(divide="ignore", invalid="ignore"):
                    t1 = (p["c"] - p["half"] - o) / d
                    t2 = (p["c"] + p["half"] - o) / d
                tn = np.nanmax(np.minimum(t1, t2), axis=-1)
                tf = np.nanmin(np.maximum(t1, t2), axis=-1)
                th = tn
                hit = (tf > tn) & (tn > 1e-6)
            closer = hit & (th < t_best)
            t_best = np.where(closer, th, t_best)
            col = np.where(closer[:, None], p["rgb"][None, :], col)
        X = o + t_best[:, None] * d
        pattern = 0.5 + 0.5 * np.sin(7.0 * X[:, 0]) * np.cos(5.0 * X[:, 2] + 3.0 * X[:, 1])
        rgb = np.clip(col * (0.7 + 0.3 * pattern[:, None])
                      + 0.01 * rng.standard_normal((W * H, 3)), 0.0, 1.0)
        z = t_best / zlen
        z = z + depth_noise * z * z * rng.standard_normal(W * H)
        z[rng.random(W * H) < missing] = 0.0
        rgbs.append(rgb.astype(np.float32))
        depths.append(z.astype(np.float32))
    return np.concatenate(rgbs), np.concatenate(depths)


def sensor_frames_torch(scene: Scene, cams: Sequence[Camera], seed: int, device: str = "cuda",
                        depth_noise: float = 0.01, missing: float = 0.02):
    """``sensor_frames`` computed with torch on ``device`` (same sensor model;
    the noise comes from a torch generator seeded with ``seed``), for frames
    too many or too large for numpy."""
    import torch

    gen = torch.Generator(device=device)
    gen.manual_seed(seed)
    f64 = torch.float64
    wall_rgb = torch.tensor([[0.8, 0.75, 0.7], [0.6, 0.65, 0.7], [0.5, 0.5, 0.45]],
                            dtype=f64, device=device)
    rlo = torch.tensor(scene.room_lo, dtype=f64, device=device)
    rhi = torch.tensor(scene.room_hi, dtype=f64, device=device)
    rgbs, depths = [], []
    for cam in cams:
        W, H = int(cam.width), int(cam.height)
        v, u = torch.meshgrid(torch.arange(H, device=device, dtype=f64) + 0.5,
                              torch.arange(W, device=device, dtype=f64) + 0.5, indexing="ij")
        dc = torch.stack([(u - cam.cx) / cam.fx, (v - cam.cy) / cam.fy, torch.ones_like(u)], -1)
        dc = dc.reshape(-1, 3)
        zlen = dc.norm(dim=-1)
        T = torch.tensor(np.asarray(cam.T_wc, np.float64).reshape(3, 4), device=device)
        d = (dc @ T[:, :3].T) / zlen[:, None]
        o = T[:, 3]
        ta = (rlo - o) / d
        tb = (rhi - o) / d
        tfar = torch.maximum(ta, tb)
        tfar = torch.where(torch.isfinite(tfar), tfar, torch.full_like(tfar, float("inf")))
        t_best, axis = tfar.min(dim=-1)
        col = wall_rgb[axis]
        for p in scene.prims:
            c = torch.tensor(p["c"], dtype=f64, device=device)
            if p["kind"] == "sphere":
                oc = o - c
                bq = d @ oc
                cq = oc @ oc - p["r"] ** 2
                disc = bq * bq - cq
                th = -bq - torch.sqrt(disc.clamp(min=0))
                hit = (disc > 0) & (th > 1e-6)
            else:
                hf = torch.tensor(p["half"], dtype=f64, device=device)
                t1 = (c - hf - o) / d
                t2 = (c + hf - o) / d
                tn = torch.nan_to_num(torch.minimum(t1, t2), nan=-float("inf")).max(dim=-1).values
                tf = torch.nan_to_num(torch.maximum(t1, t2), nan=float("inf")).min(dim=-1).values
                th = tn
                hit = (tf > tn) & (tn > 1e-6)
            closer = hit & (th < t_best)
            t_best = torch.where(closer, th, t_best)
            col = torch.where(closer[:, None], torch.tensor(p["rgb"], dtype=f64, device=device), col)
        X = o + t_best[:, None] * d
        pattern = 0.5 + 0.5 * torch.sin(7.0 * X[:, 0]) * torch.cos(5.0 * X[:, 2] + 3.0 * X[:, 1])
        noise = torch.randn((W * H, 3), generator=gen, device=device, dtype=f64)
        rgb = (col * (0.7 + 0.3 * pattern[:, None]) + 0.01 * noise).clamp(0.0, 1.0)
        z = t_best / zlen
        z = z + depth_noise * z * z * torch.randn(W * H, generator=gen, device=device, dtype=f64)
        z = torch.where(torch.rand(W * H, generator=gen, device=device, dtype=f64) < missing,
                        torch.zeros_like(z), z)
        rgbs.append(rgb.float())
        depths.append(z.float())
    return torch.cat(rgbs), torch.cat(depths)


def mixed_resolution_cameras(scene: Scene, n: int, seed: int,
                             sizes=((320, 240), (640, 480), (848, 480), (1200, 680))):
    """``n`` keyframes whose resolution is drawn uniformly from ``sizes``,
    focal length scaled with the width (525 px at 640)."""
    rng = np.random.default_rng(seed)
    base = room_cameras(scene, n, seed + 7)
    out = []
    for c in base:
        W, H = sizes[int(rng.integers(len(sizes)))]
        f = 525.0 * W / 640.0
        out.append(Camera(f, f, W / 2.0 - 0.5, H / 2.0 - 0.5, W, H, c.T_wc))
    return out


# ----------------------------------------------------- named workloads
WORKLOADS = {
    # name: (R, occupancy, n_prims, seed)
    "room256": (256, 0.10, 20, 1002),
    "room512": (512, 0.05, 20, 1003),
    "room512mix": (512, 0.05, 20, 1004),
    "house1024": (1024, 0.02, 200, 1005),   # house_scene: multi-room, 12.8 m
}

# Scene variants per workload (room_scene keyword arguments). The tracking
# workload's room is opaque with a texture that is smooth over 10 cm: on the
# semi-transparent room (about 30% of each ray's transmittance is left after
# the room, so expected depths blend several surfaces) and on per-vertex
# white-noise texture (which decorrelates within one 1.25 cm voxel), the loss
# over poses has minima other than the true pose within 3 cm of it.
WORKLOAD_STYLE = {
    "room512": dict(density_scale=8.0, vertex_noise=0.03, smooth_texture=0.2, texture_cell=0.1),
}


def workload_scene(name: str) -> Scene:
    """The room scene of workload ``name`` (``WORKLOADS``, ``WORKLOAD_STYLE``)."""
    R, occ, npr, seed = WORKLOADS[name]
    return room_scene(R, occ, npr, seed, **WORKLOAD_STYLE.get(name, {}))
