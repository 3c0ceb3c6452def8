"""FP64 CPU oracle for the Plenoxel RGB-D render, grid adjoint and pose Jacobian.

TEST INFRASTRUCTURE. Only ``tests/``, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` may import this
package. The product path (``paper_2307_03404_b300``) never imports it, and it
never imports the product path: the two share nothing but the seeded input
generators, which hold none of the method's arithmetic.

The arithmetic lives in ``plx_oracle.c`` (plain C, double precision, written
from the paper's Eq. 1-16 and Appendix A); this module only marshals numpy
arrays into it. Build it with ``python -m oracle.build`` (``__graft_entry__``'s
``build()`` does this too).

Citations (arXiv 2307.03404):
  render            Sec. 4, Eq. 1 (colour), Eq. 2 (transmittance), Eq. 3 (depth)
  grad_grid         Sec. 5.2, Eq. 4-5 (losses), Eq. 6-10 (derivatives), Eq. 11
  pose_jacobian     Sec. 5.3, Eq. 12-14, Appendix A Eq. 15-16
  render_frozen     the function whose derivative Eq. 12-14 define
  pose_step, se3_exp  Sec. 5.3 (the pose is optimised directly)
  sh_basis          Sec. 5.2 (nine SH coefficients per colour channel)
  trilerp           Appendix A, Eq. 15-16
"""
from __future__ import annotations

import ctypes as C
import os
from types import SimpleNamespace

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libplx_oracle.so")


class OrcGrid(C.Structure):
    _fields_ = [
        ("res", C.c_int32 * 3),
        ("lo", C.c_double * 3),
        ("hi", C.c_double * 3),
        ("links", C.c_void_p),
        ("density", C.c_void_p),
        ("sh", C.c_void_p),
        ("n_alloc", C.c_int64),
    ]


class OrcCamera(C.Structure):
    _fields_ = [
        ("fx", C.c_double), ("fy", C.c_double), ("cx", C.c_double), ("cy", C.c_double),
        ("width", C.c_int32), ("height", C.c_int32),
        ("T_wc", C.c_double * 12),
    ]


class OrcOpts(C.Structure):
    _fields_ = [
        ("step", C.c_double),
        ("near_t", C.c_double),
        ("stop_T", C.c_double),
        ("bg", C.c_double * 3),
        ("lambda_d", C.c_double),
        ("max_samples", C.c_int32),
        ("color_act", C.c_int32),
        ("depth_is_z", C.c_int32),
        ("dir_term", C.c_int32),
    ]


_lib = None


def _load():
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise RuntimeError(
            f"oracle library {LIB_PATH} is not built; run `python -m oracle.build`")
    lib = C.CDLL(LIB_PATH)
    P = C.c_void_p
    lib.orc_set_threads.argtypes = [C.c_int]
    lib.orc_get_threads.restype = C.c_int
    lib.orc_sh_basis.argtypes = [P, P]
    lib.orc_sh_basis_grad.argtypes = [P, P]
    lib.orc_trilerp.argtypes = [P, C.c_double, C.c_double, C.c_double, P, P]
    lib.orc_render.argtypes = [P, P, C.c_int64, P, P, P, P, P, P, P, P]
    lib.orc_render_frozen.argtypes = [P, P, C.c_int64, P, P, P, P, P, P]
    lib.orc_grad_grid.argtypes = [P, P, C.c_int64, P, P, P, P, P, P, P, P]
    lib.orc_grad_grid.restype = C.c_double
    lib.orc_pose_jacobian.argtypes = [P, P, C.c_int64, P, P, P, P, P, P, P, P, P, P]
    lib.orc_pose_jacobian.restype = C.c_double
    lib.orc_pixel_ray.argtypes = [P, P, C.c_int32, C.c_double, P, P, P, P]
    lib.orc_pixel_ray.restype = C.c_int
    lib.orc_se3_exp.argtypes = [P, P]
    lib.orc_pose_step.argtypes = [P, P, C.c_double, P, P]
    lib.orc_grow.argtypes = [P, P, P, P, C.c_int64, P, C.c_int32, P, C.c_int32, C.c_double]
    lib.orc_pose_step.restype = C.c_int
    lib.orc_grow.restype = C.c_int64
    lib.orc_pose_step_lm.argtypes = [P, P, C.c_double, P, C.c_double, C.c_double, P, P]
    lib.orc_pose_step_lm.restype = C.c_int
    _lib = lib
    return lib


def _ptr(a):
    return a.ctypes.data_as(C.c_void_p) if a is not None else None


def _f64(a, shape=None):
    a = np.ascontiguousarray(np.asarray(a, dtype=np.float64))
    if shape is not None:
        a = a.reshape(shape)
    return a


def set_threads(n: int) -> None:
    _load().orc_set_threads(int(n))


def get_threads() -> int:
    return int(_load().orc_get_threads())


class _Prepared:
    """Keeps the numpy buffers alive while C holds raw pointers to them."""

    def __init__(self, grid, cams, rays, opts):
        self.links = np.ascontiguousarray(grid.links, dtype=np.int32)
        self.density = _f64(grid.density)
        self.sh = _f64(grid.sh).reshape(-1, 27)
        g = OrcGrid()
        g.res[:] = [int(v) for v in grid.res]
        g.lo[:] = [float(v) for v in grid.lo]
        g.hi[:] = [float(v) for v in grid.hi]
        g.links = self.links.ctypes.data
        g.density = self.density.ctypes.data
        g.sh = self.sh.ctypes.data
        g.n_alloc = int(self.density.shape[0])
        self.grid = g
        cams = list(cams)
        self.cams = (OrcCamera * len(cams))()
        for i, c in enumerate(cams):
            self.cams[i].fx, self.cams[i].fy = float(c.fx), float(c.fy)
            self.cams[i].cx, self.cams[i].cy = float(c.cx), float(c.cy)
            self.cams[i].width, self.cams[i].height = int(c.width), int(c.height)
            self.cams[i].T_wc[:] = [float(v) for v in np.asarray(c.T_wc, dtype=np.float64).reshape(12)]
        if rays is None:
            cid, pix = [], []
            for i, c in enumerate(cams):
                n = int(c.width) * int(c.height)
                cid.append(np.full(n, i, np.int32))
                pix.append(np.arange(n, dtype=np.int32))
            self.cam_id = np.concatenate(cid)
            self.pix = np.concatenate(pix)
        else:
            self.cam_id = np.ascontiguousarray(rays[0], dtype=np.int32)
            self.pix = np.ascontiguousarray(rays[1], dtype=np.int32)
        self.n = int(self.pix.shape[0])
        o = OrcOpts()
        o.step = float(opts["step"])
        o.near_t = float(opts.get("near", 0.0))
        o.stop_T = float(opts.get("stop_T", 0.0))
        o.bg[:] = [float(v) for v in opts.get("bg", (0.0, 0.0, 0.0))]
        o.lambda_d = float(opts.get("lambda_d", 1.0))
        o.max_samples = int(opts.get("max_samples", 1 << 30))
        o.color_act = {"sigmoid": 0, "identity": 1}[opts.get("color_act", "sigmoid")]
        o.depth_is_z = int(bool(opts.get("depth_is_z", True)))
        o.dir_term = int(bool(opts.get("dir_term", False)))
        self.opts = o

    def args(self):
        return (C.byref(self.grid), self.cams, C.c_int64(self.n), _ptr(self.cam_id),
                _ptr(self.pix), C.byref(self.opts))


def render(grid, cams, opts, rays=None):
    """Rendered colour, expected depth, final transmittance and sample counts.

    ``rays`` is ``(cam_id, pixel)`` int32 arrays (pixel = v*W + u), or None for
    every pixel of every camera in order. ``opts`` is a dict with ``step``
    (world units) and optionally ``near``, ``stop_T``, ``bg``, ``lambda_d``,
    ``max_samples``, ``color_act`` ('sigmoid'|'identity'), ``depth_is_z``.
    """
    lib = _load()
    p = _Prepared(grid, cams, rays, opts)
    rgb = np.zeros((p.n, 3))
    depth = np.zeros(p.n)
    T = np.zeros(p.n)
    nm = np.zeros(p.n, np.int64)
    na = np.zeros(p.n, np.int64)
    lib.orc_render(*p.args(), _ptr(rgb), _ptr(depth), _ptr(T), _ptr(nm), _ptr(na))
    return SimpleNamespace(rgb=rgb, depth=depth, T_final=T, n_marched=nm, n_alloc=na)


def render_frozen(grid, cams, opts, xi, rays=None):
    """Forward with t_k and SH direction frozen at each camera's pose and the
    sample positions moved by exp(xi^) (world frame, on the left)."""
    lib = _load()
    p = _Prepared(grid, cams, rays, opts)
    xi = _f64(xi, (6,))
    rgb = np.zeros((p.n, 3))
    depth = np.zeros(p.n)
    lib.orc_render_frozen(*p.args(), _ptr(xi), _ptr(rgb), _ptr(depth))
    return SimpleNamespace(rgb=rgb, depth=depth)


def grad_grid(grid, cams, opts, rgb_t, depth_t, rays=None):
    """Loss L = L_p + lambda_d L_g and its gradient to every grid value.

    Returns grad_density [n_alloc], grad_sh [n_alloc, 27], loss, M.
    """
    lib = _load()
    p = _Prepared(grid, cams, rays, opts)
    rgb_t = _f64(rgb_t, (p.n, 3))
    depth_t = _f64(depth_t, (p.n,))
    gd = np.zeros(p.density.shape[0])
    gs = np.zeros((p.density.shape[0], 27))
    M = C.c_int64(0)
    loss = lib.orc_grad_grid(*p.args(), _ptr(rgb_t), _ptr(depth_t), _ptr(gd), _ptr(gs),
                             C.byref(M))
    return SimpleNamespace(grad_density=gd, grad_sh=gs, loss=float(loss), M=int(M.value))


def pose_jacobian(grid, cams, opts, rgb_t, depth_t, rays=None):
    """Per-ray J [n,4,6] and residual r [n,4]; H = sum J^T W J [6,6],
    b = sum J^T W r [6], loss = sum r^T W r, M."""
    lib = _load()
    p = _Prepared(grid, cams, rays, opts)
    rgb_t = _f64(rgb_t, (p.n, 3))
    depth_t = _f64(depth_t, (p.n,))
    J = np.zeros((p.n, 4, 6))
    r = np.zeros((p.n, 4))
    H = np.zeros((6, 6))
    b = np.zeros(6)
    M = C.c_int64(0)
    loss = lib.orc_pose_jacobian(*p.args(), _ptr(rgb_t), _ptr(depth_t), _ptr(J), _ptr(r),
                                 _ptr(H), _ptr(b), C.byref(M))
    return SimpleNamespace(J=J, resid=r, H=H, b=b, loss=float(loss), M=int(M.value))


def grow(res, lo, hi, links, n_alloc, cams, depth, band, depth_is_z=True):
    """Grid growth from observed depth (Sec. 6.1's dynamic grid): returns
    (new links [res_z, res_y, res_x] int32, vertices added). ``depth`` holds
    every pixel of every camera, camera after camera, row-major (float32, as
    a sensor gives it); a pixel whose depth is not positive and finite adds
    nothing."""
    lib = _load()
    links = np.array(links, dtype=np.int32, copy=True, order="C")
    r = np.array([int(v) for v in res], np.int32)
    lo_, hi_ = _f64(lo), _f64(hi)
    cams = list(cams)
    oc = (OrcCamera * len(cams))()
    for i, c in enumerate(cams):
        oc[i].fx, oc[i].fy, oc[i].cx, oc[i].cy = float(c.fx), float(c.fy), float(c.cx), float(c.cy)
        oc[i].width, oc[i].height = int(c.width), int(c.height)
        oc[i].T_wc[:] = [float(v) for v in np.asarray(c.T_wc, dtype=np.float64).reshape(12)]
    d = np.ascontiguousarray(depth, dtype=np.float32)
    if d.shape[0] != sum(int(c.width) * int(c.height) for c in cams):
        raise ValueError("depth must hold every pixel of every camera")
    added = lib.orc_grow(_ptr(r), _ptr(lo_), _ptr(hi_), _ptr(links), C.c_int64(int(n_alloc)), oc,
                         C.c_int32(len(cams)), _ptr(d), C.c_int32(int(bool(depth_is_z))),
                         C.c_double(float(band)))
    if added < 0:
        raise MemoryError("orc_grow")
    return links, int(added)


def pixel_ray(grid, cam, pixel, near=0.0):
    """(o, d, |d_c|, (t_min, t_max), hit) of one pixel's ray."""
    p = _Prepared(grid, [cam], (np.zeros(1, np.int32), np.array([pixel], np.int32)),
                  {"step": 1.0})
    o, d, n, tr = np.zeros(3), np.zeros(3), np.zeros(1), np.zeros(2)
    hit = _load().orc_pixel_ray(C.byref(p.grid), p.cams, C.c_int32(pixel), C.c_double(near),
                                _ptr(o), _ptr(d), _ptr(n), _ptr(tr))
    return o, d, float(n[0]), tr, bool(hit)


def se3_exp(xi):
    """exp of the twist (rho, phi) as a 3x4 [R | t]."""
    xi = _f64(xi, (6,))
    T = np.zeros(12)
    _load().orc_se3_exp(_ptr(xi), _ptr(T))
    return T.reshape(3, 4)


def pose_step(H, b, T_wc, damping=0.0):
    """Solve (H + damping I) xi = -b and return (exp(xi^) T_wc, xi, ok)."""
    H = _f64(H, (36,))
    b = _f64(b, (6,))
    T = _f64(T_wc, (12,)).copy()
    xi = np.zeros(6)
    st = _load().orc_pose_step(_ptr(H), _ptr(b), C.c_double(damping), _ptr(T), _ptr(xi))
    return T.reshape(3, 4), xi, st == 0


def pose_step_lm(H, b, loss, state, T_wc, lambda_init=1e-3, factor=10.0):
    """Levenberg-Marquardt pose step (see orc_pose_step_lm): returns (new pose
    [3, 4], xi, status); ``state`` (float64 [64], zeroed before the first
    call) is updated in place."""
    H = _f64(H, (36,))
    b = _f64(b, (6,))
    T = _f64(T_wc, (12,)).copy()
    assert state.dtype == np.float64 and state.shape == (64,) and state.flags.c_contiguous
    xi = np.zeros(6)
    st = _load().orc_pose_step_lm(_ptr(H), _ptr(b), C.c_double(float(loss)), _ptr(state),
                                  C.c_double(lambda_init), C.c_double(factor), _ptr(T), _ptr(xi))
    return T.reshape(3, 4), xi, int(st)


def sh_basis(d):
    d = _f64(d, (3,))
    Y = np.zeros(9)
    _load().orc_sh_basis(_ptr(d), _ptr(Y))
    return Y


def sh_basis_grad(d):
    """[9, 3]: gradient of the nine SH polynomials at d (tracking-Jacobian variant)."""
    d = _f64(d, (3,))
    G = np.zeros((9, 3))
    _load().orc_sh_basis_grad(_ptr(d), _ptr(G))
    return G


def trilerp(V, x, y, z):
    """Interpolant of corner values V[c], c = dx + 2dy + 4dz, and its gradient."""
    V = _f64(V, (8,))
    f = np.zeros(1)
    g = np.zeros(3)
    _load().orc_trilerp(_ptr(V), C.c_double(x), C.c_double(y), C.c_double(z), _ptr(f), _ptr(g))
    return float(f[0]), g


# ----------------------------------------------------------- optimisers
# Sec. 5.4: RMSProp for the mapping, Adam for the tracking on rays drawn at
# random from the current image. Plain formulas, FP64.

def rmsprop(x, g, v, lr, alpha, eps):
    """One RMSProp step: v <- alpha v + (1 - alpha) g^2, x <- x - lr g / (sqrt(v) + eps)."""
    x, g, v = (np.asarray(a, np.float64) for a in (x, g, v))
    v = alpha * v + (1.0 - alpha) * g * g
    return x - lr * g / (np.sqrt(v) + eps), v


def adam(g, m, v, t, lr, b1, b2, eps):
    """One Adam step on a parameter vector; t counts from 1. Returns (step, m, v)."""
    m = b1 * m + (1.0 - b1) * g
    v = b2 * v + (1.0 - b2) * g * g
    mh = m / (1.0 - b1 ** t)
    vh = v / (1.0 - b2 ** t)
    return -lr * mh / (np.sqrt(vh) + eps), m, v


_GOLDEN_GAMMA = 0x9E3779B97F4A7C15
_MASK = (1 << 64) - 1


def splitmix64(seed, k):
    """SplitMix64 (Steele, Lea and Flood, 2014) as a counter-based generator:
    value k of stream ``seed`` is mix(seed + (k + 1) * golden gamma)."""
    z = (int(seed) + (int(k) + 1) * _GOLDEN_GAMMA) & _MASK
    z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & _MASK
    z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & _MASK
    return z ^ (z >> 31)


def random_pixels(seed, t, n, n_pixels):
    """The n pixels of tracking iteration t: splitmix64(seed, t n + i) mod n_pixels."""
    return np.array([splitmix64(seed, t * n + i) % n_pixels for i in range(n)], np.int32)


def adam_track(grid, cam, opts, rgb_t, depth_t, n_rays, seed, iters, lr, b1=0.9, b2=0.999,
               eps=1e-8):
    """The paper's tracker: per iteration, n_rays random pixels of the frame,
    the loss gradient 2 J^T W r with respect to a left perturbation (Eq. 12-14),
    an Adam step xi and T <- exp(xi^) T. rgb_t / depth_t hold the whole frame.
    Returns the final pose and the per-iteration losses."""
    T = np.asarray(cam.T_wc, np.float64).reshape(3, 4)
    m, v = np.zeros(6), np.zeros(6)
    npx = int(cam.width) * int(cam.height)
    losses = []
    for t in range(iters):
        pix = random_pixels(seed, t, n_rays, npx)
        pj = pose_jacobian(grid, [cam.with_pose(T)], opts, np.asarray(rgb_t)[pix],
                           np.asarray(depth_t)[pix], rays=(np.zeros(n_rays, np.int32), pix))
        xi, m, v = adam(2.0 * pj.b, m, v, t + 1, lr, b1, b2, eps)
        E = np.vstack([se3_exp(xi), [0, 0, 0, 1]])
        T = (E @ np.vstack([T, [0, 0, 0, 1]]))[:3]
        losses.append(pj.loss)
    return T, losses
