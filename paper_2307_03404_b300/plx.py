"""ctypes binding of ``libplx.so`` (C ABI in ``include/plx.h``).

Argument marshalling only: every step of the render, its adjoints and the pose
step runs in the library's CUDA kernels. PyTorch provides device memory and
the current stream. Importing this module loads the library and raises if it
is missing: there is no CPU fallback.

Function names follow the C ABI (``grid_create`` -> ``plx_grid_create`` ...).
"""
from __future__ import annotations

import ctypes as C
import os
from dataclasses import dataclass
from typing import Sequence

import numpy as np
import torch

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.environ.get("PLX_LIBRARY") or os.path.join(_HERE, "libplx.so")

STORE_F32, STORE_BF16, STORE_F16, STORE_F32_BF16 = 0, 1, 2, 3
STORAGE = {"f32": STORE_F32, "bf16": STORE_BF16, "f16": STORE_F16, "f32_bf16": STORE_F32_BF16}
ACT_SIGMOID, ACT_IDENTITY = 0, 1
MAX_CAMERAS = 128
GRAD_STRIDE = 32
POSE_VIEW_DIR = 1
FINE_FORWARD, FINE_ADJOINT, FINE_POSE, FINE_BATCH = 1, 2, 4, 8

STATUS = {0: "PLX_OK", 1: "PLX_EINVAL", 2: "PLX_ENOMEM", 3: "PLX_ECUDA",
          4: "PLX_EDEVICE_CHECK", 5: "PLX_ETIMEOUT", 6: "PLX_EUNSUPPORTED"}


class PlxError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{STATUS.get(status, status)}: {msg}")
        self.status = status


class GridDesc(C.Structure):
    _fields_ = [("res", C.c_int32 * 3), ("lo", C.c_double * 3), ("hi", C.c_double * 3),
                ("n_alloc", C.c_int64), ("storage", C.c_int32), ("reserved", C.c_int32)]


class Intrinsics(C.Structure):
    _fields_ = [("fx", C.c_double), ("fy", C.c_double), ("cx", C.c_double), ("cy", C.c_double),
                ("width", C.c_int32), ("height", C.c_int32)]


class Cameras(C.Structure):
    _fields_ = [("n_cams", C.c_int32), ("reserved", C.c_int32),
                ("intr", C.POINTER(Intrinsics)), ("poses", C.c_void_p)]


class Rays(C.Structure):
    _fields_ = [("n_rays", C.c_int64), ("cam_id", C.c_void_p), ("pixel", C.c_void_p)]


class Work(C.Structure):
    _fields_ = [("cam", C.c_int32), ("mode", C.c_int32)]


WORK_MAP, WORK_TRACK = 0, 1


class LaunchConfig(C.Structure):
    _fields_ = [("block_shift", C.c_int32), ("forward_blocks", C.c_int32),
                ("adjoint_blocks", C.c_int32), ("pose_blocks", C.c_int32),
                ("batch_blocks", C.c_int32), ("fine_skip", C.c_int32),
                ("seg_rays", C.c_int32)]


class RenderOpts(C.Structure):
    _fields_ = [("step", C.c_double), ("near_t", C.c_double), ("stop_T", C.c_double),
                ("bg", C.c_float * 3), ("lambda_d", C.c_float), ("max_samples", C.c_int32),
                ("color_act", C.c_int32), ("depth_is_z", C.c_int32), ("pose_flags", C.c_int32),
                ("sample_cache", C.c_void_p), ("sample_cap", C.c_int32),
                ("sample_rays", C.c_int64), ("ray_range", C.c_void_p)]


SYMBOLS = ["plx_last_error", "plx_version", "plx_grid_create", "plx_grid_upload",
           "plx_grid_download", "plx_grid_info", "plx_grid_destroy", "plx_render_forward",
           "plx_render_backward_grid", "plx_render_backward_pose", "plx_pose_step",
           "plx_grid_check", "plx_render_backward_pose_noalloc", "plx_render_batch",
           "plx_grid_rmsprop", "plx_track_adam_step", "plx_grid_get_config",
           "plx_grid_set_config", "plx_grid_grow", "plx_pose_step_lm", "plx_sample_cache_bytes",
           "plx_probe", "plx_noalloc_error"]


def _load():
    if not os.path.exists(LIB_PATH):
        raise RuntimeError(f"{LIB_PATH} is missing: build it with "
                           "`python -m paper_2307_03404_b300.build` (there is no CPU fallback)")
    lib = C.CDLL(LIB_PATH)
    P, I32, I64, D = C.c_void_p, C.c_int32, C.c_int64, C.c_double
    lib.plx_last_error.restype = C.c_char_p
    lib.plx_version.restype = C.c_char_p
    sig = {
        "plx_grid_create": [C.POINTER(GridDesc), P, P, P, P, C.POINTER(P)],
        "plx_grid_upload": [P, P, P, P],
        "plx_grid_download": [P, P, P, P],
        "plx_grid_info": [P, C.POINTER(GridDesc)],
        "plx_grid_destroy": [P],
        "plx_grid_check": [P, P],
        "plx_render_forward": [P, C.POINTER(Cameras), C.POINTER(Rays), C.POINTER(RenderOpts),
                               P, P, P, P, P],
        "plx_render_backward_grid": [P, C.POINTER(Cameras), C.POINTER(Rays),
                                     C.POINTER(RenderOpts), P, P, P, P, P, P, P],
        "plx_render_backward_pose": [P, C.POINTER(Cameras), I32, C.POINTER(Rays),
                                     C.POINTER(RenderOpts), P, P, P, P, P, P],
        "plx_pose_step": [P, P, D, P, P, P, P],
        "plx_grid_get_config": [P, C.POINTER(LaunchConfig)],
        "plx_grid_set_config": [P, C.POINTER(LaunchConfig), P],
        "plx_grid_rmsprop": [P, P, P, C.c_float, C.c_float, C.c_float, C.c_float, I32, P],
        "plx_track_adam_step": [P, C.POINTER(Cameras), I32, C.POINTER(RenderOpts), I32, C.c_uint64,
                                P, P, P, D, D, D, D, P, P, P, P],
        "plx_render_batch": [P, C.POINTER(Cameras), C.POINTER(Work), I32, C.POINTER(RenderOpts),
                             P, P, P, P, P, P, P, P],
        "plx_pose_step_lm": [P, P, P, P, D, D, P, P, P, P],
        "plx_grid_grow": [C.POINTER(GridDesc), P, C.POINTER(Cameras), P, I32, D, P, P],
        "plx_probe": [I32, P, I64, I32, I32, I32, P],
        "plx_noalloc_error": [P, P],
        "plx_render_backward_pose_noalloc": [C.POINTER(GridDesc), P, P, C.POINTER(Cameras), I32,
                                             C.POINTER(Rays), C.POINTER(RenderOpts), P, P, P, P,
                                             P, P],
    }
    for name, args in sig.items():
        f = getattr(lib, name)
        f.argtypes = args
        f.restype = C.c_int
    lib.plx_sample_cache_bytes.argtypes = [I64, I32]
    lib.plx_sample_cache_bytes.restype = C.c_int64
    return lib


_lib = _load()


def _check(status):
    if status != 0:
        raise PlxError(status, _lib.plx_last_error().decode())


def _ptr(t):
    return None if t is None else C.c_void_p(t.data_ptr())


def _stream(stream=None):
    s = stream if stream is not None else torch.cuda.current_stream()
    return C.c_void_p(s.cuda_stream)


_NVTX = os.environ.get("PLX_NVTX") == "1"


def _ranged(fn):
    """With PLX_NVTX=1, wrap an entry point in an NVTX range of its name (for
    timeline profilers); otherwise return it unchanged."""
    if not _NVTX:
        return fn
    import functools

    @functools.wraps(fn)
    def wrapper(*a, **kw):
        torch.cuda.nvtx.range_push("plx." + fn.__name__)
        try:
            return fn(*a, **kw)
        finally:
            torch.cuda.nvtx.range_pop()

    return wrapper


def version() -> str:
    return _lib.plx_version().decode()


# ----------------------------------------------------------------- grid
class Grid:
    """Library-owned copy of a sparse grid (``plx_grid``)."""

    def __init__(self, res, lo, hi, links, density, sh, storage="f32", stream=None):
        dev = torch.device("cuda")
        links = torch.as_tensor(links).to(dev, torch.int32).contiguous()
        density = torch.as_tensor(density).to(dev, torch.float32).contiguous()
        sh = torch.as_tensor(sh).to(dev, torch.float32).reshape(-1, 27).contiguous()
        d = GridDesc()
        d.res[:] = [int(v) for v in res]
        d.lo[:] = [float(v) for v in lo]
        d.hi[:] = [float(v) for v in hi]
        d.n_alloc = int(density.shape[0])
        d.storage = STORAGE[storage] if isinstance(storage, str) else int(storage)
        h = C.c_void_p()
        _check(_lib.plx_grid_create(C.byref(d), _ptr(links), _ptr(density), _ptr(sh),
                                    _stream(stream), C.byref(h)))
        self._h = h
        self.desc = d
        self.n_alloc = int(d.n_alloc)
        self.storage = d.storage
        self.res = tuple(int(v) for v in res)
        self.lo = np.array(lo, np.float64)
        self.hi = np.array(hi, np.float64)

    @classmethod
    def from_scene(cls, grid, storage="f32"):
        return cls(grid.res, grid.lo, grid.hi, torch.from_numpy(grid.links),
                   torch.from_numpy(np.ascontiguousarray(grid.density, np.float32)),
                   torch.from_numpy(np.ascontiguousarray(grid.sh, np.float32)), storage)

    @property
    def handle(self):
        return self._h

    def upload(self, density, sh, stream=None):
        _check(_lib.plx_grid_upload(self._h, _ptr(density.contiguous()),
                                    _ptr(sh.contiguous()), _stream(stream)))
        self._autograd_values = None  # autograd.mapping_loss uploads again

    def download(self, stream=None):
        density = torch.empty(self.n_alloc, device="cuda")
        sh = torch.empty(self.n_alloc, 27, device="cuda")
        _check(_lib.plx_grid_download(self._h, _ptr(density), _ptr(sh), _stream(stream)))
        return density, sh

    def check(self, stream=None):
        _check(_lib.plx_grid_check(self._h, _stream(stream)))

    def get_config(self) -> dict:
        c = LaunchConfig()
        _check(_lib.plx_grid_get_config(self._h, C.byref(c)))
        return {f: int(getattr(c, f)) for f, _ in LaunchConfig._fields_}

    def set_config(self, stream=None, **kw):
        """Change launch choices (block_shift, fine_skip, forward_blocks,
        adjoint_blocks, pose_blocks, batch_blocks, seg_rays); results do not
        change."""
        cur = self.get_config()
        unknown = set(kw) - set(cur)
        if unknown:
            raise ValueError(f"unknown launch choices {sorted(unknown)}")
        cur.update({k: int(v) for k, v in kw.items()})
        c = LaunchConfig(**cur)
        _check(_lib.plx_grid_set_config(self._h, C.byref(c), _stream(stream)))

    def close(self):
        if getattr(self, "_h", None):
            _check(_lib.plx_grid_destroy(self._h))
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


# -------------------------------------------------------------- cameras
class CameraSet:
    """Intrinsics on the host, poses [n, 12] float64 on the device."""

    def __init__(self, cams: Sequence, poses: torch.Tensor | None = None):
        cams = list(cams)
        if not 1 <= len(cams) <= MAX_CAMERAS:
            raise ValueError(f"1..{MAX_CAMERAS} cameras")
        self._intr = (Intrinsics * len(cams))()
        for i, c in enumerate(cams):
            self._intr[i].fx, self._intr[i].fy = float(c.fx), float(c.fy)
            self._intr[i].cx, self._intr[i].cy = float(c.cx), float(c.cy)
            self._intr[i].width, self._intr[i].height = int(c.width), int(c.height)
        if poses is None:
            poses = torch.tensor(np.stack([np.asarray(c.T_wc, np.float64).reshape(12)
                                           for c in cams]), dtype=torch.float64, device="cuda")
        self.poses = poses.contiguous()
        self.sizes = [(int(c.width), int(c.height)) for c in cams]
        self.n = len(cams)

    def struct(self):
        s = Cameras()
        s.n_cams = self.n
        s.intr = C.cast(self._intr, C.POINTER(Intrinsics))
        s.poses = self.poses.data_ptr()
        return s

    def n_pixels(self, cam=None):
        if cam is not None:
            w, h = self.sizes[cam]
            return w * h
        return sum(w * h for w, h in self.sizes)


def make_rays(cam_id=None, pixel=None):
    """Rays struct plus the tensors it points to (None = dense mode). An empty
    list is passed with non-null placeholder pointers: null means dense."""
    r = Rays()
    keep = []
    if pixel is None:
        r.n_rays = 0
        return r, keep
    pixel = torch.as_tensor(pixel).to("cuda", torch.int32).contiguous()
    r.n_rays = int(pixel.shape[0])
    if cam_id is not None:
        cam_id = torch.as_tensor(cam_id).to("cuda", torch.int32).contiguous()
    if r.n_rays == 0:
        pixel = torch.zeros(1, dtype=torch.int32, device="cuda")
        cam_id = None if cam_id is None else torch.zeros(1, dtype=torch.int32, device="cuda")
    keep.append(pixel)
    r.pixel = pixel.data_ptr()
    if cam_id is not None:
        keep.append(cam_id)
        r.cam_id = cam_id.data_ptr()
    return r, keep


def make_opts(step, near=0.0, stop_T=0.0, bg=(0.0, 0.0, 0.0), lambda_d=1.0,
              max_samples=1 << 30, color_act="sigmoid", depth_is_z=True, view_dir=False):
    o = RenderOpts()
    o.step, o.near_t, o.stop_T = float(step), float(near), float(stop_T)
    o.bg[:] = [float(v) for v in bg]
    o.lambda_d = float(lambda_d)
    o.max_samples = int(min(max_samples, 2 ** 31 - 1))
    o.color_act = {"sigmoid": ACT_SIGMOID, "identity": ACT_IDENTITY}[color_act]
    o.depth_is_z = int(bool(depth_is_z))
    o.pose_flags = POSE_VIEW_DIR if view_dir else 0
    return o


def sample_cache_bytes(n_rays, cap):
    """plx_sample_cache_bytes: bytes of a sample cache for n_rays rays, cap each."""
    return int(_lib.plx_sample_cache_bytes(int(n_rays), int(cap)))


class SampleCache:
    """A sample cache (plx_render_opts.sample_cache) for calls over ``n_rays``
    rays: the forward keeps up to ``cap`` compositing samples per ray and the
    grid adjoint of the same rays reads them back. ``opts(o)`` returns a copy
    of the options naming it; ``counts()`` the number of compositing samples
    per ray of the last forward (may exceed cap)."""

    def __init__(self, n_rays, cap, device="cuda"):
        self.n_rays, self.cap = int(n_rays), int(cap)
        nbytes = sample_cache_bytes(self.n_rays, self.cap)
        if nbytes < 0:
            raise ValueError("n_rays and cap must be >= 0")
        # float32 storage: the base is 16-byte aligned as the ABI asks
        self.buf = torch.empty(max(nbytes // 4, 1), dtype=torch.float32, device=device)

    @classmethod
    def sized_for(cls, grid, cams, opts, rays=None, max_bytes=None, headroom=1.0, stream=None):
        """A cache whose cap holds every ray of this call: one probe forward
        with cap 1 counts each ray's compositing samples, and cap is their
        maximum times ``headroom`` (for later calls on other rays or grid
        values) rounded up to a multiple of 8, at most what fits in
        ``max_bytes`` (default a quarter of the free device memory)."""
        n = cams.n_pixels() if rays is None else int(rays[1].shape[0])
        probe = cls(n, 1)
        render_forward(grid, cams, probe.opts(opts), rays=rays, state=False, stream=stream)
        need = int(probe.counts().max().item()) if n > 0 else 0
        cap = max(8, (int(need * headroom) + 7) // 8 * 8)
        if max_bytes is None:
            max_bytes = torch.cuda.mem_get_info()[0] // 4
        while cap > 8 and sample_cache_bytes(n, cap) > max_bytes:
            cap -= 8
        del probe
        return cls(n, cap)

    @classmethod
    def for_batch(cls, cap, device="cuda"):
        """A cache for plx_render_batch: one row per thread slot of the
        persistent launch (512 per SM), ``cap`` samples each."""
        sms = torch.cuda.get_device_properties(torch.device(device)).multi_processor_count
        return cls(512 * sms, cap, device=device)

    def opts(self, o):
        """A copy of the options ``o`` naming this cache. The copy holds a
        reference to the cache, so its device memory lives as long as options
        that point at it (a temporary SampleCache(...).opts(o) stays valid)."""
        c = RenderOpts.from_buffer_copy(o)
        c.sample_cache = self.buf.data_ptr() if self.cap > 0 else None
        c.sample_cap = self.cap
        c.sample_rays = self.n_rays
        c._cache = self
        c._range = getattr(o, "_range", None)
        return c

    def counts(self):
        """Compositing samples per ray (int32 [n_rays]) from the last forward
        that filled this cache; only a cache with cap > 0 is ever filled."""
        if self.cap == 0:
            raise ValueError("a cache with cap 0 is never filled")
        off = 5 * self.cap * self.n_rays  # float4 [cap][n] then int32 [cap][n], in 4-byte words
        return self.buf[off:off + self.n_rays].view(torch.int32)


class RayRange:
    """A compositing-range buffer (plx_render_opts.ray_range) for calls over
    ``n_rays`` rays: the forward writes each ray's first and one-past-last
    compositing sample, and the re-marching grid adjoint of the same rays
    marches only that range (same gradients, fewer samples: the per-ray state
    a recomputing adjoint keeps, 8 bytes per ray). ``opts(o)`` returns a copy
    of the options naming it."""

    def __init__(self, n_rays, device="cuda"):
        self.n_rays = int(n_rays)
        if self.n_rays < 0:
            raise ValueError("n_rays must be >= 0")
        self.buf = torch.zeros(max(self.n_rays, 1), 2, dtype=torch.int32, device=device)

    def opts(self, o):
        """A copy of the options ``o`` naming this range buffer (the copy
        keeps the buffer, and any sample cache ``o`` names, alive)."""
        c = RenderOpts.from_buffer_copy(o)
        c.ray_range = self.buf.data_ptr()
        c._cache = getattr(o, "_cache", None)
        c._range = self
        return c

    def ranges(self):
        """[n_rays, 2] int32: first and one past the last compositing sample
        of each ray from the last forward that wrote this buffer."""
        return self.buf[:self.n_rays]


def opts_from_dict(d):
    return make_opts(d["step"], d.get("near", 0.0), d.get("stop_T", 0.0), d.get("bg", (0, 0, 0)),
                     d.get("lambda_d", 1.0), d.get("max_samples", 1 << 30),
                     d.get("color_act", "sigmoid"), d.get("depth_is_z", True),
                     d.get("dir_term", False))


# ----------------------------------------------------------- entry points
@_ranged
def render_forward(grid: Grid, cams: CameraSet, opts, rays=None, state=True, counts=False,
                   out=None, stream=None):
    """plx_render_forward. ``rays`` = (cam_id, pixel) or None (dense).
    Returns dict(rgb [n,3], depth [n], state [n] | None, counts [n,2] | None)."""
    r, keep = make_rays(*(rays if rays is not None else (None, None)))
    n = r.n_rays if rays is not None else cams.n_pixels()
    if out is None:
        out = {"rgb": torch.empty(n, 3, device="cuda"), "depth": torch.empty(n, device="cuda"),
               "state": torch.empty(n, device="cuda") if state else None,
               "counts": torch.empty(n, 2, device="cuda", dtype=torch.int32) if counts else None}
    cs = cams.struct()
    _check(_lib.plx_render_forward(grid.handle, C.byref(cs), C.byref(r), C.byref(opts),
                                   _ptr(out["rgb"]), _ptr(out["depth"]), _ptr(out.get("state")),
                                   _ptr(out.get("counts")), _stream(stream)))
    return out


@_ranged
def render_backward_grid(grid: Grid, cams: CameraSet, opts, rgb_target, depth_target, rgb,
                         depth, rays=None, grad=None, loss=None, stream=None):
    """plx_render_backward_grid. Adds into ``grad`` [n_alloc, 32] (allocated
    zeroed when None; ``grad=False``: loss only, returned grad None); returns
    (grad, loss [2] float64 = (L, M))."""
    r, keep = make_rays(*(rays if rays is not None else (None, None)))
    if grad is False:
        grad = None
    elif grad is None:
        grad = torch.zeros(grid.n_alloc, GRAD_STRIDE, device="cuda")
    if loss is None:
        loss = torch.empty(2, device="cuda", dtype=torch.float64)
    cs = cams.struct()
    _check(_lib.plx_render_backward_grid(grid.handle, C.byref(cs), C.byref(r), C.byref(opts),
                                         _ptr(rgb_target), _ptr(depth_target), _ptr(rgb),
                                         _ptr(depth), _ptr(grad), _ptr(loss), _stream(stream)))
    return grad, loss


@_ranged
def render_backward_pose(grid: Grid, cams: CameraSet, cam: int, opts, rgb_target, depth_target,
                         rays=None, out=None, stream=None):
    """plx_render_backward_pose for camera ``cam``; ``rays`` = pixel list or None.
    Returns (JtWJ [6,6], JtWr [6], loss [2]) float64 device tensors."""
    r, keep = make_rays(None, rays)
    if out is None:
        out = (torch.empty(6, 6, device="cuda", dtype=torch.float64),
               torch.empty(6, device="cuda", dtype=torch.float64),
               torch.empty(2, device="cuda", dtype=torch.float64))
    cs = cams.struct()
    _check(_lib.plx_render_backward_pose(grid.handle, C.byref(cs), int(cam), C.byref(r),
                                         C.byref(opts), _ptr(rgb_target), _ptr(depth_target),
                                         _ptr(out[0]), _ptr(out[1]), _ptr(out[2]),
                                         _stream(stream)))
    return out


@_ranged
def pose_step(JtWJ, JtWr, pose, damping=0.0, xi_out=None, status=None, stream=None):
    """plx_pose_step: pose (device float64 [12] view) <- exp(xi^) pose."""
    _check(_lib.plx_pose_step(_ptr(JtWJ), _ptr(JtWr), float(damping), _ptr(pose), _ptr(xi_out),
                              _ptr(status), _stream(stream)))


def lm_state():
    """Zeroed state for plx_pose_step_lm."""
    return torch.zeros(64, device="cuda", dtype=torch.float64)


@_ranged
def pose_step_lm(JtWJ, JtWr, loss, state, pose, lambda_init=1e-3, factor=10.0, xi_out=None,
                 status=None, stream=None):
    """plx_pose_step_lm: Gauss-Newton with Marquardt damping, accept/reject on
    the loss; pose (device float64 [12] view) updated in place."""
    _check(_lib.plx_pose_step_lm(_ptr(JtWJ), _ptr(JtWr), _ptr(loss), _ptr(state),
                                 float(lambda_init), float(factor), _ptr(pose), _ptr(xi_out),
                                 _ptr(status), _stream(stream)))


@_ranged
def render_batch(grid: Grid, cams: CameraSet, work, opts, rgb_target, depth_target, grad=None,
                 map_loss=None, out=None, stream=None):
    """plx_render_batch. ``work`` = [(cam, WORK_MAP | WORK_TRACK), ...]; targets
    hold every pixel of every item in that order. Returns (grad [n_alloc, 32] or
    None, map_loss [2] or None, JtWJ [n_track, 6, 6], JtWr [n_track, 6],
    track_loss [n_track, 2])."""
    work = list(work)
    arr = (Work * len(work))()
    for i, (c, m) in enumerate(work):
        arr[i].cam, arr[i].mode = int(c), int(m)
    n_track = sum(1 for _, m in work if m == WORK_TRACK)
    n_map = len(work) - n_track
    if grad is None and n_map:
        grad = torch.zeros(grid.n_alloc, GRAD_STRIDE, device="cuda")
    if map_loss is None and n_map:
        map_loss = torch.empty(2, device="cuda", dtype=torch.float64)
    if out is None:
        k = max(n_track, 1)
        out = (torch.empty(k, 6, 6, device="cuda", dtype=torch.float64),
               torch.empty(k, 6, device="cuda", dtype=torch.float64),
               torch.empty(k, 2, device="cuda", dtype=torch.float64))
    cs = cams.struct()
    _check(_lib.plx_render_batch(grid.handle, C.byref(cs), arr, len(work), C.byref(opts),
                                 _ptr(rgb_target), _ptr(depth_target), _ptr(grad),
                                 _ptr(map_loss), _ptr(out[0]), _ptr(out[1]), _ptr(out[2]),
                                 _stream(stream)))
    return grad, map_loss, out[0][:n_track], out[1][:n_track], out[2][:n_track]


@_ranged
def grid_rmsprop(grid: Grid, grad, state, lr, alpha=0.99, eps=1e-8, zero_grad=True, stream=None,
                 lr_density=None):
    """plx_grid_rmsprop: one RMSProp step on every stored grid value, in place
    (``lr`` for the SH values, ``lr_density`` for the density; the same if
    not given)."""
    lr_d = lr if lr_density is None else lr_density
    grid._autograd_values = None  # the stored values change
    _check(_lib.plx_grid_rmsprop(grid.handle, _ptr(grad), _ptr(state), float(lr_d), float(lr),
                                 float(alpha), float(eps), int(bool(zero_grad)), _stream(stream)))


@_ranged
def grid_grow(res, lo, hi, links: torch.Tensor, n_alloc: int, cams: CameraSet, depth, band,
              depth_is_z=True, n_new=None, stream=None):
    """Grow a link array from observed depth (``plx_grid_grow``): ``links`` (a
    CUDA int32 tensor [R_z, R_y, R_x]) is updated in place; returns the device
    int64 count of vertices added (-1 if the numbering would overflow int32).
    Asynchronous; read the count to synchronise."""
    if links.dtype != torch.int32 or not links.is_cuda or not links.is_contiguous():
        raise ValueError("links must be a contiguous CUDA int32 tensor")
    d = GridDesc()
    d.res[:] = [int(v) for v in res]
    d.lo[:] = [float(v) for v in lo]
    d.hi[:] = [float(v) for v in hi]
    d.n_alloc = int(n_alloc)
    if n_new is None:
        n_new = torch.empty(1, dtype=torch.int64, device="cuda")
    cs = cams.struct()
    _check(_lib.plx_grid_grow(C.byref(d), _ptr(links), C.byref(cs), _ptr(depth.contiguous()),
                              int(bool(depth_is_z)), float(band), _ptr(n_new), _stream(stream)))
    return n_new


def adam_state():
    """Zeroed Adam tracking state (m, v, t, last xi) for plx_track_adam_step."""
    return torch.zeros(20, device="cuda", dtype=torch.float64)


@_ranged
def track_adam_step(grid: Grid, cams: CameraSet, cam: int, opts, n_rays, seed, rgb_target,
                    depth_target, state, lr, beta1=0.9, beta2=0.999, eps=1e-8, out=None,
                    stream=None):
    """plx_track_adam_step: one Adam iteration on random rays of camera ``cam``."""
    if out is None:
        out = (torch.empty(6, 6, device="cuda", dtype=torch.float64),
               torch.empty(6, device="cuda", dtype=torch.float64),
               torch.empty(2, device="cuda", dtype=torch.float64))
    cs = cams.struct()
    _check(_lib.plx_track_adam_step(grid.handle, C.byref(cs), int(cam), C.byref(opts),
                                    int(n_rays), C.c_uint64(seed), _ptr(rgb_target),
                                    _ptr(depth_target), _ptr(state), float(lr), float(beta1),
                                    float(beta2), float(eps), _ptr(out[0]), _ptr(out[1]),
                                    _ptr(out[2]), _stream(stream)))
    return out


PROBE_RED, PROBE_GATHER, PROBE_STREAM, PROBE_RED_ROWS, PROBE_ISSUE = 0, 1, 2, 3, 4


def probe(kind, buf, group=1, ops=64, blocks=None, stream=None):
    """plx_probe: one launch of a ceiling kernel over ``buf`` (float32
    [n_rows, 32] on the device). ``blocks`` defaults to 8 per SM."""
    if blocks is None:
        blocks = 8 * torch.cuda.get_device_properties(buf.device).multi_processor_count
    _check(_lib.plx_probe(int(kind), _ptr(buf), int(buf.shape[0]), int(group), int(ops),
                          int(blocks), _stream(stream)))
