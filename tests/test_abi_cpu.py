"""Host-side checks of the C ABI that need no GPU.

The CUDA library is linked against a static CUDA runtime, so it loads on a
machine without a GPU; these tests only make calls that fail argument
validation before any CUDA call.
"""
import ctypes as C
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "plx.h")
LIB = os.path.join(ROOT, "paper_2307_03404_b300", "libplx.so")


@pytest.fixture(scope="module")
def lib():
    from paper_2307_03404_b300 import build

    build.build()
    return C.CDLL(LIB)


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(plx_[a-z_]+)\s*\(", text)))


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ["plx_grid_create", "plx_render_forward", "plx_render_backward_grid",
                     "plx_render_backward_pose", "plx_pose_step", "plx_grid_destroy",
                     "plx_grid_upload", "plx_grid_download", "plx_last_error"]:
        assert required in names


def test_library_exports_every_declared_symbol(lib):
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, missing
    out = subprocess.run(["nm", "-D", "--defined-only", LIB], capture_output=True, text=True).stdout
    exported = set(re.findall(r"\bT (plx_\w+)", out))
    assert set(declared_functions()) <= exported


def test_binding_uses_the_declared_names():
    from paper_2307_03404_b300 import plx

    assert set(plx.SYMBOLS) == set(declared_functions())
    assert plx.version().startswith("plx")


def test_ctypes_structs_match_the_c_layout(tmp_path):
    """Compile a probe against plx.h with gcc and compare sizes and offsets."""
    from paper_2307_03404_b300 import plx

    src = tmp_path / "probe.c"
    src.write_text(r"""
#include <stddef.h>
#include <stdio.h>
#include "plx.h"
#define P(T, F) printf(#T "." #F " %zu\n", offsetof(T, F))
#define S(T) printf(#T " %zu\n", sizeof(T))
int main(void) {
  S(plx_grid_desc); P(plx_grid_desc, lo); P(plx_grid_desc, hi); P(plx_grid_desc, n_alloc);
  P(plx_grid_desc, storage);
  S(plx_intrinsics); P(plx_intrinsics, width);
  S(plx_cameras); P(plx_cameras, intr); P(plx_cameras, poses);
  S(plx_rays); P(plx_rays, cam_id); P(plx_rays, pixel);
  S(plx_render_opts); P(plx_render_opts, bg); P(plx_render_opts, lambda_d);
  P(plx_render_opts, max_samples); P(plx_render_opts, depth_is_z);
  P(plx_render_opts, sample_cache); P(plx_render_opts, sample_cap);
  P(plx_render_opts, sample_rays); P(plx_render_opts, ray_range);
  return 0;
}
""")
    exe = tmp_path / "probe"
    subprocess.check_call(["gcc", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)])
    got = dict(l.split() for l in subprocess.check_output([str(exe)], text=True).splitlines())
    m = {"plx_grid_desc": plx.GridDesc, "plx_intrinsics": plx.Intrinsics,
         "plx_cameras": plx.Cameras, "plx_rays": plx.Rays, "plx_render_opts": plx.RenderOpts}
    for key, val in got.items():
        if "." in key:
            t, f = key.split(".")
            assert getattr(m[t], f).offset == int(val), key
        else:
            assert C.sizeof(m[key]) == int(val), key


def test_argument_errors_are_reported_without_touching_the_gpu(lib):
    from paper_2307_03404_b300 import plx

    lib = plx._lib
    h = C.c_void_p()
    assert lib.plx_grid_create(None, None, None, None, None, C.byref(h)) == 1
    assert b"null" in lib.plx_last_error()
    d = plx.GridDesc()
    d.res[:] = [1, 4, 4]
    d.hi[:] = [1, 1, 1]
    assert lib.plx_grid_create(C.byref(d), None, None, None, None, C.byref(h)) == 1
    assert b"res[0]" in lib.plx_last_error()
    d.res[:] = [4, 4, 4]
    d.storage = 9
    assert lib.plx_grid_create(C.byref(d), None, None, None, None, C.byref(h)) == 1
    assert b"storage" in lib.plx_last_error()
    assert lib.plx_pose_step(None, None, 0.0, None, None, None, None) == 1
    x = (C.c_double * 40)()
    assert lib.plx_pose_step(x, x, -1.0, x, None, None, None) == 1
    assert b"damping" in lib.plx_last_error()
    assert lib.plx_render_forward(None, None, None, None, None, None, None, None, None) == 1
    assert lib.plx_grid_destroy(None) == 0


def test_sample_cache_size(lib):
    """float4 [K][n] + int32 [K][n] + int32 [n]; -1 for a negative argument."""
    from paper_2307_03404_b300 import plx

    assert plx.sample_cache_bytes(0, 5) == 0
    assert plx.sample_cache_bytes(7, 0) == 28
    assert plx.sample_cache_bytes(2_457_600, 64) == 2_457_600 * (64 * 16 + 64 * 4 + 4)
    assert plx.sample_cache_bytes(-1, 4) == -1 and plx.sample_cache_bytes(4, -1) == -1
    o = plx.make_opts(0.1)
    assert o.sample_cache is None and o.sample_cap == 0


def test_sample_cache_binding_layout():
    """The binding's view of a cache matches the header's layout: counts start
    20 K n bytes in, and the options name the buffer, K and n (host buffer:
    only the arithmetic is checked here)."""
    import torch

    from paper_2307_03404_b300 import plx

    c = plx.SampleCache(10, 3, device="cpu")
    assert c.buf.numel() * 4 == plx.sample_cache_bytes(10, 3)
    cnt = c.counts()
    assert cnt.dtype == torch.int32 and cnt.numel() == 10
    assert cnt.data_ptr() - c.buf.data_ptr() == 20 * 3 * 10
    o = c.opts(plx.make_opts(0.1))
    assert o.sample_cache == c.buf.data_ptr() and o.sample_cap == 3 and o.sample_rays == 10
    off = plx.SampleCache(10, 0, device="cpu")
    assert off.opts(plx.make_opts(0.1)).sample_cache is None
    with pytest.raises(ValueError):
        off.counts()


def test_ray_range_binding_layout():
    """A compositing-range buffer is int32 [n][2], 8-byte aligned, and options
    naming it keep it alive together with a sample cache named before or
    after (host buffers: only the binding is checked here)."""
    import torch

    from paper_2307_03404_b300 import plx

    rr = plx.RayRange(10, device="cpu")
    assert rr.ranges().shape == (10, 2) and rr.ranges().dtype == torch.int32
    assert rr.buf.data_ptr() % 8 == 0
    c = plx.SampleCache(10, 3, device="cpu")
    for o in (c.opts(rr.opts(plx.make_opts(0.1))), rr.opts(c.opts(plx.make_opts(0.1)))):
        assert o.ray_range == rr.buf.data_ptr() and o.sample_cache == c.buf.data_ptr()
        assert o._range is rr and o._cache is c
    assert plx.make_opts(0.1).ray_range is None
    with pytest.raises(ValueError):
        plx.RayRange(-1, device="cpu")


def test_grid_grow_argument_errors(lib):
    from paper_2307_03404_b300 import plx

    lib = plx._lib
    x = (C.c_double * 16)()
    assert lib.plx_grid_grow(None, None, None, None, 1, 1.0, None, None) == 1
    assert b"null" in lib.plx_last_error()
    d = plx.GridDesc()
    d.res[:] = [4, 4, 4]
    d.hi[:] = [1, 1, 1]
    cams = plx.Cameras()
    cams.n_cams = 1
    assert lib.plx_grid_grow(C.byref(d), x, C.byref(cams), x, 1, -0.5, x, None) == 1
    assert b"band" in lib.plx_last_error()
    assert lib.plx_grid_grow(C.byref(d), x, C.byref(cams), x, 1, float("nan"), x, None) == 1
    cams.n_cams = 0
    assert lib.plx_grid_grow(C.byref(d), x, C.byref(cams), x, 1, 2.0, x, None) == 1
    assert b"n_cams" in lib.plx_last_error()
    d.n_alloc = -3
    assert lib.plx_grid_grow(C.byref(d), x, C.byref(cams), x, 1, 2.0, x, None) == 1
    assert b"n_alloc" in lib.plx_last_error()


def test_pose_step_lm_argument_errors(lib):
    from paper_2307_03404_b300 import plx

    lib = plx._lib
    x = (C.c_double * 64)()
    assert lib.plx_pose_step_lm(None, x, x, x, 1e-3, 10.0, x, None, None, None) == 1
    assert b"null" in lib.plx_last_error()
    assert lib.plx_pose_step_lm(x, x, x, x, -1.0, 10.0, x, None, None, None) == 1
    assert b"lambda_init" in lib.plx_last_error()
    assert lib.plx_pose_step_lm(x, x, x, x, 1e-3, 1.0, x, None, None, None) == 1
    assert lib.plx_pose_step_lm(x, x, x, x, 1e-3, float("inf"), x, None, None, None) == 1


def test_set_config_and_opts_flags_are_validated_on_the_host(lib):
    from paper_2307_03404_b300 import plx

    lib = plx._lib
    c = plx.LaunchConfig(3, 1, 2, 2, 1, 14)
    assert lib.plx_grid_set_config(None, C.byref(c), None) == 1
    o = plx.make_opts(0.1)
    o.pose_flags = 2
    assert lib.plx_render_forward(None, None, None, C.byref(o), None, None, None, None, None) == 1


def test_allocation_cap_reports_out_of_memory_before_allocating(lib):
    """Host-side fault injection: with PLX_ALLOC_CAP_BYTES below what a grid
    needs, plx_grid_create fails with PLX_ENOMEM before any device call (so
    this runs without a GPU)."""
    import subprocess
    import sys

    code = (
        "import ctypes as C\n"
        "from paper_2307_03404_b300 import plx\n"
        "d = plx.GridDesc(); d.res[:] = [64, 64, 64]; d.hi[:] = [1, 1, 1]; d.n_alloc = 1000\n"
        "x = (C.c_float * 16)(); h = C.c_void_p()\n"
        "st = plx._lib.plx_grid_create(C.byref(d), x, x, x, None, C.byref(h))\n"
        "print(st, plx._lib.plx_last_error().decode())\n")
    env = dict(os.environ, PLX_ALLOC_CAP_BYTES="100000")
    out = subprocess.run([sys.executable, "-c", code], env=env, capture_output=True, text=True,
                         cwd=ROOT, timeout=300)
    st, msg = out.stdout.strip().split(" ", 1)
    assert int(st) == 2 and "PLX_ALLOC_CAP_BYTES" in msg


def test_probe_argument_errors(lib):
    """plx_probe validates kind, buffer, sizes and group before any launch."""
    from paper_2307_03404_b300 import plx

    lib = plx._lib
    fake = C.c_void_p(0x1000)  # never dereferenced: every call below fails its checks
    assert lib.plx_probe(7, fake, 16, 1, 1, 1, None) == 1
    assert b"kind" in lib.plx_last_error()
    assert lib.plx_probe(0, None, 16, 1, 1, 1, None) == 1
    assert lib.plx_probe(0, C.c_void_p(0x1004), 16, 1, 1, 1, None) == 1
    assert b"aligned" in lib.plx_last_error()
    assert lib.plx_probe(0, fake, 0, 1, 1, 1, None) == 1
    assert b"n_rows" in lib.plx_last_error()
    assert lib.plx_probe(1, fake, 16, 33, 1, 1, None) == 1
    assert b"group" in lib.plx_last_error()
    assert lib.plx_probe(2, fake, 16, 1, 0, 1, None) == 1
    assert b"ops" in lib.plx_last_error()
    # the coalesced-row reductions ignore `group`
    assert lib.plx_probe(plx.PROBE_RED_ROWS, fake, 16, 99, 0, 1, None) == 1
    assert b"ops" in lib.plx_last_error()
    assert lib.plx_probe(plx.PROBE_ISSUE, fake, 16, 1, 2000, 1, None) == 1
    assert b"ops" in lib.plx_last_error()
    assert lib.plx_probe(5, fake, 16, 1, 1, 1, None) == 1
    assert b"kind" in lib.plx_last_error()


def test_noalloc_error_checks_its_argument(lib):
    """plx_noalloc_error rejects a null destination before touching a device."""
    from paper_2307_03404_b300 import plx

    assert plx._lib.plx_noalloc_error(None, None) == 1
    assert b"err_out" in plx._lib.plx_last_error()


def test_sample_cache_options_keep_the_cache_alive():
    """Options made by SampleCache.opts hold the cache: a temporary cache's
    device buffer is not freed (and reused) while the options live."""
    import gc
    import weakref

    from paper_2307_03404_b300 import plx

    cache = plx.SampleCache(4, 2, device="cpu")
    ref = weakref.ref(cache)
    o = cache.opts(plx.make_opts(0.1))
    del cache
    gc.collect()
    assert ref() is not None and o.sample_cap == 2
    del o
    gc.collect()
    assert ref() is None
