"""The allocation-free pose entry point against the regular one and the oracle.

``plx_render_backward_pose_noalloc`` is for callers that cannot allocate
device memory while they run (a real-time tracking loop, or an application
whose device memory belongs to another allocator). It takes the grid as plain
arrays in the record layout ``include/plx.h`` documents and keeps its scratch
in a static device array of the library. Here the records are packed with
torch exactly as the header describes, for every storage mode, and the
entry's H, b and loss are compared with ``plx_render_backward_pose`` on a grid
handle of the same storage and with the FP64 oracle on the same (rounded)
values, on two calls in a row, in dense and list mode (with out-of-range
pixels, which the entry skips and leaves out of M) and with the SH
view-direction term, and the call's error word read back with
``plx_noalloc_error``. Free device memory and the torch allocator's reserved
bytes must not change across the calls. This file is collected last so that
a run stopping at the first failure has run every other test; it also passes
alone in a fresh process.
"""
import ctypes as C

import numpy as np
import pytest
import torch

import oracle
from paper_2307_03404_b300 import plx, scenes

pytestmark = pytest.mark.gpu

STORAGES = ["f32", "bf16", "f16", "f32_bf16"]


def _norm_err(x, ref):
    return float(np.abs(x - ref).max() / max(np.abs(ref).max(), 1e-300))


def pack_records(density, sh, storage):
    """Caller-side records in the layout of include/plx.h: PLX_STORE_F32 =
    32 floats (slot 0 density, 1..27 SH, 28..31 ignored); BF16 / F16 = 32
    16-bit values in the same slots; F32_BF16 = 64 bytes, the density as a
    float in bytes 0..3 and the 27 SH as bfloat16 from byte 4."""
    n = density.shape[0]
    d = torch.from_numpy(np.ascontiguousarray(density, np.float32)).cuda()
    s = torch.from_numpy(np.ascontiguousarray(sh, np.float32)).reshape(n, 27).cuda()
    if storage == "f32":
        return torch.cat([d[:, None], s, torch.zeros(n, 4, device="cuda")], 1).contiguous()
    if storage in ("bf16", "f16"):
        dt = torch.bfloat16 if storage == "bf16" else torch.float16
        v = torch.cat([d[:, None], s, torch.zeros(n, 4, device="cuda")], 1).to(dt)
        return v.contiguous()
    rec = torch.zeros(n, 32, dtype=torch.bfloat16, device="cuda")
    rec[:, 2:29] = s.to(torch.bfloat16)
    rec.view(torch.int32)[:, 0] = d.view(torch.int32)
    return rec.contiguous()


def rounded(g, storage):
    """The grid with its values rounded as the storage rounds them (what the
    kernels see), for the oracle."""
    import copy

    if storage == "f32":
        return g
    r = copy.copy(g)
    dt = torch.float16 if storage == "f16" else torch.bfloat16
    sh = torch.from_numpy(np.asarray(g.sh, np.float32)).to(dt).float().numpy()
    den = np.asarray(g.density, np.float32)
    if storage != "f32_bf16":
        den = torch.from_numpy(den).to(dt).float().numpy()
    r.density, r.sh = den, sh
    return r


def noalloc(desc, links, records, cams, rays, o, rgb_t, depth_t):
    H = torch.full((6, 6), np.nan, dtype=torch.float64, device="cuda")
    b = torch.full((6,), np.nan, dtype=torch.float64, device="cuda")
    loss = torch.full((2,), np.nan, dtype=torch.float64, device="cuda")
    cs = cams.struct()
    stream = C.c_void_p(torch.cuda.current_stream().cuda_stream)
    st = plx._lib.plx_render_backward_pose_noalloc(
        C.byref(desc), C.c_void_p(links.data_ptr()), C.c_void_p(records.data_ptr()),
        C.byref(cs), 0, C.byref(rays), C.byref(o), C.c_void_p(rgb_t.data_ptr()),
        C.c_void_p(depth_t.data_ptr()), C.c_void_p(H.data_ptr()), C.c_void_p(b.data_ptr()),
        C.c_void_p(loss.data_ptr()), stream)
    assert st == 0, plx._lib.plx_last_error()
    torch.cuda.synchronize()
    return H.cpu().numpy(), b.cpu().numpy(), loss.cpu().numpy()


@pytest.fixture(scope="module")
def scene():
    g, cam, _ = scenes.sphere_scene()
    opts = dict(step=0.5 * g.h[0], lambda_d=0.8, depth_is_z=False, bg=(0.1, 0.1, 0.2))
    tg = oracle.render(g, [cam], opts)
    T0 = scenes.perturb_pose(cam.T_wc, 0.03, 2.0, np.random.default_rng(9))
    return g, cam.with_pose(T0), opts, tg


@pytest.mark.parametrize("storage", STORAGES)
@pytest.mark.parametrize("mode", ["dense", "list", "view_dir"])
def test_noalloc_pose_matches_regular_entry_and_oracle_twice_in_a_row(scene, storage, mode):
    g, cam, opts, tg = scene
    if mode == "view_dir":
        opts = dict(opts, dir_term=True)
    cams = plx.CameraSet([cam])
    o = plx.opts_from_dict(opts)
    npx = cam.width * cam.height
    if mode == "list":
        # a pixel list with entries outside the frame: skipped, not in M
        pix = np.random.default_rng(4).permutation(npx)[:1500].astype(np.int32)
        pix[::97] = npx + 5
        pix[3] = -1
    else:
        pix = np.arange(npx, dtype=np.int32)
    good = (pix >= 0) & (pix < npx)
    valid = good & (tg.depth[np.clip(pix, 0, npx - 1)] > 0)   # rays that miss have depth 0
    rgb_t = torch.tensor(tg.rgb[np.clip(pix, 0, npx - 1)], dtype=torch.float32, device="cuda")
    depth_t = torch.tensor(tg.depth[np.clip(pix, 0, npx - 1)], dtype=torch.float32,
                           device="cuda")
    pix_d = torch.tensor(pix, device="cuda")

    grid = plx.Grid.from_scene(g, storage)
    H_ref, b_ref, l_ref = plx.render_backward_pose(
        grid, cams, 0, o, rgb_t, depth_t, rays=pix_d if mode == "list" else None)
    torch.cuda.synchronize()
    H_ref, b_ref, l_ref = H_ref.cpu().numpy(), b_ref.cpu().numpy(), l_ref.cpu().numpy()
    if mode == "list":
        with pytest.raises(plx.PlxError):
            grid.check()  # the regular entry reports the bad entries through its grid
    grid.close()
    rp = oracle.pose_jacobian(rounded(g, storage), [cam], opts, tg.rgb[pix[good]],
                              tg.depth[pix[good]],
                              rays=(np.zeros(int(good.sum()), np.int32), pix[good]))

    links = torch.from_numpy(np.ascontiguousarray(g.links)).cuda()
    records = pack_records(g.density, g.sh, storage)
    desc = plx.GridDesc()
    desc.res[:] = list(g.res)
    desc.lo[:] = [float(v) for v in g.lo]
    desc.hi[:] = [float(v) for v in g.hi]
    desc.n_alloc = g.n_alloc
    desc.storage = plx.STORAGE[storage]
    rays = plx.Rays()
    if mode == "list":
        rays.n_rays = pix.shape[0]
        rays.pixel = C.c_void_p(pix_d.data_ptr())
    # the first call on a device finds the scratch array's address; from then
    # on a call touches no allocator at all
    noalloc(desc, links, records, cams, rays, o, rgb_t, depth_t)
    err = torch.empty(1, dtype=torch.int32, device="cuda")
    stream = C.c_void_p(torch.cuda.current_stream().cuda_stream)
    free0, reserved0 = torch.cuda.mem_get_info()[0], torch.cuda.memory_reserved()
    for call in range(2):
        H, b, loss = noalloc(desc, links, records, cams, rays, o, rgb_t, depth_t)
        assert loss[1] == l_ref[1] == rp.M == int(valid.sum()), call
        assert abs(loss[0] - l_ref[0]) <= 1e-5 * l_ref[0], call
        assert _norm_err(H, H_ref) <= 1e-4 and _norm_err(b, b_ref) <= 1e-4, call
        assert abs(loss[0] - rp.loss) <= 1e-5 * rp.loss, call
        assert _norm_err(H, rp.H) <= 1e-4 and _norm_err(b, rp.b) <= 1e-4, call
        # the call's error word: bit 0 for the out-of-range list entries
        err.fill_(-1)
        assert plx._lib.plx_noalloc_error(C.c_void_p(err.data_ptr()), stream) == 0
        torch.cuda.synchronize()
        assert int(err.item()) == (1 if mode == "list" else 0), call
    assert torch.cuda.mem_get_info()[0] == free0
    assert torch.cuda.memory_reserved() == reserved0
