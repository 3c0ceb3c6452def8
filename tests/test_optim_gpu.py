"""RMSProp grid step and Adam tracking step on the GPU against the oracle."""
import numpy as np
import pytest
import torch

import oracle
from gpu_helpers import dev
from paper_2307_03404_b300 import plx, scenes

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("storage", ["f32", "bf16", "f16", "f32_bf16"])
def test_rmsprop_step_matches_oracle(storage):
    g = scenes.tiny_grid(8, seed=3, alloc_frac=0.5)
    grid = plx.Grid.from_scene(g, storage)
    d0, s0 = grid.download()
    x0 = torch.cat([d0[:, None], s0], 1).cpu().numpy().astype(np.float64)
    rng = np.random.default_rng(4)
    n = g.n_alloc
    gr = np.zeros((n, 32), np.float32)
    gr[:, :28] = rng.standard_normal((n, 28)).astype(np.float32)
    st = np.zeros((n, 32), np.float32)
    st[:, :28] = rng.uniform(0, 2, (n, 28)).astype(np.float32)
    grad, state = dev(gr), dev(st)
    plx.grid_rmsprop(grid, grad, state, lr=0.01, lr_density=0.5, alpha=0.9, eps=1e-6,
                     zero_grad=True)
    d1, s1 = grid.download()
    torch.cuda.synchronize()
    x1 = torch.cat([d1[:, None], s1], 1).cpu().numpy()
    lr = np.full(28, 0.01)
    lr[0] = 0.5  # density
    xr, vr = oracle.rmsprop(x0, gr[:, :28], st[:, :28], lr, 0.9, 1e-6)
    np.testing.assert_allclose(state.cpu().numpy()[:, :28], vr, rtol=1e-6)
    assert np.all(grad.cpu().numpy() == 0)
    if storage == "f32":
        np.testing.assert_allclose(x1, xr, rtol=1e-6, atol=1e-7)
    else:
        # stored 16-bit: the update rounded to nearest, so within one unit in the last place
        ulp = {"bf16": 2.0 ** -7, "f16": 2.0 ** -10, "f32_bf16": 2.0 ** -7}[storage]
        tol = np.abs(xr) * ulp + 1e-6
        if storage == "f32_bf16":
            np.testing.assert_allclose(x1[:, 0], xr[:, 0], rtol=1e-6, atol=1e-7)
            assert np.all(np.abs(x1[:, 1:] - xr[:, 1:]) <= tol[:, 1:])
        else:
            assert np.all(np.abs(x1 - xr) <= tol)
    grid.close()


def test_adam_tracking_matches_oracle_and_captures_in_a_graph():
    g, cam, _ = scenes.sphere_scene()
    opts = dict(step=0.5 * g.h[0], lambda_d=1.0, depth_is_z=False)
    ref = oracle.render(g, [cam], opts)
    T0 = scenes.perturb_pose(cam.T_wc, 0.03, 2.0, np.random.default_rng(5))
    n_rays, seed, iters, lr = 512, 7, 6, 3e-3
    T_ref, loss_ref = oracle.adam_track(g, cam.with_pose(T0), opts, ref.rgb, ref.depth, n_rays,
                                        seed, iters, lr)
    grid = plx.Grid.from_scene(g, "f32")
    cams = plx.CameraSet([cam.with_pose(T0)])
    o = plx.opts_from_dict(opts)
    rgb_t, depth_t = dev(ref.rgb), dev(ref.depth)
    state = plx.adam_state()
    losses = []
    for _ in range(iters):
        H, b, loss = plx.track_adam_step(grid, cams, 0, o, n_rays, seed, rgb_t, depth_t, state, lr)
        losses.append(loss[0].item())
    T = cams.poses[0].cpu().numpy().reshape(3, 4)
    np.testing.assert_allclose(losses, loss_ref, rtol=1e-4)
    assert np.abs(T - T_ref).max() <= 1e-3 * lr * iters
    assert state[12].item() == iters
    # the same loop captured in one CUDA graph from the same start
    cams.poses.copy_(dev(T0.reshape(1, 12), torch.float64))
    state.zero_()
    out = (torch.empty(6, 6, device="cuda", dtype=torch.float64),
           torch.empty(6, device="cuda", dtype=torch.float64),
           torch.empty(2, device="cuda", dtype=torch.float64))
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph, stream=s):
        for _ in range(iters):
            plx.track_adam_step(grid, cams, 0, o, n_rays, seed, rgb_t, depth_t, state, lr, out=out)
    graph.replay()
    torch.cuda.synchronize()
    T2 = cams.poses[0].cpu().numpy().reshape(3, 4)
    np.testing.assert_array_equal(T2, T)
    grid.close()
