"""The autograd wrapper's gradient against the oracle's (which finite
differences of the oracle's forward pin) and against central differences of
its own GPU loss."""
import numpy as np
import pytest
import torch

import oracle
from paper_2307_03404_b300 import autograd, plx, scenes

pytestmark = pytest.mark.gpu


def test_mapping_loss_backward_matches_oracle():
    g, cam, gp = scenes.sphere_scene()
    opts_d = dict(step=0.5 * g.h[0], lambda_d=0.5, depth_is_z=False, bg=(0.1, 0.2, 0.3))
    tg = oracle.render(gp, [cam], opts_d)
    grid = plx.Grid.from_scene(g, "f32")
    cams = plx.CameraSet([cam])
    o = plx.opts_from_dict(opts_d)
    dens = torch.tensor(g.density, device="cuda", requires_grad=True)
    sh = torch.tensor(g.sh, device="cuda", requires_grad=True)
    rgb_t = torch.tensor(tg.rgb, dtype=torch.float32, device="cuda")
    depth_t = torch.tensor(tg.depth, dtype=torch.float32, device="cuda")
    loss, rgb, depth = autograd.mapping_loss(dens, sh, grid, cams, o, rgb_t, depth_t)
    (3.0 * loss).backward()
    ref = oracle.grad_grid(g, [cam], opts_d, tg.rgb, tg.depth)
    assert abs(loss.item() - ref.loss) <= 1e-5 * ref.loss
    gd = dens.grad.cpu().numpy()
    gs = sh.grad.cpu().numpy()
    assert np.abs(gd - 3 * ref.grad_density).max() <= 1e-4 * np.abs(3 * ref.grad_density).max()
    assert np.abs(gs - 3 * ref.grad_sh).max() <= 1e-4 * np.abs(3 * ref.grad_sh).max()
    # one optimiser step through autograd lowers the loss
    with torch.no_grad():
        dens -= 50.0 * dens.grad
        sh -= 50.0 * sh.grad
    loss2, _, _ = autograd.mapping_loss(dens, sh, grid, cams, o, rgb_t, depth_t)
    assert loss2.item() < loss.item()
    grid.close()


@pytest.mark.parametrize("part", ["sh", "density"])
def test_mapping_loss_gradient_matches_finite_differences(part):
    """Directional derivative of the GPU loss through autograd against a
    central difference of the same GPU loss. SH directions are smooth (sigmoid
    colour); density directions move only vertices of density 40, where the
    interpolated density stays positive wherever they have weight, so no
    sample crosses the ReLU kink."""
    g, cam, gp = scenes.sphere_scene()
    opts_d = dict(step=0.5 * g.h[0], lambda_d=0.5, depth_is_z=False, bg=(0.1, 0.2, 0.3))
    tg = oracle.render(gp, [cam], opts_d)
    grid = plx.Grid.from_scene(g, "f32")
    cams = plx.CameraSet([cam])
    o = plx.opts_from_dict(opts_d)
    rgb_t = torch.tensor(tg.rgb, dtype=torch.float32, device="cuda")
    depth_t = torch.tensor(tg.depth, dtype=torch.float32, device="cuda")
    d0 = torch.tensor(g.density, device="cuda")
    s0 = torch.tensor(g.sh, device="cuda")
    gen = torch.Generator(device="cuda").manual_seed(11)
    vd = torch.zeros_like(d0)
    vs = torch.zeros_like(s0)
    if part == "sh":
        vs = torch.randn(s0.shape, device="cuda", generator=gen)
        eps = 1e-2
    else:
        vd = torch.randn(d0.shape, device="cuda", generator=gen) * (d0 == 40.0)
        eps = 0.5
    dens = d0.clone().requires_grad_(True)
    sh = s0.clone().requires_grad_(True)
    loss, _, _ = autograd.mapping_loss(dens, sh, grid, cams, o, rgb_t, depth_t)
    loss.backward()
    dd = float((dens.grad * vd).sum() + (sh.grad * vs).sum())
    with torch.no_grad():
        lp, _, _ = autograd.mapping_loss(d0 + eps * vd, s0 + eps * vs, grid, cams, o, rgb_t,
                                         depth_t)
        lm, _, _ = autograd.mapping_loss(d0 - eps * vd, s0 - eps * vs, grid, cams, o, rgb_t,
                                         depth_t)
    fd = (lp.item() - lm.item()) / (2 * eps)
    assert abs(dd) > 0
    assert abs(fd - dd) <= 2e-3 * abs(dd), (fd, dd)
    grid.close()
