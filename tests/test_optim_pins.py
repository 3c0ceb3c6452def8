"""Pins of the oracle's optimisers and random-ray generator (Sec. 5.4):
RMSProp and Adam against torch.optim on the CPU, SplitMix64 against its
published value, and the oracle's Adam tracker reducing the loss."""
import os

import numpy as np
import pytest
import torch

import oracle
from paper_2307_03404_b300 import scenes

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def test_rmsprop_matches_torch():
    rng = np.random.default_rng(0)
    x0 = rng.standard_normal(50)
    p = torch.nn.Parameter(torch.tensor(x0))
    opt = torch.optim.RMSprop([p], lr=0.01, alpha=0.95, eps=1e-6)
    x, v = x0.copy(), np.zeros(50)
    for _ in range(5):
        g = rng.standard_normal(50)
        p.grad = torch.tensor(g)
        opt.step()
        x, v = oracle.rmsprop(x, g, v, 0.01, 0.95, 1e-6)
    np.testing.assert_allclose(x, p.detach().numpy(), rtol=1e-13)


def test_adam_matches_torch():
    rng = np.random.default_rng(1)
    x0 = rng.standard_normal(6)
    p = torch.nn.Parameter(torch.tensor(x0))
    opt = torch.optim.Adam([p], lr=0.003, betas=(0.8, 0.99), eps=1e-7)
    x, m, v = x0.copy(), np.zeros(6), np.zeros(6)
    for t in range(1, 7):
        g = rng.standard_normal(6)
        p.grad = torch.tensor(g)
        opt.step()
        step, m, v = oracle.adam(g, m, v, t, 0.003, 0.8, 0.99, 1e-7)
        x = x + step
    np.testing.assert_allclose(x, p.detach().numpy(), rtol=1e-12)


def test_splitmix64_published_value():
    for line in open(os.path.join(GOLDEN, "splitmix64.txt")):
        if line.startswith("#") or not line.strip():
            continue
        seed, k, val = line.split()
        assert oracle.splitmix64(int(seed), int(k)) == int(val, 16)


def test_random_pixels_are_in_range_and_spread():
    px = oracle.random_pixels(11, 3, 4000, 3072)
    assert px.min() >= 0 and px.max() < 3072
    counts = np.bincount(px, minlength=3072)
    assert counts.max() <= 8 and (counts > 0).mean() > 0.6


def test_adam_tracker_lowers_the_loss():
    g, cam, _ = scenes.sphere_scene()
    opts = dict(step=0.5 * g.h[0], lambda_d=1.0, depth_is_z=False)
    ref = oracle.render(g, [cam], opts)
    T0 = scenes.perturb_pose(cam.T_wc, 0.03, 2.0, np.random.default_rng(5))
    T, losses = oracle.adam_track(g, cam.with_pose(T0), opts, ref.rgb, ref.depth, 512, 7, 40,
                                  lr=3e-3)
    assert np.mean(losses[-5:]) < 0.25 * np.mean(losses[:5])
