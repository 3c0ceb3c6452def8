"""Pins of the oracle's Levenberg-Marquardt pose step (Gauss-Newton with
Marquardt's damping; the step the tracking loop takes on the device)."""
import numpy as np

import oracle
from paper_2307_03404_b300 import scenes


def spd(rng, n=6):
    A = rng.standard_normal((n, n))
    return A @ A.T + 0.5 * np.eye(n)


def damped(H, lam):
    d = np.diag(H)
    return H + lam * np.diag(d + 1e-12 * d.max())


def test_first_call_is_the_damped_gauss_newton_step():
    rng = np.random.default_rng(1)
    H, b = spd(rng), rng.standard_normal(6)
    T = scenes.look_at((0.3, 0.2, -1.0), (0, 0, 0))
    st = np.zeros(64)
    T1, xi, status = oracle.pose_step_lm(H, b, 0.5, st, T, lambda_init=0.01)
    assert status == 0 and st[3] == 1 and st[2] == 1 and st[0] == 0.01
    np.testing.assert_allclose(xi, np.linalg.solve(damped(H, 0.01), -b), rtol=1e-12)
    np.testing.assert_allclose(T1, _compose(oracle.se3_exp(xi), T), atol=1e-14)
    # lambda 0: the plain GN step
    st = np.zeros(64)
    _, xi0, _ = oracle.pose_step_lm(H, b, 0.5, st, T, lambda_init=0.0)
    np.testing.assert_allclose(xi0, np.linalg.solve(H, -b), rtol=1e-11)


def _compose(E, T):
    out = np.zeros((3, 4))
    out[:, :3] = E[:, :3] @ T[:, :3]
    out[:, 3] = E[:, :3] @ T[:, 3] + E[:, 3]
    return out


def test_a_worse_loss_is_rejected_and_the_accepted_pose_restored():
    rng = np.random.default_rng(2)
    H, b = spd(rng), rng.standard_normal(6)
    H2, b2 = spd(rng), rng.standard_normal(6)
    T = scenes.look_at((0.3, 0.2, -1.0), (0, 0, 0))
    st = np.zeros(64)
    T1, _, _ = oracle.pose_step_lm(H, b, 1.0, st, T, lambda_init=0.1, factor=10.0)
    T2, xi2, status = oracle.pose_step_lm(H2, b2, 2.0, st, T1, lambda_init=0.1, factor=10.0)
    assert status == 2 and st[3] == 0 and st[0] == 1.0 and st[1] == 1.0
    # the step restarts from T with the accepted H, b and ten times the damping
    np.testing.assert_allclose(xi2, np.linalg.solve(damped(H, 1.0), -b), rtol=1e-12)
    np.testing.assert_allclose(T2, _compose(oracle.se3_exp(xi2), T), atol=1e-14)
    # a better loss is accepted at the new pose and the damping goes down
    T3, xi3, status = oracle.pose_step_lm(H2, b2, 0.5, st, T2, lambda_init=0.1, factor=10.0)
    assert status == 0 and st[0] == 0.1 and st[1] == 0.5
    np.testing.assert_allclose(xi3, np.linalg.solve(damped(H2, 0.1), -b2), rtol=1e-12)
    np.testing.assert_allclose(st[4:16], T2.reshape(12))


def test_heavy_damping_is_scaled_gradient_descent():
    rng = np.random.default_rng(3)
    H, b = spd(rng), rng.standard_normal(6)
    st = np.zeros(64)
    lam = 1e8
    _, xi, _ = oracle.pose_step_lm(H, b, 1.0, st, np.hstack([np.eye(3), np.zeros((3, 1))]),
                                   lambda_init=lam)
    gd = -b / (lam * np.diag(H))
    np.testing.assert_allclose(xi, gd, rtol=1e-6)


def test_loop_on_a_small_scene_lowers_the_loss_monotonically():
    g, cam, _ = scenes.sphere_scene()
    opts = dict(step=0.5 * g.h[0], lambda_d=1.0, depth_is_z=False)
    ref = oracle.render(g, [cam], opts)
    T = scenes.perturb_pose(cam.T_wc, 0.03, 2.0, np.random.default_rng(5))
    st = np.zeros(64)
    accepted = []
    for _ in range(12):
        pj = oracle.pose_jacobian(g, [cam.with_pose(T)], opts, ref.rgb, ref.depth)
        T, _, status = oracle.pose_step_lm(pj.H, pj.b, pj.loss, st, T)
        if status == 0:
            accepted.append(pj.loss)
    assert all(a >= c for a, c in zip(accepted, accepted[1:]))
    assert accepted[-1] < 1e-3 * accepted[0]
