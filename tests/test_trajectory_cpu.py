"""The trajectory metrics (ATE, RPE over 1 m of path) on trajectories whose
errors are known in closed form."""
import numpy as np

from paper_2307_03404_b300 import trajectory


def straight_line(n=41, step=0.1):
    P = np.zeros((n, 3, 4))
    P[:, :, :3] = np.eye(3)
    P[:, 0, 3] = step * np.arange(n)
    return P


def rot_z(a):
    c, s = np.cos(a), np.sin(a)
    return np.array([[c, -s, 0.0], [s, c, 0.0], [0.0, 0.0, 1.0]])


def test_identical_trajectories_have_no_error():
    g = straight_line()
    assert trajectory.ate(g, g) == 0.0
    assert trajectory.rpe(g, g) == (0.0, 0.0)


def test_path_pairs_every_metre():
    g = straight_line(41, 0.1)              # 4 m in 0.1 m steps
    pairs = trajectory.path_pairs(g, 1.0)
    # float sums of 0.1 reach 1.0 at the 10th or 11th step; pairs chain end to start
    assert len(pairs) in (3, 4)
    assert pairs[0][0] == 0
    assert all(a[1] == b[0] for a, b in zip(pairs, pairs[1:]))
    for i, j in pairs:
        assert 0.999 <= 0.1 * (j - i) <= 1.101


def test_constant_offset_is_all_ate_and_no_rpe():
    g = straight_line()
    e = g.copy()
    e[:, :, 3] += np.array([0.03, -0.04, 0.0])
    assert abs(trajectory.ate(e, g) - 0.05) < 1e-12
    t, r = trajectory.rpe(e, g)
    assert t < 1e-12 and r < 1e-9


def test_scale_drift_gives_known_relative_error():
    g = straight_line(41, 0.1)
    e = g.copy()
    e[:, 0, 3] *= 1.1                        # 10% too far per metre
    t, r = trajectory.rpe(e, g)
    steps = [j - i for i, j in trajectory.path_pairs(g)]
    want = np.sqrt(np.mean([(0.01 * k) ** 2 for k in steps]))  # 0.1 x (0.1 m x k)
    assert abs(t - want) < 1e-12 and r < 1e-9
    x = 0.1 * np.arange(41)
    assert abs(trajectory.ate(e, g) - np.sqrt(np.mean((0.1 * x) ** 2))) < 1e-12


def test_rotation_drift_gives_known_relative_angle():
    g = straight_line(41, 0.1)
    e = g.copy()
    w = np.radians(0.5)                      # 0.5 degree extra yaw per frame
    for k in range(41):
        e[k, :, :3] = rot_z(w * k)
    t, r = trajectory.rpe(e, g)
    steps = [j - i for i, j in trajectory.path_pairs(g)]
    assert abs(r - np.sqrt(np.mean([(0.5 * k) ** 2 for k in steps]))) < 1e-9
    # the positions are right, but the relative translation is read in the
    # rotated frame: |R_i^T d - d| for a 1 m step d along x
    assert t > 0.0
    assert trajectory.ate(e, g) < 1e-15
    assert abs(trajectory.rotation_angle_deg(rot_z(np.radians(37.0))) - 37.0) < 1e-9


def test_pose_error_closed_form():
    """A camera moved 3 cm and turned 2 degrees about any axis: (3, 2)."""
    from scipy.spatial.transform import Rotation

    from paper_2307_03404_b300.trajectory import pose_error

    rng = np.random.default_rng(2)
    T = np.zeros((3, 4))
    T[:, :3] = Rotation.random(random_state=3).as_matrix()
    T[:, 3] = rng.standard_normal(3)
    u = rng.standard_normal(3)
    u /= np.linalg.norm(u)
    E = T.copy()
    E[:, :3] = Rotation.from_rotvec(np.deg2rad(2.0) * u[::-1]).as_matrix() @ T[:, :3]
    E[:, 3] += 0.03 * u
    d_cm, d_deg = pose_error(E, T)
    assert abs(d_cm - 3.0) < 1e-12 and abs(d_deg - 2.0) < 1e-9
