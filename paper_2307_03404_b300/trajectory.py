"""Trajectory error metrics of Sec. 6.1 (tracking accuracy): the absolute
trajectory error (ATE) and the relative pose error in translation and rotation
(RPE_t, RPE_r) as defined by Sturm et al. (2012), RPE over 1 m of travelled
path. Host-side numpy: these evaluate a tracked sequence, they are not on the
GPU path.

Poses are camera-to-world [3, 4] (or [4, 4]) matrices in the map frame. The
tracked sequence starts from the true first pose in the frame the map was
built in, so no alignment is applied.
"""
from __future__ import annotations

import numpy as np


def _h(P):
    """[N, 4, 4] homogeneous matrices from [N, 3, 4] or [N, 4, 4]."""
    P = np.asarray(P, np.float64)
    if P.shape[-2:] == (4, 4):
        return P
    out = np.zeros(P.shape[:-2] + (4, 4))
    out[..., :3, :] = P
    out[..., 3, 3] = 1.0
    return out


def _inv(T):
    R, t = T[..., :3, :3], T[..., :3, 3]
    out = np.zeros_like(T)
    Rt = np.swapaxes(R, -1, -2)
    out[..., :3, :3] = Rt
    out[..., :3, 3] = -np.einsum("...ij,...j->...i", Rt, t)
    out[..., 3, 3] = 1.0
    return out


def rotation_angle_deg(R):
    """Angle of a rotation matrix, in degrees (from its trace, clipped)."""
    c = (np.trace(R, axis1=-2, axis2=-1) - 1.0) / 2.0
    return np.degrees(np.arccos(np.clip(c, -1.0, 1.0)))


def ate(est, gt):
    """RMSE of the camera-centre differences over all frames (metres)."""
    e, g = _h(est), _h(gt)
    d = e[:, :3, 3] - g[:, :3, 3]
    return float(np.sqrt(np.mean(np.sum(d * d, axis=1))))


def path_pairs(gt, delta=1.0):
    """Frame pairs (i, j) a travelled distance `delta` apart along the true
    path: starting at frame 0, j is the first frame at which the path length
    since i reaches `delta`; the next pair starts at j."""
    g = _h(gt)
    steps = np.linalg.norm(np.diff(g[:, :3, 3], axis=0), axis=1)
    pairs, i, acc = [], 0, 0.0
    for k, s in enumerate(steps, start=1):
        acc += s
        if acc >= delta:
            pairs.append((i, k))
            i, acc = k, 0.0
    return pairs


def rpe(est, gt, delta=1.0):
    """(RPE_t in metres, RPE_r in degrees): RMSE over the `path_pairs` of the
    error of the relative motion, E = (Q_i^-1 Q_j)^-1 (P_i^-1 P_j), Q true and
    P estimated. (nan, nan) when the path is shorter than `delta`."""
    e, g = _h(est), _h(gt)
    pairs = path_pairs(gt, delta)
    if not pairs:
        return float("nan"), float("nan")
    i, j = np.array(pairs).T
    rel_g = _inv(g[i]) @ g[j]
    rel_e = _inv(e[i]) @ e[j]
    E = _inv(rel_g) @ rel_e
    t = np.linalg.norm(E[:, :3, 3], axis=1)
    r = rotation_angle_deg(E[:, :3, :3])
    return float(np.sqrt(np.mean(t * t))), float(np.sqrt(np.mean(r * r)))


def pose_error(est, gt):
    """(camera-centre distance in cm, rotation angle in degrees) between two
    camera-to-world poses."""
    e, g = _h(est), _h(gt)
    d = 100.0 * float(np.linalg.norm(e[:3, 3] - g[:3, 3]))
    return d, float(rotation_angle_deg(e[:3, :3] @ g[:3, :3].T))
