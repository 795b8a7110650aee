"""Seeded candidate manipulator trajectories (inputs only).

Each trajectory is a camera-pose sequence of uneven length.  Positions follow
Catmull-Rom splines of the direction and of the radius through four control
points on a shell of radii [r_min, r_max] around one of the PoIs; orientations look at that PoI with a
small random tilt (a rotation of up to ``jitter_deg`` about a random axis).
Output: float32 poses (total, 7) and int32 CSR offsets (n_traj + 1).
"""

from __future__ import annotations

import math

import numpy as np

from .poses import look_at_rotation, make_poses, rotation_to_quaternion


def _catmull_rom(p0, p1, p2, p3, t):
    t = t[:, None]
    return 0.5 * ((2.0 * p1) + (-p0 + p2) * t + (2.0 * p0 - 5.0 * p1 + 4.0 * p2 - p3) * t * t
                  + (-p0 + 3.0 * p1 - 3.0 * p2 + p3) * t * t * t)


def _axis_angle(axis, angle):
    axis = axis / np.linalg.norm(axis)
    k = np.array([[0.0, -axis[2], axis[1]], [axis[2], 0.0, -axis[0]], [-axis[1], axis[0], 0.0]])
    return np.eye(3) + math.sin(angle) * k + (1.0 - math.cos(angle)) * (k @ k)


def random_trajectories(pois, n_traj: int, seed: int, len_range=(5, 40), r_min: float = 0.3,
                        r_max: float = 0.8, jitter_deg: float = 3.0):
    """``n_traj`` smooth trajectories around ``pois`` (k, 3); lengths uniform in len_range."""
    rng = np.random.default_rng(seed)
    pois = np.asarray(pois, dtype=np.float64).reshape(-1, 3)
    lengths = rng.integers(len_range[0], len_range[1] + 1, size=n_traj)
    offsets = np.zeros(n_traj + 1, dtype=np.int64)
    offsets[1:] = np.cumsum(lengths)
    all_pos, all_rot = [], []
    for t_idx in range(n_traj):
        poi = pois[rng.integers(len(pois))]
        d = rng.standard_normal((4, 3))
        d /= np.linalg.norm(d, axis=1, keepdims=True)
        # keep consecutive control points on the same side of the PoI
        for k in range(1, 4):
            if np.dot(d[k], d[k - 1]) < 0.0:
                d[k] = -d[k]
            d[k] = d[k - 1] + 0.6 * d[k]
            d[k] /= np.linalg.norm(d[k])
        radii = rng.uniform(r_min, r_max, size=4)
        t = np.linspace(0.0, 1.0, int(lengths[t_idx]))
        # spline the direction and the radius separately so the path keeps to the shell
        u = _catmull_rom(d[0], d[1], d[2], d[3], t)
        u /= np.linalg.norm(u, axis=1, keepdims=True)
        r = np.clip(_catmull_rom(*[np.array([x]) for x in radii], t)[:, 0], r_min, r_max)
        pos = poi[None, :] + r[:, None] * u
        rot = look_at_rotation(pos, poi)
        for k in range(len(pos)):
            ang = math.radians(jitter_deg) * rng.random()
            rot[k] = rot[k] @ _axis_angle(rng.standard_normal(3), ang)
        all_pos.append(pos)
        all_rot.append(rot)
    pos = np.concatenate(all_pos)
    rot = np.concatenate(all_rot)
    poses = make_poses(pos, rotation_to_quaternion(rot))
    return poses, offsets.astype(np.int32)


def horizon_trajectories(poi, n_traj: int, horizon: int, seed: int, r_min: float = 0.3, r_max: float = 0.8,
                         jitter_deg: float = 40.0):
    """``n_traj`` candidate trajectories of exactly ``horizon`` states around one PoI.

    The same construction as ``random_trajectories`` (spline of the
    direction and of the radius through four control points; look-at
    orientation tilted by up to ``jitter_deg`` about a random axis), drawn in
    whole arrays so that tens of thousands of candidates take well under a
    second.
    """
    rng = np.random.default_rng(seed)
    poi = np.asarray(poi, dtype=np.float64).reshape(3)
    d = rng.standard_normal((n_traj, 4, 3))
    d /= np.linalg.norm(d, axis=2, keepdims=True)
    for k in range(1, 4):
        flip = np.sum(d[:, k] * d[:, k - 1], axis=1) < 0.0
        d[flip, k] = -d[flip, k]
        d[:, k] = d[:, k - 1] + 0.6 * d[:, k]
        d[:, k] /= np.linalg.norm(d[:, k], axis=1, keepdims=True)
    radii = rng.uniform(r_min, r_max, size=(n_traj, 4))
    t = np.linspace(0.0, 1.0, horizon)[None, :, None]
    u = _catmull_rom_batch(d[:, 0, None], d[:, 1, None], d[:, 2, None], d[:, 3, None], t)
    u /= np.linalg.norm(u, axis=2, keepdims=True)
    rr = radii[:, :, None, None]
    r = np.clip(_catmull_rom_batch(rr[:, 0], rr[:, 1], rr[:, 2], rr[:, 3], t)[..., 0], r_min, r_max)
    pos = (poi[None, None, :] + r[..., None] * u).reshape(-1, 3)
    rot = look_at_rotation(pos, poi)
    axis = rng.standard_normal((len(pos), 3))
    axis /= np.linalg.norm(axis, axis=1, keepdims=True)
    ang = math.radians(jitter_deg) * rng.random(len(pos))
    K = np.zeros((len(pos), 3, 3))
    K[:, 0, 1], K[:, 0, 2], K[:, 1, 2] = -axis[:, 2], axis[:, 1], -axis[:, 0]
    K[:, 1, 0], K[:, 2, 0], K[:, 2, 1] = axis[:, 2], -axis[:, 1], axis[:, 0]
    tilt = np.eye(3)[None] + np.sin(ang)[:, None, None] * K + (1.0 - np.cos(ang))[:, None, None] * (K @ K)
    rot = rot @ tilt
    poses = make_poses(pos, rotation_to_quaternion(rot))
    offsets = (np.arange(n_traj + 1) * horizon).astype(np.int32)
    return poses, offsets


def _catmull_rom_batch(p0, p1, p2, p3, t):
    return 0.5 * ((2.0 * p1) + (-p0 + p2) * t + (2.0 * p0 - 5.0 * p1 + 4.0 * p2 - p3) * t * t
                  + (-p0 + 3.0 * p1 - 3.0 * p2 + p3) * t * t * t)
