"""Seeded camera poses around a point of interest (inputs only).

A pose is 7 float32 values ``[px, py, pz, qw, qx, qy, qz]``: the camera
position in world metres and the unit quaternion of the camera-to-world
rotation.  Camera frame: +z is the optical axis, +x points right and +y
points down in the image.

Perspective positions follow Section III ("Perspective Selection"): N_P
points around the PoI, either on a sphere, on a shell of radii, or uniform in
a ball of radius r_S by Muller's method (Eq. 1).  The orientation of every
perspective looks from its position towards the PoI.  The roll about the
optical axis is not fixed by the paper; here the image x axis is horizontal:
``x_cam = normalize(z_cam x up)`` with ``up = +z`` (``+x`` when the optical
axis is within ~2.6 degrees of vertical), ``y_cam = z_cam x x_cam``.
"""

from __future__ import annotations

import math

import numpy as np

GOLDEN_ANGLE = math.pi * (3.0 - math.sqrt(5.0))


def fibonacci_directions(n: int) -> np.ndarray:
    """n unit vectors on a Fibonacci (golden-angle) sphere, FP64, shape (n, 3).

    Point k has z = 1 - (2k + 1)/n and azimuth k * golden_angle.
    """
    k = np.arange(n, dtype=np.float64)
    z = 1.0 - (2.0 * k + 1.0) / n
    r = np.sqrt(np.maximum(0.0, 1.0 - z * z))
    phi = k * GOLDEN_ANGLE
    return np.stack([r * np.cos(phi), r * np.sin(phi), z], axis=1)


def muller_draws(n: int, seed: int):
    """The random numbers Eq. 1 consumes: X ~ N(0, 1)^3 per point and X_R ~ U(0, 1)."""
    rng = np.random.default_rng(seed)
    x = rng.standard_normal((n, 3))
    xr = rng.random(n)
    return x, xr


def muller_ball(x: np.ndarray, xr: np.ndarray, r_s: float) -> np.ndarray:
    """Eq. 1: p = r_S * X_R^(1/3) * X / |X|, uniform in the ball of radius r_S.

    ``x`` holds normal draws (n, 3) and ``xr`` uniform draws (n,); the cube
    root of a uniform radius fraction gives a uniform density in the ball.
    """
    norm = np.sqrt(np.sum(x * x, axis=1, keepdims=True))
    return r_s * np.cbrt(xr)[:, None] * x / norm


def look_at_rotation(pos: np.ndarray, poi) -> np.ndarray:
    """Camera-to-world rotation matrices (n, 3, 3), FP64, columns x_cam, y_cam, z_cam."""
    pos = np.atleast_2d(np.asarray(pos, dtype=np.float64))
    poi = np.asarray(poi, dtype=np.float64)
    z = poi[None, :] - pos
    z /= np.linalg.norm(z, axis=1, keepdims=True)
    up = np.tile(np.array([0.0, 0.0, 1.0]), (len(z), 1))
    vertical = np.abs(z[:, 2]) > 0.999
    up[vertical] = np.array([1.0, 0.0, 0.0])
    x = np.cross(z, up)
    x /= np.linalg.norm(x, axis=1, keepdims=True)
    y = np.cross(z, x)
    return np.stack([x, y, z], axis=2)


def rotation_to_quaternion(r: np.ndarray) -> np.ndarray:
    """Unit quaternions (w, x, y, z) with w >= 0 for rotation matrices (n, 3, 3), FP64."""
    r = np.asarray(r, dtype=np.float64)
    n = r.shape[0]
    q = np.empty((n, 4))
    tr = r[:, 0, 0] + r[:, 1, 1] + r[:, 2, 2]
    for k in range(n):
        m = r[k]
        if tr[k] > 0.0:
            s = math.sqrt(tr[k] + 1.0) * 2.0
            q[k] = [0.25 * s, (m[2, 1] - m[1, 2]) / s, (m[0, 2] - m[2, 0]) / s, (m[1, 0] - m[0, 1]) / s]
        elif m[0, 0] > m[1, 1] and m[0, 0] > m[2, 2]:
            s = math.sqrt(1.0 + m[0, 0] - m[1, 1] - m[2, 2]) * 2.0
            q[k] = [(m[2, 1] - m[1, 2]) / s, 0.25 * s, (m[0, 1] + m[1, 0]) / s, (m[0, 2] + m[2, 0]) / s]
        elif m[1, 1] > m[2, 2]:
            s = math.sqrt(1.0 + m[1, 1] - m[0, 0] - m[2, 2]) * 2.0
            q[k] = [(m[0, 2] - m[2, 0]) / s, (m[0, 1] + m[1, 0]) / s, 0.25 * s, (m[1, 2] + m[2, 1]) / s]
        else:
            s = math.sqrt(1.0 + m[2, 2] - m[0, 0] - m[1, 1]) * 2.0
            q[k] = [(m[1, 0] - m[0, 1]) / s, (m[0, 2] + m[2, 0]) / s, (m[1, 2] + m[2, 1]) / s, 0.25 * s]
    q /= np.linalg.norm(q, axis=1, keepdims=True)
    q[q[:, 0] < 0] *= -1.0
    return q


def make_poses(pos: np.ndarray, quat: np.ndarray) -> np.ndarray:
    """Pack positions (n, 3) and quaternions (n, 4) into float32 poses (n, 7)."""
    out = np.empty((len(pos), 7), dtype=np.float32)
    out[:, :3] = pos
    out[:, 3:] = quat
    return np.ascontiguousarray(out)


def look_at_poses(pos: np.ndarray, poi) -> np.ndarray:
    """Poses at ``pos`` whose optical axes point at ``poi``."""
    return make_poses(pos, rotation_to_quaternion(look_at_rotation(pos, poi)))


def sphere_views(poi, n: int, radius: float) -> np.ndarray:
    """n poses on the sphere of ``radius`` around ``poi`` (Fibonacci layout)."""
    pos = np.asarray(poi, dtype=np.float64)[None, :] + radius * fibonacci_directions(n)
    return look_at_poses(pos, poi)


def shell_views(poi, n: int, r_min: float, r_max: float, seed: int) -> np.ndarray:
    """n poses on Fibonacci directions with radii drawn uniformly in [r_min, r_max]."""
    rng = np.random.default_rng(seed)
    radii = rng.uniform(r_min, r_max, size=n)
    pos = np.asarray(poi, dtype=np.float64)[None, :] + radii[:, None] * fibonacci_directions(n)
    return look_at_poses(pos, poi)


def ball_views(poi, n: int, r_s: float, seed: int) -> np.ndarray:
    """n poses uniform in the ball of radius r_S around ``poi`` (Eq. 1), looking at it."""
    x, xr = muller_draws(n, seed)
    pos = np.asarray(poi, dtype=np.float64)[None, :] + muller_ball(x, xr, r_s)
    return look_at_poses(pos, poi)
