"""Seeded synthetic depth scans (inputs only).

The paper inserts point clouds from an end-effector Azure Kinect; recordings
are not available, so an analytic tabletop scene is rendered by a pinhole
depth camera instead: floor, a table on four legs, and boxes and spheres on
the table.  Each pixel's ray (through the pixel centre) is intersected with
every primitive in FP64; the nearest hit within the camera's range is the
pixel's point (optionally perturbed along the ray by Gaussian range noise),
pixels that see nothing within range give no point.  Output: float32 world
points (n, 3), pixel order.  No voxel arithmetic happens here.
"""

from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np

from .poses import look_at_poses


@dataclass
class Scene:
    floor_z: float
    boxes: np.ndarray      # (k, 2, 3) axis-aligned boxes (lo, hi), metres
    spheres: np.ndarray    # (m, 4) centre and radius, metres


def tabletop_scene(seed: int = 0, n_objects: int = 40, extent: float = 2.56) -> Scene:
    """Floor, a 1.6 x 1.0 m table top at 0.75 m on four legs, objects of 3-15 cm on it."""
    rng = np.random.default_rng(seed)
    c = extent / 2
    top = 0.75
    boxes = [[[c - 0.8, c - 0.5, top - 0.04], [c + 0.8, c + 0.5, top]]]
    for sx in (-1, 1):
        for sy in (-1, 1):
            lx, ly = c + sx * 0.72, c + sy * 0.42
            boxes.append([[lx - 0.03, ly - 0.03, 0.02], [lx + 0.03, ly + 0.03, top - 0.04]])
    spheres = []
    for _ in range(n_objects):
        x, y = rng.uniform(c - 0.75, c + 0.75), rng.uniform(c - 0.45, c + 0.45)
        if rng.random() < 0.5:
            h = rng.uniform(0.03, 0.15, 3)
            boxes.append([[x - h[0] / 2, y - h[1] / 2, top], [x + h[0] / 2, y + h[1] / 2, top + h[2]]])
        else:
            r = rng.uniform(0.03, 0.08)
            spheres.append([x, y, top + r, r])
    return Scene(0.02, np.array(boxes, np.float64), np.array(spheres, np.float64).reshape(-1, 4))


def _rotation(q):
    w, x, y, z = (float(v) for v in q)
    return np.array([[1 - 2 * (y * y + z * z), 2 * (x * y - w * z), 2 * (x * z + w * y)],
                     [2 * (x * y + w * z), 1 - 2 * (x * x + z * z), 2 * (y * z - w * x)],
                     [2 * (x * z - w * y), 2 * (y * z + w * x), 1 - 2 * (x * x + y * y)]])


def depth_points(scene: Scene, pose, width: int, height: int, fov_h: float, fov_v: float, max_depth: float,
                 noise: float = 0.0, seed: int = 0) -> np.ndarray:
    """The point cloud of one depth image taken from camera ``pose`` (7,)."""
    th, tv = math.tan(fov_h / 2), math.tan(fov_v / 2)
    u = (2.0 * (np.arange(width) + 0.5) / width - 1.0) * th
    v = (2.0 * (np.arange(height) + 0.5) / height - 1.0) * tv
    cu, cv = np.meshgrid(u, v)
    dirs = np.stack([cu, cv, np.ones_like(cu)], -1).reshape(-1, 3)
    dirs /= np.linalg.norm(dirs, axis=1, keepdims=True)
    d = dirs @ _rotation(pose[3:7]).T
    o = np.asarray(pose[:3], np.float64)
    t = np.full(len(d), np.inf)
    with np.errstate(divide="ignore", invalid="ignore"):
        tf = (scene.floor_z - o[2]) / d[:, 2]
        t = np.where((tf > 0) & np.isfinite(tf), np.minimum(t, tf), t)
        for lo, hi in scene.boxes:
            t1, t2 = (lo - o) / d, (hi - o) / d
            near = np.nanmax(np.minimum(t1, t2), axis=1)
            far = np.nanmin(np.maximum(t1, t2), axis=1)
            hit = (near <= far) & (near > 0)
            t = np.where(hit, np.minimum(t, near), t)
        for cx, cy, cz, r in scene.spheres:
            oc = o - np.array([cx, cy, cz])
            b = d @ oc
            disc = b * b - (oc @ oc - r * r)
            ts = -b - np.sqrt(np.maximum(disc, 0.0))
            t = np.where((disc >= 0) & (ts > 0), np.minimum(t, ts), t)
    keep = t <= max_depth
    t = t[keep]
    if noise > 0:
        t = t + np.random.default_rng(seed).normal(0.0, noise, len(t))
    return (o[None, :] + t[:, None] * d[keep]).astype(np.float32)


def scan_poses(poi, n: int, seed: int, r_min: float = 0.6, r_max: float = 1.2, min_height: float = 0.35):
    """n camera poses above the table around ``poi``, looking at it."""
    rng = np.random.default_rng(seed)
    out = []
    while len(out) < n:
        v = rng.standard_normal(3)
        v /= np.linalg.norm(v)
        if v[2] * r_max < min_height:
            continue
        out.append(np.asarray(poi) + v * rng.uniform(r_min, r_max))
    return look_at_poses(np.array(out), poi)
