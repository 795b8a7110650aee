"""CPU oracle of the voxel-map update from a depth point cloud -- TEST INFRASTRUCTURE, NOT PRODUCT CODE.

Section III: every captured point cloud is thinned by a voxel filter and
inserted into the probabilistic voxel map whose states and occupancy
probabilities P(v) the IG is computed from.  The paper names the libraries
(PCL's voxel filter, UfoMap) but not the update; this module restates the
standard occupancy-grid insertion in UfoMap's discrete form:

* voxel filter: each point is represented by the map voxel that contains it
  (leaf size = s_Vox); each distinct endpoint voxel inside the map is
  observed as occupied once per scan ("hit");
* free space: a ray from the sensor position to the centre of each point's
  voxel (the FP32 reference walk of the IG path, clipped to the map) marks
  every voxel it visits as observed free ("miss"), at most once per scan;
  a voxel that is also a hit in the same scan is only a hit;
* update of an FP32 probability map: the Bayes / log-odds update written as
  a ratio, P' = P p / (P p + (1 - P)(1 - p)) with p = p_hit or p_miss,
  clamped to [P_min, P_max]; state maps: hit -> occupied (2), miss -> free (1);
* points that are not finite, farther than max_range from the sensor (when
  max_range > 0), or 2^22 voxels or more from the map origin on some axis
  (where voxel centres stop being exact in FP32), are ignored.

Readings (the paper is silent): p_hit 0.7, p_miss 0.4, clamping [0.1192,
0.971] (the defaults of the OctoMap / UfoMap family); the ratio form keeps
every step an IEEE basic operation, so this oracle and the GPU agree bit for
bit (numpy float32 rounds every operation).  The walk is the oracle's FP32
reference walk (``oracle.trace``), pinned separately against brute force.
"""

from __future__ import annotations

import numpy as np

from . import trace

P_HIT, P_MISS, P_MIN, P_MAX = 0.7, 0.4, 0.1192, 0.971
f32 = np.float32


def update_f32(P, p, p_min=P_MIN, p_max=P_MAX):
    """One observation with likelihood p of P (scalar or array), FP32 in a fixed order, clamped."""
    P, p = np.asarray(P, np.float32), f32(p)
    a = P * p
    b = (f32(1.0) - P) * (f32(1.0) - p)
    q = a / (a + b)
    lo, hi = f32(p_min), f32(p_max)
    return np.where(q < lo, lo, np.where(q > hi, hi, q)).astype(np.float32)


def scan_sets(points, sensor, dims, voxel_size, origin=(0.0, 0.0, 0.0), max_range=0.0):
    """(hit set, miss set) of linear voxel indices for one scan (miss excludes hits).

    Array arithmetic: numpy rounds every float32 element operation exactly as
    the scalar operation would.
    """
    nx, ny, nz = dims
    inv_s = f32(1.0 / float(f32(voxel_size)))
    org = np.asarray(origin, np.float32)
    o = (np.asarray(sensor, np.float32) - org) * inv_s
    p = np.asarray(points, np.float32).reshape(-1, 3)
    p = p[np.all(np.isfinite(p), axis=1)]
    if max_range > 0:
        dd = p - np.asarray(sensor, np.float32)
        r2 = (dd[:, 0] * dd[:, 0] + dd[:, 1] * dd[:, 1]) + dd[:, 2] * dd[:, 2]
        p = p[r2 <= f32(max_range) * f32(max_range)]
    q = (p - org) * inv_s
    q = q[np.all(np.abs(q) < f32(2.0 ** 22), axis=1)]
    idx = np.unique(np.floor(q).astype(np.int64), axis=0)       # distinct endpoint voxels: one ray each
    inside = np.all((idx >= 0) & (idx < np.array([nx, ny, nz])), axis=1)
    hits = set(((idx[inside, 2] * ny + idx[inside, 1]) * nx + idx[inside, 0]).tolist())
    misses = set()
    for e in idx:
        d = (e.astype(np.float32) + f32(0.5)) - o
        misses.update(trace(dims, o, d, "f32").tolist())
    return hits, misses - hits


def insert(grid, points, sensor, voxel_size, origin=(0.0, 0.0, 0.0), p_hit=P_HIT, p_miss=P_MISS, p_min=P_MIN,
           p_max=P_MAX, max_range=0.0):
    """The map after one scan.  ``grid`` (nz, ny, nx): float32 P or uint8 states (not modified)."""
    nz, ny, nx = grid.shape
    hits, misses = scan_sets(points, sensor, (nx, ny, nz), voxel_size, origin, max_range)
    out = grid.copy()
    flat = out.reshape(-1)
    h = np.array(sorted(hits), np.int64)
    m = np.array(sorted(misses), np.int64)
    if grid.dtype == np.float32:
        flat[h] = update_f32(flat[h], p_hit, p_min, p_max)
        flat[m] = update_f32(flat[m], p_miss, p_min, p_max)
    else:
        flat[h] = 2
        flat[m] = 1
    return out
