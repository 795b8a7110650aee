"""CPU oracle of the IG interpolation and the IG cost -- TEST INFRASTRUCTURE, NOT PRODUCT CODE.

Section IV ("Orientation Factor O(x_k) and IG G(x_k)" and "Cost Function Extension")
turns a buffer of information distributions (IDs; each one is N_P
perspective start points p_P,j with their IGs g_P,j) into a cost for a
candidate trajectory x_0..x_K:

* ``idw`` -- the inner fraction of Eq. 3: inverse-distance-weighted mean of
  one ID's gains at a camera position, with distance power p.
* ``id_buffer_gain`` -- Eq. 3: G(x_k), the sum over the N_B buffered IDs of
  that fraction weighted by 1 / (N_B - u), u = 0 the oldest.
* ``orientation_factor`` -- O(x_k): the cosine of the angle between the
  camera's optical axis and the direction to the PoI; zero when the PoI is
  outside the field of view.
* ``ig_cost`` -- c_I(x_0..x_K) = sum_k w_I / (O(x_k) G(x_k) + eps).

Everything is FP64 numpy, except the one yes/no decision "is the PoI inside
the field of view", which is taken in FP32 in a fixed operation order (no
fused multiply-add), the precision the GPU kernel takes it in, so both sides
decide alike on boundary cases.

Readings where the paper is silent:

* The buffer is ordered oldest first: with n <= N_B IDs stored, ID m
  (m = 0 oldest) has u = N_B - n + m, so the newest ID always weighs 1.
* Eq. 3 is used as printed: the ID weights 1 / (N_B - u) are not
  normalised.
* d_P,j is the Euclidean distance from the query camera position to the
  start point of perspective j.  A query that coincides with one or more
  start points takes, for that ID, the mean gain of those points (the limit
  of the weighted mean).  An ID with no perspectives contributes nothing.
* "Orientation outside the FoV": the PoI direction, in camera coordinates
  (x right, y down, z the optical axis), is inside when z > 0,
  |x| <= z tan(FoV_h / 2) and |y| <= z tan(FoV_v / 2).  A camera at the PoI
  has O = 0.
"""

from __future__ import annotations

import math

import numpy as np

EPS = 1e-7   # the paper's epsilon in c_I


def idw(query, persp, g, p=2.0):
    """Eq. 3's inner fraction at one position ``query`` (3,) for one ID.

    ``persp`` (n, 3) are the perspective start points p_P,j, ``g`` (n,) their
    IGs g_P,j.  Returns sum_j g_j d_j^-p / sum_j d_j^-p.
    """
    persp = np.asarray(persp, np.float64).reshape(-1, 3)
    g = np.asarray(g, np.float64).reshape(-1)
    if persp.shape[0] == 0:
        return 0.0
    d = np.sqrt(np.sum((persp - np.asarray(query, np.float64)) ** 2, axis=1))
    hit = d == 0.0
    if hit.any():
        return float(np.mean(g[hit]))
    w = d ** (-float(p))
    return float(np.sum(g * w) / np.sum(w))


def id_buffer_gain(query, ids, n_b, p=2.0):
    """G(x_k) of Eq. 3 at one position; ``ids`` lists (positions, gains), oldest first."""
    n = len(ids)
    if n > n_b:
        raise ValueError("more IDs than the buffer holds")
    total = 0.0
    for m, (persp, g) in enumerate(ids):
        u = n_b - n + m
        total += idw(query, persp, g, p) / (n_b - u)
    return total


def _rot_f32(q):
    """Camera-to-world rotation of the unit quaternion (w, x, y, z), every operation rounded to FP32."""
    f32 = np.float32
    w, x, y, z = (f32(v) for v in q)
    xx, yy, zz = x * x, y * y, z * z
    xy, xz, yz = x * y, x * z, y * z
    wx, wy, wz = w * x, w * y, w * z
    one, two = f32(1.0), f32(2.0)
    return [[one - two * (yy + zz), two * (xy - wz), two * (xz + wy)],
            [two * (xy + wz), one - two * (xx + zz), two * (yz - wx)],
            [two * (xz - wy), two * (yz + wx), one - two * (xx + yy)]]


def fov_tangents(fov_h, fov_v):
    """tan(FoV / 2) per axis, in FP64 from the FP32 angles, then rounded once to FP32."""
    return (np.float32(math.tan(float(np.float32(fov_h)) * 0.5)),
            np.float32(math.tan(float(np.float32(fov_v)) * 0.5)))


def poi_in_view(pose, poi, fov_h, fov_v):
    """FP32 decision: is the PoI inside the field of view of camera ``pose`` (7,)?

    c = R^T (p_PoI - p), each component ((R0k v0 + R1k v1) + R2k v2); inside
    iff c_z > 0, |c_x| <= c_z tan_h and |c_y| <= c_z tan_v.
    """
    f32 = np.float32
    R = _rot_f32(pose[3:7])
    v = [f32(f32(poi[a]) - f32(pose[a])) for a in range(3)]
    c = [f32(f32(f32(R[0][k] * v[0]) + f32(R[1][k] * v[1])) + f32(R[2][k] * v[2])) for k in range(3)]
    th, tv = fov_tangents(fov_h, fov_v)
    return bool(c[2] > 0 and abs(c[0]) <= f32(c[2] * th) and abs(c[1]) <= f32(c[2] * tv))


def orientation_factor(pose, poi, fov_h, fov_v):
    """O(x_k): cos of the angle between the optical axis and the PoI direction, 0 outside the FoV."""
    pos = np.asarray(pose[:3], np.float64)
    v = np.asarray(poi, np.float64) - pos
    dist = float(np.linalg.norm(v))
    if dist == 0.0 or not poi_in_view(pose, poi, fov_h, fov_v):
        return 0.0
    w, x, y, z = (float(t) for t in pose[3:7])
    axis = np.array([2 * (x * z + w * y), 2 * (y * z - w * x), 1 - 2 * (x * x + y * y)])  # R e_z
    return float(axis @ v / dist)


def ig_cost(poses, offsets, poi, fov_h, fov_v, ids, n_b, p=2.0, w_i=1.0, eps=EPS):
    """Per query pose G and O, and per trajectory c_I = sum_k w_I / (O G + eps).

    ``poses`` (n, 7) camera poses (position, quaternion w x y z) of all
    trajectories back to back; trajectory t owns rows offsets[t]..offsets[t+1].
    """
    poses = np.asarray(poses, np.float64)
    G = np.array([id_buffer_gain(q[:3], ids, n_b, p) for q in poses])
    O = np.array([orientation_factor(np.asarray(q, np.float32), poi, fov_h, fov_v) for q in poses])
    term = w_i / (O * G + eps)
    cost = np.array([term[offsets[t]:offsets[t + 1]].sum() for t in range(len(offsets) - 1)])
    return G, O, cost
