"""CPU oracle of the learned IG surrogate -- TEST INFRASTRUCTURE, NOT PRODUCT CODE.

The paper's Section III computes IG by raycasting.  The learned surrogate
(not in the paper) predicts a perspective's mean ray IG from a view-aligned
occupancy crop and the pose, so that only the most promising perspectives
are raycast exactly.  This module restates, plainly and in FP64 numpy, what
the CUDA surrogate computes, so the GPU kernels can be checked:

* ``frustum_crop``: the crop is a 32 x 32 x 32 grid of sample points inside
  the camera frustum: sample (i, j, k) lies on the ray through pixel centre
  (i, j) of a 32 x 32 image spanning the field of view, at depth fraction
  (k + 1/2) / 32 of the far plane d_Cam.  Each sample reads the map voxel
  that contains it; channels 0 / 1 / 2 are one-hot unknown / free /
  occupied, channels 3..7 are zero, samples outside the map are all zero.
  The sample arithmetic is FP32 in one fixed order (numpy rounds every
  float32 operation separately), as on the GPU, so crops are byte-exact.
* ``forward`` / ``backward``: four 3x3x3 convolutions (padding 1; strides
  2, 2, 2, 1; ReLU), flatten, concatenation with 8 pose features, a hidden
  layer of 128 ReLU units and one linear output; loss = mean squared error.
  Tensors are NDHWC; a convolution weight is [C_out, 27 * C_in] with the
  tap index (dz * 3 + dy) * 3 + dx and the input channel fastest.
* ``adam``: the Adam update.
"""

from __future__ import annotations

import math

import numpy as np

CROP = 32
C0 = 8
LAYERS = ((8, 16, 2), (16, 32, 2), (32, 64, 2), (64, 64, 1))   # (C_in, C_out, stride)
FEATS = 8
HIDDEN = 128


# --------------------------------------------------------------------------
# Frustum crop
# --------------------------------------------------------------------------

def crop_consts(fov_h: float, fov_v: float, max_range: float, crop: int = CROP):
    """Pixel-centre grid of the crop in the camera frame, FP64 then rounded once to FP32."""
    dh = float(max_range) * math.tan(float(np.float32(fov_h)) * 0.5)
    dv = float(max_range) * math.tan(float(np.float32(fov_v)) * 0.5)
    f32 = np.float32
    return {"x0": f32(-dh + dh / crop), "xs": f32(2.0 * dh / crop), "y0": f32(-dv + dv / crop),
            "ys": f32(2.0 * dv / crop), "zc": f32(max_range), "n": crop}


def _rot_f32(q):
    f32 = np.float32
    w, x, y, z = (f32(v) for v in q)
    xx, yy, zz = x * x, y * y, z * z
    xy, xz, yz = x * y, x * z, y * z
    wx, wy, wz = w * x, w * y, w * z
    one, two = f32(1.0), f32(2.0)
    return [[one - two * (yy + zz), two * (xy - wz), two * (xz + wy)],
            [two * (xy + wz), one - two * (xx + zz), two * (yz - wx)],
            [two * (xz - wy), two * (yz + wx), one - two * (xx + yy)]]


def voxel_class(value, occ_threshold=0.7, free_threshold=0.3):
    """0 unknown, 1 free, 2 occupied (state maps: the state itself, >= 2 occupied)."""
    if isinstance(value, (np.floating, float)) and not isinstance(value, (np.integer, int)):
        v = np.float32(value)
        return 2 if v > np.float32(occ_threshold) else (1 if v < np.float32(free_threshold) else 0)
    s = int(value)
    return 2 if s >= 2 else s


def frustum_crop(grid, voxel_size, origin, pose, cc, occ_threshold=0.7, free_threshold=0.3):
    """One-hot crop (n, n, n, 8) uint8 indexed [k, j, i, channel], and 8 pose features (float32)."""
    f32 = np.float32
    n = cc["n"]
    nz, ny, nx = grid.shape
    dims = (nx, ny, nz)
    inv_s = f32(1.0 / float(np.float32(voxel_size)))
    R = _rot_f32(pose[3:7])
    o = [f32((f32(pose[a]) - f32(origin[a])) * inv_s) for a in range(3)]
    out = np.zeros((n, n, n, C0), np.uint8)
    prob = grid.dtype == np.float32
    for k in range(n):
        fr = f32(f32(k + 0.5) / f32(n))
        for j in range(n):
            cy = f32(cc["y0"] + f32(f32(j) * cc["ys"]))
            for i in range(n):
                cx = f32(cc["x0"] + f32(f32(i) * cc["xs"]))
                p = (f32(cx * fr), f32(cy * fr), f32(cc["zc"] * fr))
                idx = []
                for a in range(3):
                    w = f32(f32(f32(R[a][0] * p[0]) + f32(R[a][1] * p[1])) + f32(R[a][2] * p[2]))
                    q = f32(o[a] + f32(w * inv_s))
                    idx.append(math.floor(float(q)))
                if all(0 <= idx[a] < dims[a] for a in range(3)):
                    v = grid[idx[2], idx[1], idx[0]]
                    c = voxel_class(v, occ_threshold, free_threshold) if prob else voxel_class(int(v))
                    out[k, j, i, c] = 1
    return out, pose_features(pose, voxel_size, origin, dims)


def crop_codes(onehot):
    """One-hot crops (..., 8) -> class codes (...,): 0 no channel set (outside the map), else 1 + channel."""
    oh = np.asarray(onehot)
    return np.where(oh.any(axis=-1), oh.argmax(axis=-1) + 1, 0).astype(np.uint8)


def codes_to_onehot(codes, dtype=np.float64):
    """Class codes (...,) -> one-hot (..., 8): code c sets channel c - 1, code 0 nothing."""
    c = np.asarray(codes).astype(np.int64)
    out = np.zeros(c.shape + (C0,), dtype)
    np.put_along_axis(out, np.maximum(c - 1, 0)[..., None], (c > 0)[..., None].astype(dtype), axis=-1)
    return out


def pose_features(pose, voxel_size, origin, dims):
    """(position - origin) / map extent per axis, the quaternion, and a constant 1."""
    f32 = np.float32
    feats = np.zeros(FEATS, np.float32)
    for a in range(3):
        ext = f32(f32(dims[a]) * f32(voxel_size))
        feats[a] = f32(f32(f32(pose[a]) - f32(origin[a])) / ext)
    feats[3:7] = np.asarray(pose[3:7], np.float32)
    feats[7] = 1.0
    return feats


# --------------------------------------------------------------------------
# Network
# --------------------------------------------------------------------------

def conv3d(x, w, b, stride):
    """NDHWC 3x3x3 convolution, padding 1: out[o] = b + sum_tap w[:, tap] . x[o*s + d - 1]."""
    n, d, h, wd, cin = x.shape
    cout = w.shape[0]
    do = (d - 1) // stride + 1
    xp = np.zeros((n, d + 2, h + 2, wd + 2, cin), x.dtype)
    xp[:, 1:-1, 1:-1, 1:-1] = x
    out = np.zeros((n, do, do, do, cout), np.float64) + b
    for dz in range(3):
        for dy in range(3):
            for dx in range(3):
                tap = (dz * 3 + dy) * 3 + dx
                patch = xp[:, dz:dz + stride * do:stride, dy:dy + stride * do:stride, dx:dx + stride * do:stride]
                out += patch @ w[:, tap * cin:(tap + 1) * cin].T
    return out


def conv3d_backward(x, w, dout, stride):
    """Gradients of conv3d w.r.t. its input, weight and bias."""
    n, d, h, wd, cin = x.shape
    do = dout.shape[1]
    xp = np.zeros((n, d + 2, h + 2, wd + 2, cin), np.float64)
    xp[:, 1:-1, 1:-1, 1:-1] = x
    dxp = np.zeros_like(xp)
    dw = np.zeros_like(w, dtype=np.float64)
    flat = dout.reshape(-1, dout.shape[-1])
    for dz in range(3):
        for dy in range(3):
            for dx in range(3):
                tap = (dz * 3 + dy) * 3 + dx
                sl = (slice(None), slice(dz, dz + stride * do, stride), slice(dy, dy + stride * do, stride),
                      slice(dx, dx + stride * do, stride))
                patch = xp[sl].reshape(-1, cin)
                dw[:, tap * cin:(tap + 1) * cin] += flat.T @ patch
                dxp[sl] += dout @ w[:, tap * cin:(tap + 1) * cin]
    return dxp[:, 1:-1, 1:-1, 1:-1], dw, flat.sum(axis=0)


def init_params(seed: int, layers=LAYERS, crop=CROP, hidden=HIDDEN, feats=FEATS):
    """He-normal weights, zero biases (FP32)."""
    rng = np.random.default_rng(seed)
    p = {}
    size = crop
    for i, (cin, cout, s) in enumerate(layers):
        p[f"w{i}"] = (rng.standard_normal((cout, 27 * cin)) * math.sqrt(2.0 / (27 * cin))).astype(np.float32)
        p[f"b{i}"] = np.zeros(cout, np.float32)
        size = (size - 1) // s + 1
    flat = size ** 3 * layers[-1][1]
    p["f1"] = (rng.standard_normal((hidden, flat + feats)) * math.sqrt(2.0 / (flat + feats))).astype(np.float32)
    p["g1"] = np.zeros(hidden, np.float32)
    p["f2"] = (rng.standard_normal(hidden) * math.sqrt(1.0 / hidden)).astype(np.float32)
    p["g2"] = np.zeros(1, np.float32)
    return p


def _bf16(a):
    """Round to BF16 (nearest even), returned as float64."""
    a32 = np.asarray(a, np.float32)
    u = a32.view(np.uint32).astype(np.uint64)
    u = ((u + 0x7FFF + ((u >> 16) & 1)) >> 16) << 16
    return u.astype(np.uint32).view(np.float32).astype(np.float64)


def forward(params, crops, feats, layers=LAYERS, bf16_activations=False):
    """Predictions (n,) and the cache backward needs.  ``crops`` (n, D, D, D, C0)."""
    rnd = _bf16 if bf16_activations else (lambda a: np.asarray(a, np.float64))
    x = rnd(crops)
    acts = [x]
    for i, (cin, cout, s) in enumerate(layers):
        z = conv3d(acts[-1], np.asarray(params[f"w{i}"], np.float64), np.asarray(params[f"b{i}"], np.float64), s)
        acts.append(rnd(np.maximum(z, 0.0)))
    n = x.shape[0]
    X = np.concatenate([acts[-1].reshape(n, -1), rnd(feats)], axis=1)
    h = rnd(np.maximum(X @ np.asarray(params["f1"], np.float64).T + params["g1"], 0.0))
    y = h @ np.asarray(params["f2"], np.float64) + float(params["g2"][0])
    return y, {"acts": acts, "X": X, "h": h}


def loss_and_grads(params, crops, feats, targets, layers=LAYERS, bf16_activations=False, target_scale=1.0):
    """MSE loss and the gradient of every parameter (dict like ``params``).

    The loss is mean (y - c t)^2 with the target scale c.  With ``bf16_activations`` the
    quantities the GPU stores in BF16 are rounded to BF16 here too: the forward activations
    (see ``forward``), and in the backward pass the hidden-layer gradient dh and the gradient
    with respect to every convolution's input after its ReLU mask (each computed in full
    precision, then rounded once), so that the remaining differences are those of FP32 versus
    FP64 accumulation.
    """
    rnd = _bf16 if bf16_activations else (lambda a: np.asarray(a, np.float64))
    y, c = forward(params, crops, feats, layers, bf16_activations)
    n = len(y)
    t = np.asarray(targets, np.float64) * float(target_scale)
    loss = float(np.mean((y - t) ** 2))
    dy = 2.0 * (y - t) / n
    g = {"g2": np.array([dy.sum()]), "f2": c["h"].T @ dy}
    dh = rnd(np.outer(dy, np.asarray(params["f2"], np.float64)) * (c["h"] > 0))
    g["f1"] = dh.T @ c["X"]
    g["g1"] = dh.sum(axis=0)
    dX = dh @ np.asarray(params["f1"], np.float64)
    acts = c["acts"]
    da = rnd(dX[:, :acts[-1][0].size].reshape(acts[-1].shape) * (acts[-1] > 0))
    for i in range(len(layers) - 1, -1, -1):
        cin, cout, s = layers[i]
        dxin, dw, db = conv3d_backward(acts[i], np.asarray(params[f"w{i}"], np.float64), da, s)
        g[f"w{i}"] = dw
        g[f"b{i}"] = db
        if i > 0:
            da = rnd(dxin * (acts[i] > 0))
    return loss, g


def adam(params, grads, m, v, step, lr, beta1=0.9, beta2=0.999, eps=1e-8):
    """One Adam update in FP64 on copies; returns (params, m, v)."""
    out_p, out_m, out_v = {}, {}, {}
    for k in params:
        g = np.asarray(grads[k], np.float64)
        mk = beta1 * np.asarray(m[k], np.float64) + (1.0 - beta1) * g
        vk = beta2 * np.asarray(v[k], np.float64) + (1.0 - beta2) * g * g
        mh = mk / (1.0 - beta1 ** step)
        vh = vk / (1.0 - beta2 ** step)
        out_p[k] = np.asarray(params[k], np.float64) - lr * mh / (np.sqrt(vh) + eps)
        out_m[k], out_v[k] = mk, vk
    return out_p, out_m, out_v
