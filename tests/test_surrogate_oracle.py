"""Pins of the surrogate oracle (no GPU): brute-force convolution, finite
differences for every gradient, a hand-computed Adam step, crop geometry."""

import math

import numpy as np
import pytest

from oracle import surrogate as S
from workload import poses

TINY = ((8, 4, 1), (4, 4, 2))


def brute_conv(x, w, b, s):
    n, d, _, _, cin = x.shape
    cout = w.shape[0]
    do = (d - 1) // s + 1
    out = np.zeros((n, do, do, do, cout))
    for bi in range(n):
        for oz in range(do):
            for oy in range(do):
                for ox in range(do):
                    for co in range(cout):
                        acc = b[co]
                        for dz in range(3):
                            for dy in range(3):
                                for dx in range(3):
                                    iz, iy, ix = oz * s + dz - 1, oy * s + dy - 1, ox * s + dx - 1
                                    if 0 <= iz < d and 0 <= iy < d and 0 <= ix < d:
                                        tap = (dz * 3 + dy) * 3 + dx
                                        for ci in range(cin):
                                            acc += x[bi, iz, iy, ix, ci] * w[co, tap * cin + ci]
                        out[bi, oz, oy, ox, co] = acc
    return out


@pytest.mark.parametrize("stride", [1, 2])
def test_conv3d_matches_brute_force(stride):
    rng = np.random.default_rng(stride)
    x = rng.standard_normal((2, 5, 5, 5, 2))
    w = rng.standard_normal((3, 27 * 2))
    b = rng.standard_normal(3)
    assert np.allclose(S.conv3d(x, w, b, stride), brute_conv(x, w, b, stride), atol=1e-12)


@pytest.mark.parametrize("stride", [1, 2])
def test_conv3d_backward_matches_finite_differences(stride):
    rng = np.random.default_rng(10 + stride)
    x = rng.standard_normal((1, 4, 4, 4, 2))
    w = rng.standard_normal((3, 54))
    b = rng.standard_normal(3)
    dout = rng.standard_normal(S.conv3d(x, w, b, stride).shape)
    dx, dw, db = S.conv3d_backward(x, w, dout, stride)
    f = lambda xx, ww, bb: float(np.sum(S.conv3d(xx, ww, bb, stride) * dout))  # noqa: E731
    eps = 1e-6
    for idx in [(0, 1, 2, 3, 1), (0, 0, 0, 0, 0), (0, 3, 3, 3, 1)]:
        xp, xm = x.copy(), x.copy()
        xp[idx] += eps
        xm[idx] -= eps
        assert abs((f(xp, w, b) - f(xm, w, b)) / (2 * eps) - dx[idx]) < 1e-6
    for idx in [(0, 0), (2, 53), (1, 27)]:
        wp, wm = w.copy(), w.copy()
        wp[idx] += eps
        wm[idx] -= eps
        assert abs((f(x, wp, b) - f(x, wm, b)) / (2 * eps) - dw[idx]) < 1e-6
    assert np.allclose(db, dout.reshape(-1, 3).sum(0))


def test_network_gradients_match_finite_differences():
    rng = np.random.default_rng(3)
    p = S.init_params(5, layers=TINY, crop=8, hidden=6)
    p = {k: v.astype(np.float64) + 0.05 * rng.standard_normal(v.shape) for k, v in p.items()}
    crops = (rng.random((3, 8, 8, 8, 8)) < 0.3).astype(np.float64)
    feats = rng.standard_normal((3, 8))
    t = rng.standard_normal(3)
    loss, g = S.loss_and_grads(p, crops, feats, t, layers=TINY)
    eps = 1e-6
    for k in p:
        flat = p[k].reshape(-1)
        for j in rng.choice(flat.size, size=min(4, flat.size), replace=False):
            pp = {kk: vv.copy() for kk, vv in p.items()}
            pm = {kk: vv.copy() for kk, vv in p.items()}
            pp[k].reshape(-1)[j] += eps
            pm[k].reshape(-1)[j] -= eps
            num = (S.loss_and_grads(pp, crops, feats, t, layers=TINY)[0]
                   - S.loss_and_grads(pm, crops, feats, t, layers=TINY)[0]) / (2 * eps)
            assert abs(num - g[k].reshape(-1)[j]) <= 1e-6 + 1e-5 * abs(num), (k, j, num, g[k].reshape(-1)[j])


def test_target_scale_is_the_loss_of_scaled_targets():
    """loss_and_grads(t, target_scale=c) is the loss of the targets c t: the finite difference of
    mean (y - c t)^2 in a parameter matches its gradient, and it equals passing c t directly."""
    rng = np.random.default_rng(4)
    p = S.init_params(6, layers=TINY, crop=8, hidden=6)
    p = {k: v.astype(np.float64) + 0.05 * rng.standard_normal(v.shape) for k, v in p.items()}
    crops = (rng.random((3, 8, 8, 8, 8)) < 0.3).astype(np.float64)
    feats = rng.standard_normal((3, 8))
    t = rng.uniform(20.0, 90.0, 3)
    loss, g = S.loss_and_grads(p, crops, feats, t, layers=TINY, target_scale=0.01)
    y, _ = S.forward(p, crops, feats, layers=TINY)
    assert abs(loss - np.mean((y - 0.01 * t) ** 2)) < 1e-15
    loss2, g2 = S.loss_and_grads(p, crops, feats, 0.01 * t, layers=TINY)
    assert loss == loss2 and all(np.array_equal(g[k], g2[k]) for k in g)
    eps = 1e-6
    pp = {kk: vv.copy() for kk, vv in p.items()}
    pm = {kk: vv.copy() for kk, vv in p.items()}
    pp["g2"][0] += eps
    pm["g2"][0] -= eps
    num = (S.loss_and_grads(pp, crops, feats, t, layers=TINY, target_scale=0.01)[0]
           - S.loss_and_grads(pm, crops, feats, t, layers=TINY, target_scale=0.01)[0]) / (2 * eps)
    assert abs(num - g["g2"][0]) < 1e-7


def test_bf16_modelling_of_the_backward_pass():
    """With BF16 modelling the backward pass rounds dh and the masked input gradients: it stays close
    to the exact gradients (within a few BF16 units) but is not identical on random parameters, and it
    is identical when every such value is exactly representable (weights in {-1, 0, 1}, integer
    biases and inputs, dyadic residuals)."""
    rng = np.random.default_rng(7)
    p = S.init_params(8, layers=TINY, crop=8, hidden=6)
    p = {k: v.astype(np.float64) + 0.05 * rng.standard_normal(v.shape) for k, v in p.items()}
    crops = (rng.random((3, 8, 8, 8, 8)) < 0.3).astype(np.float64)
    feats = S._bf16(rng.standard_normal((3, 8)))
    t = rng.standard_normal(3)
    _, g = S.loss_and_grads(p, crops, feats, t, layers=TINY)
    _, gb = S.loss_and_grads(p, crops, feats, t, layers=TINY, bf16_activations=True)
    rel = {k: np.linalg.norm(gb[k] - g[k]) / max(np.linalg.norm(g[k]), 1e-30) for k in g}
    assert max(rel.values()) < 5e-2 and any(r > 0 for r in rel.values()), rel
    # exact case: integer weights and biases, dyadic residuals
    q = {k: np.sign(rng.standard_normal(v.shape)) * (rng.random(v.shape) < 0.15) for k, v in p.items()}
    for k in q:
        if k.startswith("b") or k.startswith("g"):
            q[k] = np.abs(q[k])
    crops4 = (rng.random((4, 8, 8, 8, 8)) < 0.3).astype(np.float64)
    ones = np.ones((4, 8))
    y, _ = S.forward(q, crops4, ones, layers=TINY)
    tq = y - np.array([1.0, -2.0, 1.0, 1.0])              # batch of 4: dy = 2 e / 4 is dyadic
    crops = crops4
    _, g = S.loss_and_grads(q, crops, ones, tq, layers=TINY)
    _, gb = S.loss_and_grads(q, crops, ones, tq, layers=TINY, bf16_activations=True)
    assert all(np.array_equal(g[k], gb[k]) for k in g)
    assert all(np.abs(g[k]).max() > 0 for k in g)


def test_bf16_modelling_rounds_the_stored_backward_values():
    """One sample through convolutions whose outputs are single voxels: the bias gradient of layer 0
    is then the (masked) input gradient at that voxel and g1's gradient is dh itself -- with BF16
    modelling both are BF16 values, without it they are not."""
    rng = np.random.default_rng(11)
    layers = ((8, 4, 8), (4, 4, 1))          # crop 8: stride 8 leaves one voxel, then one voxel
    p = S.init_params(12, layers=layers, crop=8, hidden=6)
    p = {k: v.astype(np.float64) + 0.3 * rng.standard_normal(v.shape) + 0.2 for k, v in p.items()}
    crops = (rng.random((1, 8, 8, 8, 8)) < 0.5).astype(np.float64)
    feats = rng.standard_normal((1, 8))
    t = np.array([-3.7])
    _, gb = S.loss_and_grads(p, crops, feats, t, layers=layers, bf16_activations=True)
    _, g = S.loss_and_grads(p, crops, feats, t, layers=layers)
    for k in ("g1", "b0"):
        assert np.abs(gb[k]).max() > 0, k
        assert np.array_equal(S._bf16(gb[k]), gb[k]), k
        assert not np.array_equal(S._bf16(g[k]), g[k]), k


def test_adam_two_steps_by_hand():
    p = {"a": np.array([1.0])}
    m = {"a": np.zeros(1)}
    v = {"a": np.zeros(1)}
    p1, m1, v1 = S.adam(p, {"a": np.array([0.5])}, m, v, 1, lr=0.1)
    # step 1: m = 0.05, v = 0.00025, m_hat = 0.5, v_hat = 0.25 -> p = 1 - 0.1 * 0.5 / (0.5 + 1e-8)
    assert abs(p1["a"][0] - (1.0 - 0.1 * 0.5 / (0.5 + 1e-8))) < 1e-15
    p2, _, _ = S.adam(p1, {"a": np.array([-1.0])}, m1, v1, 2, lr=0.1)
    m2 = 0.9 * 0.05 - 0.1
    v2 = 0.999 * 0.00025 + 0.001
    exp = p1["a"][0] - 0.1 * (m2 / (1 - 0.81)) / (math.sqrt(v2 / (1 - 0.999 ** 2)) + 1e-8)
    assert abs(p2["a"][0] - exp) < 1e-15


def test_bf16_rounding():
    vals = np.array([1.0, 1.0 + 2 ** -8, 1.0 + 3 * 2 ** -8, -2.5, 3.1415926], np.float32)
    r = S._bf16(vals)
    assert r[0] == 1.0 and r[1] == 1.0 and r[2] == 1.0 + 2 ** -6 and r[3] == -2.5
    assert abs(r[4] - 3.140625) < 1e-12


def _sample_points(pose, cc, voxel_size):
    """FP64 positions of the crop samples, an independent restatement."""
    q = np.asarray(pose[3:], np.float64)
    w, x, y, z = q
    R = np.array([[1 - 2 * (y * y + z * z), 2 * (x * y - w * z), 2 * (x * z + w * y)],
                  [2 * (x * y + w * z), 1 - 2 * (x * x + z * z), 2 * (y * z - w * x)],
                  [2 * (x * z - w * y), 2 * (y * z + w * x), 1 - 2 * (x * x + y * y)]])
    n = cc["n"]
    k, j, i = np.meshgrid(np.arange(n), np.arange(n), np.arange(n), indexing="ij")
    fr = (k + 0.5) / n
    cx = float(cc["x0"]) + i * float(cc["xs"])
    cy = float(cc["y0"]) + j * float(cc["ys"])
    pc = np.stack([cx * fr, cy * fr, float(cc["zc"]) * fr], -1)
    return (np.asarray(pose[:3], np.float64) + pc @ R.T) / voxel_size


@pytest.mark.parametrize("shift", [(0.0, 0.0, 0.0), (0.25, -0.5, 0.125)])
def test_frustum_crop_occupied_block(shift):
    """The crop of a known block; with the map's origin and the camera moved by the same vector
    (second case), positions are taken relative to the origin and nothing changes."""
    n = 8
    g = np.ones((40, 40, 40), np.uint8)           # all free
    g[21:24, 19:22, 24:27] = 2                    # occupied block x 24..26, y 19..21, z 21..23
    poi = np.array([25.5, 20.5, 22.5]) * 0.01
    pose = poses.look_at_poses(poi[None] + np.array([[0.06, -0.05, 0.04]]), poi)[0]
    cc = S.crop_consts(math.radians(60), math.radians(45), 0.2, crop=n)
    moved = pose.copy()
    moved[:3] = (pose[:3].astype(np.float64) + np.array(shift)).astype(moved.dtype)
    crop, feats = S.frustum_crop(g, 0.01, shift, moved, cc)
    pts = _sample_points(pose, cc, 0.01)
    inside = np.all((pts >= 0) & (pts < 40), axis=-1)
    cell = np.floor(pts).astype(int)
    near_edge = np.any(np.abs(pts - np.round(pts)) < 1e-4, axis=-1)
    want_occ = inside & (np.abs(cell[..., 0] - 25) <= 1) & (np.abs(cell[..., 1] - 20) <= 1) & \
        (np.abs(cell[..., 2] - 22) <= 1)
    assert want_occ.sum() > 0
    got_occ = crop[..., 2] == 1
    assert np.all((got_occ == want_occ) | near_edge)
    assert np.all(crop[..., 1][inside & ~want_occ & ~near_edge] == 1)
    assert np.all(crop[~inside].sum(-1) == 0)
    assert np.all(crop.sum(-1) <= 1) and np.all(crop[..., 3:] == 0)
    assert np.allclose(feats[:3], pose[:3] / 0.4, atol=1e-6) and feats[7] == 1.0


def test_frustum_crop_probability_classes():
    p = np.full((20, 20, 20), 0.5, np.float32)
    p[:, :, :10] = 0.1
    p[:, :, 15:] = 0.95
    pose = poses.look_at_poses(np.array([[0.02, 0.1, 0.1]]), np.array([0.19, 0.1, 0.1]))[0]
    cc = S.crop_consts(math.radians(30), math.radians(20), 0.15, crop=6)
    crop, _ = S.frustum_crop(p, 0.01, (0, 0, 0), pose, cc)
    pts = _sample_points(pose, cc, 0.01)
    x = np.floor(pts[..., 0]).astype(int)
    ok = np.all(np.abs(pts - np.round(pts)) > 1e-4, axis=-1)
    cls = np.where(x < 10, 1, np.where(x < 15, 0, 2))
    assert np.all((crop.argmax(-1) == cls)[ok])


def test_crop_codes_round_trip():
    rng = np.random.default_rng(9)
    codes = rng.integers(0, 4, (3, 5, 5, 5)).astype(np.uint8)
    oh = S.codes_to_onehot(codes)
    assert oh.shape == (3, 5, 5, 5, 8) and np.all(oh.sum(-1) == (codes > 0))
    assert np.all(oh[codes == 2][:, 1] == 1.0) and np.all(oh[..., 3:] == 0.0)
    assert np.array_equal(S.crop_codes(oh), codes)
