"""Pins of the IG-interpolation / IG-cost oracle (no GPU): closed forms,
limits, invariants and hand-computed cases of Eq. 3, the orientation factor
and c_I."""

import math
from fractions import Fraction

import numpy as np
import pytest

from oracle import idw as I


def test_single_perspective_returns_its_gain():
    assert I.idw([0.3, -0.2, 0.5], [[1.0, 2.0, 3.0]], [7.25]) == 7.25


def test_constant_gains_are_reproduced_anywhere():
    rng = np.random.default_rng(0)
    pts = rng.standard_normal((50, 3))
    for q in rng.standard_normal((5, 3)):
        assert abs(I.idw(q, pts, np.full(50, 3.5)) - 3.5) < 1e-14


def test_equidistant_points_give_the_plain_mean():
    # the six vertices of an octahedron around the query
    c = np.array([0.2, -0.1, 0.4])
    pts = c + 0.3 * np.array([[1, 0, 0], [-1, 0, 0], [0, 1, 0], [0, -1, 0], [0, 0, 1], [0, 0, -1]])
    g = np.array([1.0, 2.0, 4.0, 8.0, 16.0, 32.0])
    assert abs(I.idw(c, pts, g) - 63.0 / 6.0) < 1e-13


def test_two_collinear_points_by_hand():
    # query at x = 1: distance 1 to p0 (x = 0) and 3 to p1 (x = 4); p = 2:
    # (2 / 1 + 12 / 9) / (1 / 1 + 1 / 9) = (18 + 12) / 10 = 3
    assert abs(I.idw([1, 0, 0], [[0, 0, 0], [4, 0, 0]], [2.0, 12.0]) - 3.0) < 1e-14
    # p = 1: (2 / 1 + 12 / 3) / (1 + 1 / 3) = 6 / (4 / 3) = 4.5
    assert abs(I.idw([1, 0, 0], [[0, 0, 0], [4, 0, 0]], [2.0, 12.0], p=1.0) - 4.5) < 1e-14


def test_power_zero_is_the_mean_and_large_power_the_nearest():
    rng = np.random.default_rng(1)
    pts = rng.standard_normal((20, 3))
    g = rng.random(20)
    q = rng.standard_normal(3)
    assert abs(I.idw(q, pts, g, p=0.0) - g.mean()) < 1e-14
    # nearest point at distance 0.5, the others at 0.6..1.5: (0.5 / 0.6)^400 ~ 1e-32
    dirs = rng.standard_normal((20, 3))
    dirs /= np.linalg.norm(dirs, axis=1, keepdims=True)
    r = np.concatenate([[0.5], rng.uniform(0.6, 1.5, 19)])
    assert abs(I.idw(q, q + dirs * r[:, None], g, p=400.0) - g[0]) < 1e-12


def test_coincident_query_takes_the_mean_of_the_coincident_points():
    pts = [[0, 0, 0], [1, 1, 1], [0, 0, 0], [2, 0, 0]]
    assert I.idw([0, 0, 0], pts, [3.0, 100.0, 5.0, 100.0]) == 4.0
    assert I.idw([2, 0, 0], pts, [3.0, 100.0, 5.0, 9.0]) == 9.0


def test_rigid_motion_invariance():
    rng = np.random.default_rng(2)
    pts = rng.standard_normal((30, 3))
    g = rng.random(30) * 10
    q = rng.standard_normal(3)
    Q, _ = np.linalg.qr(rng.standard_normal((3, 3)))
    t = rng.standard_normal(3)
    a = I.idw(q, pts, g)
    b = I.idw(Q @ q + t, pts @ Q.T + t, g)
    assert abs(a - b) <= 1e-12 * abs(a)


def test_weighted_mean_lies_between_the_extreme_gains():
    rng = np.random.default_rng(3)
    pts = rng.standard_normal((40, 3))
    g = rng.random(40) * 7 + 1
    for q in rng.standard_normal((10, 3)):
        v = I.idw(q, pts, g, p=2.0)
        assert g.min() <= v <= g.max()


def test_empty_id_contributes_nothing():
    assert I.idw([0, 0, 0], np.zeros((0, 3)), np.zeros(0)) == 0.0


def test_buffer_of_identical_ids_scales_by_the_harmonic_number():
    rng = np.random.default_rng(4)
    pts = rng.standard_normal((25, 3))
    g = rng.random(25)
    q = rng.standard_normal(3)
    h10 = float(sum(Fraction(1, k) for k in range(1, 11)))   # 7381 / 2520
    assert abs(h10 - 7381 / 2520) < 1e-15
    one = I.idw(q, pts, g)
    assert abs(I.id_buffer_gain(q, [(pts, g)] * 10, 10) - h10 * one) < 1e-12
    assert abs(I.id_buffer_gain(q, [(pts, g)], 10) - one) < 1e-15   # the newest ID weighs 1


def test_buffer_weights_by_hand():
    # two IDs in a buffer of 10: u = 8 (older, weight 1/2) and u = 9 (newer, weight 1)
    pts = np.array([[0.0, 0, 0], [1, 0, 0]])
    old = (pts, np.array([4.0, 4.0]))
    new = (pts, np.array([10.0, 10.0]))
    assert abs(I.id_buffer_gain([0.3, 0.2, 0.1], [old, new], 10) - (4.0 / 2 + 10.0)) < 1e-14
    assert abs(I.id_buffer_gain([0.3, 0.2, 0.1], [new, old], 10) - (10.0 / 2 + 4.0)) < 1e-14
    with pytest.raises(ValueError):
        I.id_buffer_gain([0, 0, 0], [old] * 3, 2)


IDENT = np.array([0.0, 0.0, 0.0, 1.0, 0.0, 0.0, 0.0], np.float32)   # camera at the origin looking along +z


def test_orientation_factor_on_axis_and_behind():
    assert I.orientation_factor(IDENT, [0.0, 0.0, 2.0], math.radians(60), math.radians(45)) == 1.0
    assert I.orientation_factor(IDENT, [0.0, 0.0, -2.0], math.radians(60), math.radians(45)) == 0.0
    assert I.orientation_factor(IDENT, [0.0, 0.0, 0.0], math.radians(60), math.radians(45)) == 0.0


@pytest.mark.parametrize("deg,inside", [(10.0, True), (29.0, True), (31.0, False), (-25.0, True), (-33.0, False)])
def test_orientation_factor_horizontal(deg, inside):
    t = math.radians(deg)
    poi = [0.7 * math.sin(t), 0.0, 0.7 * math.cos(t)]
    o = I.orientation_factor(IDENT, poi, math.radians(60), math.radians(45))
    assert (abs(o - math.cos(t)) < 1e-7) if inside else o == 0.0


@pytest.mark.parametrize("deg,inside", [(20.0, True), (-21.0, True), (23.0, False), (-24.0, False)])
def test_orientation_factor_vertical(deg, inside):
    t = math.radians(deg)
    poi = [0.0, 0.5 * math.sin(t), 0.5 * math.cos(t)]
    o = I.orientation_factor(IDENT, poi, math.radians(60), math.radians(45))
    assert (abs(o - math.cos(t)) < 1e-7) if inside else o == 0.0


def test_orientation_factor_look_at_and_roll():
    from workload import poses
    rng = np.random.default_rng(5)
    poi = np.array([0.4, 0.5, 0.3])
    pos = poi + rng.standard_normal((20, 3)) * 0.4
    ps = poses.look_at_poses(pos, poi)
    for p in ps:
        assert abs(I.orientation_factor(p, poi, math.radians(60), math.radians(45)) - 1.0) < 1e-6
    # a roll about the optical axis keeps an on-axis PoI on axis
    a = 0.7
    roll = np.array([math.cos(a / 2), 0.0, 0.0, math.sin(a / 2)])  # rotation about camera z
    for p in ps[:5]:
        q = p[3:]
        w1, x1, y1, z1 = q
        w2, x2, y2, z2 = roll
        qr = [w1 * w2 - x1 * x2 - y1 * y2 - z1 * z2, w1 * x2 + x1 * w2 + y1 * z2 - z1 * y2,
              w1 * y2 - x1 * z2 + y1 * w2 + z1 * x2, w1 * z2 + x1 * y2 - y1 * x2 + z1 * w2]
        pr = np.concatenate([p[:3], qr]).astype(np.float32)
        assert abs(I.orientation_factor(pr, poi, math.radians(60), math.radians(45)) - 1.0) < 1e-6


def test_ig_cost_by_hand():
    pts = np.array([[0.0, 0, 1], [0.1, 0, 1]])
    ids = [(pts, np.array([5.0, 5.0]))]
    ps = np.stack([IDENT, IDENT, IDENT]).astype(np.float64)
    ps[2, 2] = 3.0   # third camera sits beyond the PoI: PoI behind it, O = 0
    G, O, c = I.ig_cost(ps, [0, 2, 3], [0, 0, 2.0], math.radians(60), math.radians(45), ids, 1, w_i=2.0)
    assert np.allclose(G, 5.0) and list(O) == [1.0, 1.0, 0.0]
    assert abs(c[0] - 2 * 2.0 / (5.0 + 1e-7)) < 1e-12
    assert abs(c[1] - 2.0 / 1e-7) < 1e-3
    _, _, c0 = I.ig_cost(ps, [0, 3], [0, 0, 2.0], math.radians(60), math.radians(45), ids, 1, w_i=0.0)
    assert c0[0] == 0.0
