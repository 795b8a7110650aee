"""Pins of the map-update oracle (no GPU): closed forms of the occupancy
update, hand-worked scans on a small map, and the free space of random scans
against the brute-force (slab-test) walk."""

import math

import numpy as np
import pytest

import oracle
from oracle import insert as I

f32 = np.float32


def ulps(a, b):
    return abs(float(a) - float(b)) / float(np.spacing(f32(b)))


def test_repeated_hits_and_misses_follow_the_closed_form_then_clamp():
    for p, lim in ((I.P_HIT, I.P_MAX), (I.P_MISS, I.P_MIN)):
        P = f32(0.5)
        for k in range(1, 40):
            P = I.update_f32(P, p)
            exact = p ** k / (p ** k + (1 - p) ** k)        # k equal observations: log-odds add up
            if (p > 0.5 and exact < lim) or (p < 0.5 and exact > lim):
                assert ulps(P, exact) <= 4 * k, (p, k, P, exact)
            else:
                assert P == f32(lim), (p, k, P)


def test_one_hit_from_unknown_lands_exactly_on_p_hit_and_one_miss_on_p_miss():
    assert I.update_f32(0.5, I.P_HIT) == f32(0.7)
    assert I.update_f32(0.5, I.P_MISS) == f32(0.4)


def test_hit_then_miss_is_the_product_rule():
    exact = 0.7 * 0.4 / (0.7 * 0.4 + 0.3 * 0.6)             # 0.28 / 0.46
    a = I.update_f32(I.update_f32(0.5, I.P_HIT), I.P_MISS)
    b = I.update_f32(I.update_f32(0.5, I.P_MISS), I.P_HIT)
    assert ulps(a, exact) <= 3 and ulps(b, exact) <= 3


def _row(grid):
    return grid[1, 1, :]


UNKNOWN = np.full((3, 3, 10), 0.5, np.float32)    # nz, ny, nx; voxel 1 m, origin 0
SENSOR = (0.5, 1.5, 1.5)


def test_single_point_by_hand():
    g = I.insert(UNKNOWN, [[7.5, 1.5, 1.5]], SENSOR, 1.0)
    assert np.all(_row(g)[:7] == f32(0.4)) and _row(g)[7] == f32(0.7) and np.all(_row(g)[8:] == 0.5)
    g[1, 1, :] = 0.5
    assert np.all(g == 0.5)                                   # nothing else touched


def test_single_point_by_hand_with_the_map_moved():
    """The same scan with the map's origin, the sensor and the point all moved by (-4, 2, 0.5) m:
    positions are taken relative to the origin, so the update is the same (dyadic values, exact in FP32)."""
    shift = np.array([-4.0, 2.0, 0.5])
    g = I.insert(UNKNOWN, [np.array([7.5, 1.5, 1.5]) + shift], tuple(np.array(SENSOR) + shift), 1.0,
                 origin=tuple(shift))
    assert np.array_equal(g, I.insert(UNKNOWN, [[7.5, 1.5, 1.5]], SENSOR, 1.0))


def test_points_in_one_voxel_are_one_hit():
    g = I.insert(UNKNOWN, [[7.2, 1.5, 1.5], [7.8, 1.1, 1.9], [7.5, 1.5, 1.5]], SENSOR, 1.0)
    assert _row(g)[7] == f32(0.7)


def test_a_voxel_hit_and_crossed_in_one_scan_is_only_a_hit():
    g = I.insert(UNKNOWN, [[7.5, 1.5, 1.5], [4.5, 1.5, 1.5]], SENSOR, 1.0)
    assert _row(g)[4] == f32(0.7) and _row(g)[7] == f32(0.7)
    assert all(_row(g)[x] == f32(0.4) for x in (0, 1, 2, 3, 5, 6))


def test_endpoint_outside_the_map_carves_free_space_only():
    g = I.insert(UNKNOWN, [[15.5, 1.5, 1.5]], SENSOR, 1.0)
    assert np.all(_row(g) == f32(0.4))


def test_max_range_and_non_finite_points_are_ignored():
    g = I.insert(UNKNOWN, [[7.5, 1.5, 1.5], [np.nan, 1.5, 1.5], [np.inf, 1.0, 1.0]], SENSOR, 1.0, max_range=5.0)
    assert np.all(g == 0.5)
    g = I.insert(UNKNOWN, [[4.5, 1.5, 1.5]], SENSOR, 1.0, max_range=5.0)
    assert _row(g)[4] == f32(0.7)
    assert np.all(I.insert(UNKNOWN, [[2.0 ** 22, 1.5, 1.5]], SENSOR, 1.0) == 0.5)   # too far from the origin
    g = I.insert(UNKNOWN, [[2.0 ** 22 - 1.0, 1.5, 1.5]], SENSOR, 1.0)
    assert np.all(_row(g) == f32(0.4))


def test_state_maps_take_the_latest_observation():
    st = np.full((3, 3, 10), 2, np.uint8)                     # everything occupied
    g = I.insert(st, [[7.5, 1.5, 1.5]], SENSOR, 1.0)
    assert list(_row(g)) == [1] * 7 + [2, 2, 2]


def test_repeated_scans_converge_to_the_clamps():
    g = UNKNOWN
    for _ in range(12):
        g = I.insert(g, [[7.5, 1.5, 1.5]], SENSOR, 1.0)
    assert np.all(_row(g)[:7] == f32(I.P_MIN)) and _row(g)[7] == f32(I.P_MAX)


def test_free_space_equals_the_brute_force_walk(orc):
    rng = np.random.default_rng(3)
    dims = (12, 9, 7)
    vs = 0.05
    for trial in range(20):
        sensor = rng.uniform([-0.1, -0.1, -0.1], [0.7, 0.5, 0.4])
        pts = rng.uniform([-0.1, -0.1, -0.1], [0.7, 0.5, 0.4], (25, 3)).astype(np.float32)
        hits, misses = I.scan_sets(pts, sensor, dims, vs)
        inv_s = f32(1.0 / float(f32(vs)))
        o = [f32(f32(sensor[a]) * inv_s) for a in range(3)]
        ref_hits, ref_free, skip = set(), set(), False
        for p in pts:
            idx = [int(math.floor(float(f32(f32(p[a]) * inv_s)))) for a in range(3)]
            if all(0 <= idx[a] < dims[a] for a in range(3)):
                ref_hits.add((idx[2] * dims[1] + idx[1]) * dims[0] + idx[0])
            d = [f32(f32(idx[a] + 0.5) - o[a]) for a in range(3)]
            if orc.min_tie_gap(dims, o, d) < 1e-6:
                skip = True
            ref_free.update(int(v) for v in orc.trace(dims, o, d, "brute"))
        if skip:
            continue
        assert hits == ref_hits, trial
        assert misses == ref_free - ref_hits, trial
