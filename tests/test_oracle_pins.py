"""Pins of the CPU oracle against things other than itself (no GPU).

Each test ties one part of the oracle to a fact fixed by the paper or by
mathematics: hand-worked cases, brute-force voxel enumeration on tiny maps,
closed-form voxel counts, invariants (occlusion, monotonicity, permutation),
and geometric identities of the endpoint grid (Section III).
"""

import json
import math
import os

import numpy as np
import pytest

from workload import poses as wposes
from workload import scenes

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "hand_cases.json")
TIE = 1e-6  # parameter gap below which exact and FP32 walks may order crossings differently


def lin(dims, xyz):
    x, y, z = xyz
    return (z * dims[1] + y) * dims[0] + x


def states_grid(dims, occupied=(), fill=0):
    g = np.full((dims[2], dims[1], dims[0]), fill, np.uint8)
    for x, y, z in occupied:
        g[z, y, x] = 2
    return g


def random_segments(rng, dims, n, inside_frac=0.5, max_len=None):
    """Generic random segments in voxel units: some start inside, some outside."""
    dims = np.asarray(dims, np.float64)
    max_len = max_len or 2.0 * dims.max()
    o = np.empty((n, 3))
    inside = rng.random(n) < inside_frac
    o[inside] = rng.random((inside.sum(), 3)) * dims
    o[~inside] = rng.uniform(-0.5, 1.5, size=((~inside).sum(), 3)) * dims
    dirs = rng.standard_normal((n, 3))
    dirs /= np.linalg.norm(dirs, axis=1, keepdims=True)
    length = rng.uniform(0.1, max_len, size=(n, 1))
    return o.astype(np.float32), (dirs * length).astype(np.float32)


# --------------------------------------------------------------------------
# Hand-worked cases
# --------------------------------------------------------------------------

def test_hand_cases_all_walks(orc):
    spec = json.load(open(GOLDEN))
    for case in spec["cases"]:
        dims = case["dims"]
        g = states_grid(dims, case["occupied"])
        m = orc.Map(g)
        o = np.array(case["o"], np.float32)
        d = np.array(case["d"], np.float32)
        full = [lin(dims, v) for v in case["full_sequence"]]
        occl = [lin(dims, v) for v in case["occluded_sequence"]]
        prm = orc.params("count")
        for walk in ("brute", "f64", "f32"):
            assert list(orc.trace(dims, o, d, walk)) == full, (case["name"], walk)
            assert list(orc.trace_occluded(m, o, d, prm, walk)) == occl, (case["name"], walk)
            ig, st = orc.segments_ig(m, o, d, prm, walk)
            assert ig[0] == case["count_ig"] and st[0] == case["steps"], (case["name"], walk)


def test_hand_tie_cases(orc):
    """Segments exactly through voxel edges and corners: the definition (brute force) keeps the
    voxels crossed over a positive length; the stepping walks take the tie-break x, then y, then z."""
    for case in json.load(open(GOLDEN))["tie_cases"]:
        dims = case["dims"]
        o = np.array(case["o"], np.float32)
        d = np.array(case["d"], np.float32)
        assert list(orc.trace(dims, o, d, "brute")) == [lin(dims, v) for v in case["definition_sequence"]], \
            case["name"]
        for walk in ("f64", "f32"):
            assert list(orc.trace(dims, o, d, walk)) == [lin(dims, v) for v in case["stepping_sequence"]], \
                (case["name"], walk)


def test_tie_gap_by_hand(orc):
    """The smallest parameter gap between crossings of different axes (or a crossing and a clip
    end): zero for segments through an edge or corner; 8/15 - 1/2 = 1/30 for the worked diagonal
    (x crossings at 1/6, 1/2, 5/6, the y crossing at 8/15, ends at 0 and 1)."""
    spec = json.load(open(GOLDEN))
    for case in spec["tie_cases"]:
        o = np.array(case["o"], np.float32)
        d = np.array(case["d"], np.float32)
        assert orc.min_tie_gap(case["dims"], o, d) == 0.0, case["name"]
    case = next(c for c in spec["cases"] if c["name"] == "diagonal_in_plane_hits_wall")
    gap = orc.min_tie_gap(case["dims"], np.array(case["o"], np.float32), np.array(case["d"], np.float32))
    assert abs(gap - 1.0 / 30.0) < 1e-7, gap


def test_segments_start_at_the_camera_in_voxel_units(orc):
    """A ray starts at the camera position p_P, in voxel units (p_P - origin) / s_Vox, and the central
    ray of an identity pose runs d_Cam along +z.  Dyadic values make both exact in FP32."""
    m = orc.Map(np.zeros((8, 8, 8), np.uint8), 0.25, (-1.0, 2.0, 0.5))
    pose = np.array([0.0, 3.0, 1.5, 1.0, 0.0, 0.0, 0.0], np.float32)
    o, d = orc.view_rays(m, orc.camera(3, 3, 1.0, 1.0, 0.5), pose)
    assert np.array_equal(o, np.tile(np.float32([4.0, 4.0, 4.0]), (9, 1)))
    assert np.array_equal(d[4], np.float32([0.0, 0.0, 2.0]))


def test_hand_case_eq2(orc):
    spec = json.load(open(GOLDEN))["eq2_case"]
    dims = spec["dims"]
    p = np.full((dims[2], dims[1], dims[0]), 0.5, np.float32)
    for key, val in spec["p"].items():
        x, y, z = map(int, key.split(","))
        p[z, y, x] = val
    m = orc.Map(p)
    o = np.array(spec["o"], np.float32)
    d = np.array(spec["d"], np.float32)
    ig, st = orc.segments_ig(m, o, d, orc.params("eq2"), "f64")
    assert abs(ig[0] - spec["ig"]) < 1e-7 and st[0] == spec["steps"]
    ig2, st2 = orc.segments_ig(m, o, d, orc.params("eq2", include_hit=False), "f64")
    assert abs(ig2[0] - spec["ig_without_hit"]) < 1e-7 and st2[0] == spec["steps"]


# --------------------------------------------------------------------------
# Walks against brute force, and FP32 against FP64
# --------------------------------------------------------------------------

@pytest.mark.parametrize("dims", [(16, 16, 16), (7, 5, 9), (1, 12, 3)])
def test_walks_match_brute_force(orc, dims):
    rng = np.random.default_rng(sum(dims))
    o, d = random_segments(rng, dims, 400)
    ties = 0
    for k in range(len(o)):
        if orc.min_tie_gap(dims, o[k], d[k]) < TIE:
            ties += 1
            continue
        ref = orc.trace(dims, o[k], d[k], "brute")
        assert np.array_equal(orc.trace(dims, o[k], d[k], "f64"), ref), k
        assert np.array_equal(orc.trace(dims, o[k], d[k], "f32"), ref), k
    assert ties < 0.05 * len(o)


def test_f32_walk_differs_from_f64_only_at_ties(orc):
    rng = np.random.default_rng(7)
    dims = (256, 256, 256)
    o, d = random_segments(rng, dims, 3000, max_len=160.0)
    mismatches = 0
    for k in range(len(o)):
        a = orc.trace(dims, o[k], d[k], "f32")
        b = orc.trace(dims, o[k], d[k], "f64")
        if not np.array_equal(a, b):
            mismatches += 1
            assert orc.min_tie_gap(dims, o[k], d[k]) < TIE, k
    assert mismatches <= 0.01 * len(o)


def test_walk_is_a_connected_monotone_path(orc):
    """Consecutive voxels differ by one step on one axis, always the ray's direction."""
    rng = np.random.default_rng(11)
    dims = np.array((32, 20, 24))
    o, d = random_segments(rng, dims, 300)
    for k in range(len(o)):
        seq = orc.trace(dims, o[k], d[k], "f32")
        if len(seq) < 2:
            continue
        x = seq % dims[0]
        y = (seq // dims[0]) % dims[1]
        z = seq // (dims[0] * dims[1])
        steps = np.stack([np.diff(x), np.diff(y), np.diff(z)], 1)
        assert np.all(np.abs(steps).sum(1) == 1)
        for a in range(3):
            assert np.all(steps[:, a] * np.sign(d[k][a]) >= 0)


# --------------------------------------------------------------------------
# Closed forms
# --------------------------------------------------------------------------

def test_all_unknown_count_closed_form(orc):
    """Inside the map, a generic segment crosses 1 + sum_a |floor(e_a) - floor(o_a)| voxels."""
    dims = (40, 40, 40)
    m = orc.Map(scenes.uniform_states((40, 40, 40), 0))
    rng = np.random.default_rng(3)
    o = rng.uniform(1.0, 39.0, (500, 3)).astype(np.float32)
    e = rng.uniform(1.0, 39.0, (500, 3)).astype(np.float32)
    d = (e.astype(np.float64) - o).astype(np.float32)
    prm = orc.params("count")
    for k in range(len(o)):
        if orc.min_tie_gap(dims, o[k], d[k]) < TIE:
            continue
        end = o[k].astype(np.float64) + d[k].astype(np.float64)
        expect = 1 + int(np.abs(np.floor(end) - np.floor(o[k].astype(np.float64))).sum())
        for walk in ("f64", "f32"):
            ig, st = orc.segments_ig(m, o[k], d[k], prm, walk)
            assert ig[0] == expect and st[0] == expect, (k, walk)


def test_all_free_and_all_occupied(orc):
    dims = (24, 24, 24)
    free = orc.Map(scenes.uniform_states((24, 24, 24), 1))
    occ = orc.Map(scenes.uniform_states((24, 24, 24), 2))
    rng = np.random.default_rng(5)
    o, d = random_segments(rng, dims, 300)
    prm = orc.params("count")
    for k in range(len(o)):
        full = orc.trace(dims, o[k], d[k], "f32")
        ig, st = orc.segments_ig(free, o[k], d[k], prm)
        assert ig[0] == 0 and st[0] == len(full)
        ig, st = orc.segments_ig(occ, o[k], d[k], prm)
        assert ig[0] == 0 and st[0] == min(1, len(full))


def test_all_occupied_eq2_gains_entry_voxel(orc):
    p = np.full((10, 10, 10), 0.9, np.float32)
    p[0, 0, 0] = 0.8
    m = orc.Map(p)
    o = np.array([0.3, 0.4, 0.6], np.float32)
    d = np.array([5.0, 3.0, 2.0], np.float32)
    ig, st = orc.segments_ig(m, o, d, orc.params("eq2"))
    assert st[0] == 1 and abs(ig[0] - (1.0 - float(np.float32(0.8)))) < 1e-12
    ig, st = orc.segments_ig(m, o, d, orc.params("eq2", include_hit=False))
    assert st[0] == 1 and ig[0] == 0.0


@pytest.mark.parametrize("axis,sign", [(0, 1), (0, -1), (1, 1), (1, -1), (2, 1), (2, -1)])
def test_axis_aligned_lengths(orc, axis, sign):
    dims = (20, 20, 20)
    o = np.array([10.37, 10.61, 10.23], np.float32)
    d = np.zeros(3, np.float32)
    d[axis] = sign * 6.5
    seq = orc.trace(dims, o, d, "f32")
    start = math.floor(o[axis])
    end = math.floor(o[axis] + d[axis])
    assert len(seq) == abs(end - start) + 1
    # beyond the map: clipped to the box
    d[axis] = sign * 100.0
    seq = orc.trace(dims, o, d, "f32")
    assert len(seq) == (20 - start if sign > 0 else start + 1)


def test_occlusion_wall_closed_form(orc):
    """Unknown space with an occupied wall at x = 17: the count is the unknown voxels before it."""
    g = scenes.uniform_states((32, 32, 32), 0)
    g[:, :, 17] = 2
    m = orc.Map(g)
    rng = np.random.default_rng(9)
    prm = orc.params("count")
    for _ in range(200):
        o = np.array([rng.uniform(0.0, 16.9), rng.uniform(8, 24), rng.uniform(8, 24)], np.float32)
        d = np.array([rng.uniform(20.0, 30.0), rng.uniform(-3, 3), rng.uniform(-3, 3)], np.float32)
        if orc.min_tie_gap((32, 32, 32), o, d) < TIE:
            continue
        # voxels crossed while x < 17: 1 + crossings of x planes 1..17 excluded + y/z planes before t17
        t17 = (17.0 - float(o[0])) / float(d[0])
        p17 = o.astype(np.float64) + t17 * d.astype(np.float64)
        # x planes floor(o_x)+1 .. 16 are crossed before the wall; y and z planes up to t17
        yz = np.abs(np.floor(p17[1:]) - np.floor(o[1:].astype(np.float64))).sum()
        before = 1 + (16 - math.floor(o[0])) + int(yz)
        ig, st = orc.segments_ig(m, o, d, prm)
        assert ig[0] == before and st[0] == before + 1


# --------------------------------------------------------------------------
# Invariants
# --------------------------------------------------------------------------

def test_ray_stops_at_first_occupied(orc):
    dims = (24, 24, 24)
    g = scenes.random_states((24, 24, 24), 0.3, 0.05, seed=1)
    m = orc.Map(g)
    flat = g.reshape(-1)
    rng = np.random.default_rng(2)
    o, d = random_segments(rng, dims, 300)
    prm = orc.params("count")
    for k in range(len(o)):
        full = orc.trace(dims, o[k], d[k], "f32")
        seq = orc.trace_occluded(m, o[k], d[k], prm, "f32")
        assert np.array_equal(seq, full[:len(seq)])
        assert np.all(flat[seq[:-1]] != 2) if len(seq) else True
        if len(seq) < len(full):
            assert flat[seq[-1]] == 2


@pytest.mark.parametrize("metric", ["count", "eq2", "entropy"])
def test_revealing_voxels_never_increases_ig(orc, metric):
    rng = np.random.default_rng(21)
    dims = (20, 20, 20)
    n = 20 * 20 * 20
    p = np.full(n, 0.5, np.float32)
    known = rng.random(n) < 0.4
    p[known] = rng.choice([0.05, 0.15, 0.85, 0.95], size=known.sum()).astype(np.float32)
    before = orc.Map(p.reshape(20, 20, 20).copy())
    p2 = p.copy()
    unk = np.flatnonzero(~known)
    reveal = rng.choice(unk, size=len(unk) // 3, replace=False)
    p2[reveal] = rng.choice([0.02, 0.2, 0.8, 0.98], size=len(reveal)).astype(np.float32)
    after = orc.Map(p2.reshape(20, 20, 20))
    o, d = random_segments(rng, dims, 400)
    prm = orc.params(metric)
    ig0, _ = orc.segments_ig(before, o, d, prm)
    ig1, _ = orc.segments_ig(after, o, d, prm)
    assert np.all(ig1 <= ig0 + 1e-12)
    assert np.any(ig1 < ig0)


def test_view_ig_is_permutation_invariant_sum_of_rays(orc):
    from workload import configs
    w = configs.exact64(seed=3, n_views=4)
    m = orc.Map(w.grid)
    cam = orc.camera_of(w.camera)
    prm = orc.params("count")
    ig, st = orc.views_ig(m, w.poses, cam, prm)
    for v in range(4):
        o, d = orc.view_rays(m, cam, w.poses[v])
        perm = np.random.default_rng(v).permutation(len(o))
        rig, rst = orc.segments_ig(m, o[perm], d[perm], prm)
        assert abs(rig.sum() - ig[v]) < 1e-9 and rst.sum() == st[v]
    igm, _ = orc.views_ig(m, w.poses, cam, orc.params("count", reduce="mean"))
    assert np.allclose(igm, ig / (64 * 48), rtol=1e-15)


def test_traj_ig_is_sum_over_csr_ranges(orc):
    from workload import configs
    w = configs.exact64(seed=1, n_views=12)
    m = orc.Map(w.grid)
    cam = orc.camera_of(w.camera)
    prm = orc.params("count")
    offsets = np.array([0, 3, 3, 8, 12], np.int32)  # includes an empty trajectory
    tig, tst = orc.traj_ig(m, w.poses, offsets, cam, prm, threads=2)
    vig, vst = orc.views_ig(m, w.poses, cam, prm)
    for t in range(4):
        assert tig[t] == vig[offsets[t]:offsets[t + 1]].sum()
        assert tst[t] == vst[offsets[t]:offsets[t + 1]].sum()


def test_threads_do_not_change_results(orc):
    from workload import configs
    w = configs.exact64(seed=2, n_views=10)
    m = orc.Map(w.grid)
    cam = orc.camera_of(w.camera)
    a = orc.views_ig(m, w.poses, cam, orc.params("count"), threads=1)
    b = orc.views_ig(m, w.poses, cam, orc.params("count"), threads=4)
    assert np.array_equal(a[0], b[0]) and np.array_equal(a[1], b[1])


# --------------------------------------------------------------------------
# Gains (Eq. 2 and the entropy / count variants)
# --------------------------------------------------------------------------

def test_long_sums_are_accumulated_in_fp64(orc):
    """Every voxel at P = 0.3 (unknown: not above 0.7, not below 0.3) gains H(0.3) and none occludes,
    so a perspective's entropy IG is its voxel steps x H(0.3) -- to FP64 precision, over ~10^5 terms."""
    p = float(np.float32(0.3))                          # the map stores P in FP32
    h = -p * math.log2(p) - (1.0 - p) * math.log2(1.0 - p)
    m = orc.Map(np.full((48, 48, 48), 0.3, np.float32), 0.01)
    pose = wposes.look_at_poses(np.array([[0.24, 0.24, 0.01]]), np.array([0.24, 0.24, 0.24]))
    ig, st = orc.views_ig(m, pose, orc.camera(40, 30, 1.0, 0.8, 0.5), orc.params("entropy"), "f32")
    assert st[0] > 50_000
    assert abs(ig[0] - st[0] * h) <= 1e-11 * st[0] * h, (ig[0], st[0] * h)


def test_entropy_values(orc):
    assert orc.entropy(0.5) == 1.0
    assert orc.entropy(0.0) == 0.0 and orc.entropy(1.0) == 0.0
    assert abs(orc.entropy(0.25) - (0.5 + 0.75 * math.log2(4.0 / 3.0))) < 1e-15
    for p in (0.01, 0.1, 0.3, 0.42):
        assert abs(orc.entropy(p) - orc.entropy(1.0 - p)) < 1e-15
        assert orc.entropy(p) < 1.0


def test_gain_table(orc):
    vals = np.array([0.9, 0.1, 0.5, 0.7, 0.3, 0.70000005], np.float32).reshape(1, 1, 6)
    m = orc.Map(vals)
    eq2 = orc.params("eq2")
    cnt = orc.params("count")
    ent = orc.params("entropy")
    g, occ = orc.voxel_gain(m, 0, eq2)
    assert occ and abs(g - (1.0 - float(vals[0, 0, 0]))) < 1e-15
    g, occ = orc.voxel_gain(m, 1, eq2)
    assert not occ and g == float(vals[0, 0, 1])
    g, occ = orc.voxel_gain(m, 2, eq2)
    assert not occ and g == 1.0
    assert orc.voxel_gain(m, 3, eq2) == (1.0, False)      # p = 0.7 is not > 0.7: unknown
    assert orc.voxel_gain(m, 4, eq2) == (1.0, False)      # p = 0.3 is not < 0.3: unknown
    assert orc.voxel_gain(m, 5, eq2)[1]                   # next float above 0.7: occupied
    assert orc.voxel_gain(m, 2, cnt) == (1.0, False)
    assert orc.voxel_gain(m, 1, cnt) == (0.0, False)
    assert orc.voxel_gain(m, 0, cnt) == (0.0, True)
    g, occ = orc.voxel_gain(m, 0, ent)
    assert occ and abs(g - orc.entropy(float(vals[0, 0, 0]))) < 1e-15
    st = orc.Map(np.array([0, 1, 2], np.uint8).reshape(1, 1, 3))
    assert orc.voxel_gain(st, 0, cnt) == (1.0, False)
    assert orc.voxel_gain(st, 1, cnt) == (0.0, False)
    assert orc.voxel_gain(st, 2, cnt) == (0.0, True)


# --------------------------------------------------------------------------
# Endpoint grid (Section III "Endpoint Calculation")
# --------------------------------------------------------------------------

def _rot(q):
    w, x, y, z = q
    return np.array([[1 - 2 * (y * y + z * z), 2 * (x * y - w * z), 2 * (x * z + w * y)],
                     [2 * (x * y + w * z), 1 - 2 * (x * x + z * z), 2 * (y * z - w * x)],
                     [2 * (x * z - w * y), 2 * (y * z + w * x), 1 - 2 * (x * x + y * y)]])


@pytest.mark.parametrize("grid_mode", ["corners", "centers"])
@pytest.mark.parametrize("range_mode", ["planar", "spherical"])
def test_endpoint_grid_geometry(orc, grid_mode, range_mode):
    W, H = 9, 7
    fh, fv, rng_m = math.radians(60.0), math.radians(45.0), 1.0
    cam = orc.camera(W, H, fh, fv, rng_m, grid_mode, range_mode)
    poi = np.array([0.32, 0.3, 0.35])
    pose = wposes.look_at_poses(np.array([[0.1, 0.8, 0.5]]), poi)[0]
    m = orc.Map(np.zeros((8, 8, 8), np.uint8))
    o, d = orc.view_rays(m, cam, pose)
    s = 0.01
    R = _rot(pose[3:].astype(np.float64))
    cam_dirs = (d.astype(np.float64) * s) @ R     # world -> camera frame
    dh, dv = rng_m * math.tan(fh / 2), rng_m * math.tan(fv / 2)
    # every ray starts at the camera position
    assert np.allclose(o * s, pose[:3], atol=1e-6)
    if range_mode == "planar":
        assert np.allclose(cam_dirs[:, 2], rng_m, atol=1e-5)       # far plane at d_Cam
        xs = cam_dirs[:, 0].reshape(H, W)
        ys = cam_dirs[:, 1].reshape(H, W)
        if grid_mode == "corners":                                  # border rays at +-d_h, +-d_v
            assert np.allclose(xs[:, 0], -dh, atol=1e-5) and np.allclose(xs[:, -1], dh, atol=1e-5)
            assert np.allclose(ys[0], -dv, atol=1e-5) and np.allclose(ys[-1], dv, atol=1e-5)
        else:
            assert np.allclose(xs[:, 0], -dh + dh / W, atol=1e-5)
            assert np.allclose(ys[-1], dv - dv / H, atol=1e-5)
        assert np.allclose(np.diff(xs, axis=1), np.diff(xs, axis=1)[0, 0], atol=1e-5)
    else:
        assert np.allclose(np.linalg.norm(cam_dirs, axis=1), rng_m, atol=1e-5)
    # the central ray (odd W, H) looks at the PoI
    c = cam_dirs[(H // 2) * W + W // 2]
    to_poi = (poi - pose[:3].astype(np.float64)) @ R
    assert np.allclose(c / np.linalg.norm(c), to_poi / np.linalg.norm(to_poi), atol=1e-6)


def test_perspectives_nearer_the_poi_gain_less(orc):
    """Section III: perspectives close to the PoI meet the object sooner and gain less."""
    g = scenes.uniform_states((64, 64, 64), 0)
    occ = np.zeros(g.shape, bool)
    scenes.fill_sphere(occ, (32.0, 32.0, 32.0), 6.0)
    g[occ] = 2
    m = orc.Map(g)
    cam = orc.camera(32, 24, math.radians(60.0), math.radians(45.0), 1.0)
    poi = np.array([0.32, 0.32, 0.32])
    near = wposes.sphere_views(poi, 16, 0.12)
    far = wposes.sphere_views(poi, 16, 0.30)
    ig_near, _ = orc.views_ig(m, near, cam, orc.params("count"))
    ig_far, _ = orc.views_ig(m, far, cam, orc.params("count"))
    assert np.all(ig_near < ig_far)
