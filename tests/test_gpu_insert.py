"""Map update from depth scans on the GPU against the oracle (GPU required).

Bar: bit-exact maps (FP32 probabilities, uint8 and 2-bit states) after every
scan -- the update uses IEEE basic operations in one fixed order and the
walk is the FP32 reference walk, so nothing is left to rounding order.
"""

import math

import numpy as np
import pytest
import torch

import oracle
import paper_2503_22588_gb300 as nbt
from oracle import insert as I
from workload import sensor

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    nbt.build()
    oracle.build()


def small_scans(n_scans, seed, width=64, height=48):
    sc = sensor.tabletop_scene(seed, n_objects=25)
    poi = np.array([1.28, 1.28, 0.8])
    ps = sensor.scan_poses(poi, n_scans, seed)
    return [(p, sensor.depth_points(sc, p, width, height, math.radians(75), math.radians(65), 3.0, 0.003, seed + k))
            for k, p in enumerate(ps)]


def gpu_map(grid, vs, enc):
    return nbt.Map.from_grid(torch.from_numpy(grid).cuda(), vs, (0.0, 0.0, 0.0), enc)


@pytest.mark.parametrize("enc", ["f32", "u8", "u2"])
def test_scans_match_the_oracle_bit_for_bit(enc):
    n, vs = 64, 0.04                      # 2.56 m at 4 cm: scans reach past the map on every side
    grid = np.full((n, n, n), 0.5, np.float32) if enc == "f32" else np.zeros((n, n, n), np.uint8)
    m = gpu_map(grid, vs, enc)
    ref = grid
    for k, (pose, pts) in enumerate(small_scans(4, 7)):
        m.insert_points(torch.from_numpy(pts).cuda(), pose[:3])
        ref = I.insert(ref, pts, pose[:3], vs)
        got = m.download().cpu().numpy()
        if enc == "f32":
            assert np.array_equal(got.view(np.uint32), ref.view(np.uint32)), k
        else:
            assert np.array_equal(got, ref), k
        assert (ref != grid).sum() > 100
    m.close()


def test_range_limit_outside_points_and_non_finite_points():
    n, vs = 40, 0.05
    grid = np.full((n, n, n), 0.5, np.float32)
    rng = np.random.default_rng(1)
    pts = rng.uniform(-1.0, 3.0, (3000, 3)).astype(np.float32)      # many endpoints outside the 2 m map
    pts[::97] = np.nan
    pts[5] = [np.inf, 0.0, 0.0]
    pts[6] = [2.0 ** 22 * vs, 0.5, 0.5]
    s = (0.9, 1.1, 1.3)
    for mr in (0.0, 0.8):
        m = gpu_map(grid, vs, "f32")
        m.insert_points(torch.from_numpy(pts).cuda(), s, max_range=mr)
        want = I.insert(grid, pts, s, vs, max_range=mr)
        assert np.array_equal(m.download().cpu().numpy().view(np.uint32), want.view(np.uint32)), mr
        m.close()


def test_sensor_outside_the_map_and_shifted_origin():
    n, vs, org = 32, 0.05, (-0.4, 0.3, -0.2)
    grid = np.full((n, n, n), 0.5, np.float32)
    rng = np.random.default_rng(2)
    pts = (np.array(org) + rng.uniform(0.0, 1.6, (2000, 3))).astype(np.float32)
    s = (-1.5, 2.9, 0.4)                                             # outside the map box
    m = nbt.Map.from_grid(torch.from_numpy(grid).cuda(), vs, org, "f32")
    m.insert_points(torch.from_numpy(pts).cuda(), s)
    want = I.insert(grid, pts, s, vs, org)
    assert np.array_equal(m.download().cpu().numpy().view(np.uint32), want.view(np.uint32))
    m.close()


def test_repeated_scans_clamp_and_custom_probabilities():
    n, vs = 32, 0.05
    grid = np.full((n, n, n), 0.5, np.float32)
    (pose, pts), = small_scans(1, 3, 32, 24)
    pts = pts * np.float32(0.6)                                      # bring the scene into the 1.6 m map
    s = pose[:3] * 0.6
    m = gpu_map(grid, vs, "f32")
    ref = grid
    for k in range(10):                   # odd scans (the last one too) use the custom probabilities
        kw = dict(p_hit=0.9, p_miss=0.2, p_min=0.05, p_max=0.99) if k % 2 else {}
        m.insert_points(torch.from_numpy(pts).cuda(), s, **{"prob_hit": kw.get("p_hit", 0.7),
                                                            "prob_miss": kw.get("p_miss", 0.4),
                                                            "clamp_min": kw.get("p_min", 0.1192),
                                                            "clamp_max": kw.get("p_max", 0.971)})
        ref = I.insert(ref, pts, s, vs, **kw)
    assert np.array_equal(m.download().cpu().numpy().view(np.uint32), ref.view(np.uint32))
    assert (ref == np.float32(0.99)).any() and (ref == np.float32(0.05)).any()
    m.close()


def test_insert_then_ig_sees_the_update():
    """The derived gain table is rebuilt after an insert: IG on the updated map equals the oracle's."""
    n, vs = 48, 0.05
    grid = np.full((n, n, n), 0.5, np.float32)
    (pose, pts), = small_scans(1, 5, 48, 36)
    pts = pts * np.float32(0.9)
    m = gpu_map(grid, vs, "f32")
    cam = nbt.camera(16, 12, math.radians(60), math.radians(45), 1.0)
    prm = nbt.ig_params("entropy")
    poi = np.full(3, n * vs / 2)
    from workload import poses
    views = poses.shell_views(poi, 8, 0.5, 0.9, 1)
    before, _ = nbt.views_ig(m, torch.from_numpy(views).cuda(), cam, prm)
    m.insert_points(torch.from_numpy(pts).cuda(), pose[:3] * 0.9)
    after, _ = nbt.views_ig(m, torch.from_numpy(views).cuda(), cam, prm)
    ref = I.insert(grid, pts, pose[:3] * 0.9, vs)
    want, _ = oracle.views_ig(oracle.Map(ref, vs, (0, 0, 0)), views, oracle.camera(16, 12, math.radians(60),
                                                                                    math.radians(45), 1.0),
                              oracle.params("entropy"), "f32", 4)
    after = after.cpu().numpy().astype(np.float64)
    assert np.max(np.abs(after - want) / np.maximum(np.abs(want), 1e-30)) <= 1e-5
    assert not np.allclose(after, before.cpu().numpy())
    m.close()


def test_empty_scan_invalid_arguments_and_bricked_maps():
    from paper_2503_22588_gb300 import NbtError
    grid = np.full((16, 16, 16), 0.5, np.float32)
    m = gpu_map(grid, 0.05, "f32")
    m.insert_points(torch.zeros((0, 3), device="cuda"), (0.1, 0.1, 0.1))
    assert np.all(m.download().cpu().numpy() == 0.5)
    pts = torch.rand((10, 3), device="cuda")
    for kw in (dict(prob_hit=0.5), dict(prob_miss=0.5), dict(clamp_min=0.9, clamp_max=0.8),
               dict(max_range=float("inf"))):
        with pytest.raises(NbtError):
            m.insert_points(pts, (0.1, 0.1, 0.1), **kw)
    with pytest.raises(NbtError):
        m.insert_points(pts, (1e9, 0.1, 0.1))                         # sensor beyond 2^22 voxels
    m.close()
    b = nbt.Map.from_grid(torch.from_numpy(grid).cuda(), 0.05, (0, 0, 0), "f32", 8)
    with pytest.raises(NbtError):
        b.insert_points(pts, (0.1, 0.1, 0.1))
    assert np.array_equal(b.download().cpu().numpy(), grid)          # download works for bricked layouts
    b.close()


def test_fullsize_kinect_scan_into_256_map():
    """One 640 x 576 scan (the benchmark's size) into a 256^3 FP32 map: the whole map bit-exact."""
    sc = sensor.tabletop_scene(0)
    poi = np.array([1.28, 1.28, 0.8])
    pose = sensor.scan_poses(poi, 1, 0)[0]
    pts = sensor.depth_points(sc, pose, 640, 576, math.radians(75), math.radians(65), 3.86, 0.002, 1)
    grid = np.full((256, 256, 256), 0.5, np.float32)
    m = gpu_map(grid, 0.01, "f32")
    stats = torch.zeros(3, dtype=torch.int64, device="cuda")
    m.insert_points(torch.from_numpy(pts).cuda(), pose[:3], stats=stats)
    want = I.insert(grid, pts, pose[:3], 0.01)
    assert np.array_equal(m.download().cpu().numpy().view(np.uint32), want.view(np.uint32))
    hits, _ = I.scan_sets(pts, pose[:3], (256, 256, 256), 0.01)
    assert int(stats[0]) == len(hits) and int(stats[1]) >= len(hits) and int(stats[2]) > int(stats[1])
    m.close()
