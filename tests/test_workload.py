"""Pins of the seeded input generators (no GPU)."""

import math

import numpy as np

from workload import configs, poses, scenes, trajectories


def test_fibonacci_sphere_closed_form():
    """Centred Fibonacci lattice: heights 1 - (2k + 1)/n (symmetric about the equator), successive
    azimuths one golden angle apart, 2 pi / phi^2 = 137.50776405... degrees."""
    n = 257
    p = poses.fibonacci_directions(n)
    assert np.allclose(np.linalg.norm(p, axis=1), 1.0, atol=1e-14)
    assert np.allclose(np.diff(p[:, 2]), -2.0 / n, atol=1e-14)
    assert abs(p[0, 2] - (1.0 - 1.0 / n)) < 1e-14 and abs(p[-1, 2] + (1.0 - 1.0 / n)) < 1e-14
    assert abs(p[:, 2].mean()) < 1e-14
    phi = (1.0 + math.sqrt(5.0)) / 2.0
    golden = 2.0 * math.pi / phi ** 2
    assert abs(math.degrees(golden) - 137.50776405003785) < 1e-9
    az = np.arctan2(p[:, 1], p[:, 0])
    dphi = np.mod(np.diff(az), 2 * math.pi)
    assert np.allclose(dphi, golden, atol=1e-12)


def test_eq1_uniform_in_ball():
    """Eq. 1: |p|^3 / r_S^3 is uniform on [0, 1] and directions are isotropic."""
    x, xr = poses.muller_draws(200_000, seed=4)
    r_s = 1.0
    p = poses.muller_ball(x, xr, r_s)
    u = np.linalg.norm(p, axis=1) ** 3 / r_s ** 3
    assert np.all(u <= 1.0 + 1e-12)
    assert abs(u.mean() - 0.5) < 5e-3
    hist, _ = np.histogram(u, bins=10, range=(0, 1))
    assert np.all(np.abs(hist / len(u) - 0.1) < 5e-3)
    dirs = p / np.linalg.norm(p, axis=1, keepdims=True)
    assert np.all(np.abs(dirs.mean(axis=0)) < 1e-2)
    # without the cube root the radii would crowd the centre: mean |p|^3 would be 1/4
    p_wrong = r_s * xr[:, None] * x / np.linalg.norm(x, axis=1, keepdims=True)
    assert abs((np.linalg.norm(p_wrong, axis=1) ** 3).mean() - 0.25) < 5e-3


def test_look_at_orientation():
    rng = np.random.default_rng(0)
    poi = np.array([1.0, 2.0, 0.5])
    pos = poi + rng.standard_normal((100, 3))
    pos[0] = poi + np.array([0.0, 0.0, 0.7])  # vertical optical axis
    R = poses.look_at_rotation(pos, poi)
    for k in range(len(pos)):
        assert np.allclose(R[k].T @ R[k], np.eye(3), atol=1e-12)
        assert abs(np.linalg.det(R[k]) - 1.0) < 1e-12
        to = (poi - pos[k]) / np.linalg.norm(poi - pos[k])
        assert np.allclose(R[k][:, 2], to, atol=1e-12)
        if abs(to[2]) < 0.999:
            assert abs(R[k][2, 0]) < 1e-12          # image x axis horizontal
            assert R[k][2, 1] <= 1e-12              # image y axis points down
    q = poses.rotation_to_quaternion(R)
    assert np.allclose(np.linalg.norm(q, axis=1), 1.0)
    for k in range(len(pos)):
        w, x, y, z = q[k]
        Rq = np.array([[1 - 2 * (y * y + z * z), 2 * (x * y - w * z), 2 * (x * z + w * y)],
                       [2 * (x * y + w * z), 1 - 2 * (x * x + z * z), 2 * (y * z - w * x)],
                       [2 * (x * z - w * y), 2 * (y * z + w * x), 1 - 2 * (x * x + y * y)]])
        assert np.allclose(Rq, R[k], atol=1e-12)


def test_scene_generators_are_seeded_and_shaped():
    a = scenes.boxes_spheres(32, 10, seed=3)
    b = scenes.boxes_spheres(32, 10, seed=3)
    assert np.array_equal(a, b) and a.dtype == np.uint8 and a.shape == (32, 32, 32)
    assert np.all(a[:, :, 16:] == 0) and np.any(a[:, :, :16] == 2)
    p = scenes.tabletop_probabilities(64, 20, seed=1)
    assert p.dtype == np.float32 and np.all((p >= 0) & (p <= 1))
    assert np.any(p == 0.5) and np.any(p > 0.7) and np.any(p < 0.3)
    r = scenes.room_states(64, 40, 0.4, seed=2)
    assert abs((r == 0).mean() - 0.4) < 0.08


def test_probability_recipe():
    """Unknown voxels hold P = 0.5 exactly (overriding occupied), free P ~ Beta(2, 8) (mean 0.2,
    variance 16/1100) and occupied P ~ Beta(8, 2) (mean 0.8, same variance)."""
    occ = np.zeros((40, 40, 40), bool)
    occ[:, :, :12] = True
    unk = np.zeros_like(occ)
    unk[:, :, 30:] = True
    unk[:, :, 8:12] = True                       # overlaps the occupied slab
    p = scenes.probabilities_from_masks(occ, unk, seed=0).astype(np.float64)
    free = ~occ & ~unk
    occ_only = occ & ~unk
    assert np.all(p[unk] == 0.5)
    assert abs(p[free].mean() - 0.2) < 0.005 and abs(p[free].var() - 16 / 1100) < 1e-3
    assert abs(p[occ_only].mean() - 0.8) < 0.005 and abs(p[occ_only].var() - 16 / 1100) < 1e-3
    st = scenes.states_from_masks(occ, unk)
    assert np.all(st[unk] == 0) and np.all(st[occ_only] == 2) and np.all(st[free] == 1)


def test_box_fill_uses_voxel_centres():
    m = np.zeros((8, 8, 8), bool)
    scenes.fill_box(m, (1.4, 2.6, 0.0), (3.5, 4.4, 1.0))
    xs = np.unique(np.nonzero(m)[2])
    ys = np.unique(np.nonzero(m)[1])
    zs = np.unique(np.nonzero(m)[0])
    assert list(xs) == [1, 2] and list(ys) == [3] and list(zs) == [0]


def test_trajectories_csr():
    pois = np.array([[1.0, 1.0, 1.0]])
    p, off = trajectories.random_trajectories(pois, 20, seed=5, len_range=(5, 40))
    assert off[0] == 0 and off[-1] == len(p) and np.all(np.diff(off) >= 5) and np.all(np.diff(off) <= 40)
    assert p.dtype == np.float32 and p.shape[1] == 7
    assert np.allclose(np.linalg.norm(p[:, 3:], axis=1), 1.0, atol=1e-6)
    d = np.min(np.linalg.norm(p[:, None, :3] - pois[None], axis=2), axis=1)
    assert np.all(d > 0.3 - 1e-6) and np.all(d < 0.8 + 1e-6)


def test_catmull_rom_interpolates_its_inner_control_points():
    """A Catmull-Rom segment runs from p1 (t = 0) to p2 (t = 1) with tangents (p2 - p0)/2 and (p3 - p1)/2."""
    rng = np.random.default_rng(1)
    p0, p1, p2, p3 = rng.standard_normal((4, 3))
    t = np.array([0.0, 1.0, 1e-6, 1.0 - 1e-6])
    c = trajectories._catmull_rom(p0, p1, p2, p3, t)
    assert np.allclose(c[0], p1, atol=1e-14) and np.allclose(c[1], p2, atol=1e-14)
    assert np.allclose((c[2] - c[0]) / 1e-6, (p2 - p0) / 2, atol=1e-5)
    assert np.allclose((c[1] - c[3]) / 1e-6, (p3 - p1) / 2, atol=1e-5)
    b = trajectories._catmull_rom_batch(p0[None, None], p1[None, None], p2[None, None], p3[None, None],
                                        t[None, :, None])
    assert np.allclose(b[0], c, atol=1e-14)


def _axis_angles_deg(p, pois):
    """Angle between each pose's optical axis (R e_z) and the direction to its nearest PoI."""
    w, x, y, z = (p[:, 3 + k].astype(np.float64) for k in range(4))
    axis = np.stack([2 * (x * z + w * y), 2 * (y * z - w * x), 1 - 2 * (x * x + y * y)], axis=1)
    pos = p[:, :3].astype(np.float64)
    poi = pois[np.argmin(np.linalg.norm(pos[:, None] - pois[None], axis=2), axis=1)]
    to = (poi - pos) / np.linalg.norm(poi - pos, axis=1, keepdims=True)
    return np.degrees(np.arccos(np.clip(np.sum(axis * to, axis=1), -1.0, 1.0)))


def test_trajectory_orientations_look_at_the_poi_within_the_jitter():
    pois = np.array([[1.0, 1.0, 1.0]])
    p, _ = trajectories.random_trajectories(pois, 30, seed=2, jitter_deg=3.0)
    a = _axis_angles_deg(p, pois)
    assert a.max() <= 3.0 + 1e-3 and a.max() > 1.0
    q, _ = trajectories.horizon_trajectories(pois[0], 50, 11, seed=3, jitter_deg=10.0)
    b = _axis_angles_deg(q, pois)
    assert b.max() <= 10.0 + 1e-3 and b.max() > 5.0


def test_workload_presets_small():
    w = configs.exact64()
    assert w.grid.shape == (64, 64, 64) and w.poses.shape == (64, 7) and w.rays_per_pose == 3072
    d = np.linalg.norm(w.poses[:, :3] - w.pois[0], axis=1)
    assert np.allclose(d, 0.5, atol=1e-6)


def test_depth_scan_points_lie_on_the_scene_and_in_range():
    import math
    from workload import sensor
    sc = sensor.tabletop_scene(2, n_objects=10)
    poi = np.array([1.28, 1.28, 0.8])
    pose = sensor.scan_poses(poi, 1, 4)[0]
    pts = sensor.depth_points(sc, pose, 48, 36, math.radians(75), math.radians(65), 3.0).astype(np.float64)
    assert len(pts) > 1000
    o = pose[:3].astype(np.float64)
    assert np.all(np.linalg.norm(pts - o, axis=1) <= 3.0 + 1e-5)
    # every point is on the floor, on a box face or on a sphere (float32 rounding aside)
    tol = 2e-5
    on = np.abs(pts[:, 2] - sc.floor_z) < tol
    for lo, hi in sc.boxes:
        inside = np.all((pts >= lo - tol) & (pts <= hi + tol), axis=1)
        face = np.any((np.abs(pts - lo) < tol) | (np.abs(pts - hi) < tol), axis=1)
        on |= inside & face
    for cx, cy, cz, r in sc.spheres:
        on |= np.abs(np.linalg.norm(pts - [cx, cy, cz], axis=1) - r) < tol
    assert on.all()
    # points are in front of the camera, inside its field of view
    w, x, y, z = pose[3:].astype(np.float64)
    axis = np.array([2 * (x * z + w * y), 2 * (y * z - w * x), 1 - 2 * (x * x + y * y)])
    v = (pts - o) / np.linalg.norm(pts - o, axis=1, keepdims=True)
    assert np.all(v @ axis > math.cos(math.radians(55)))


def test_horizon_trajectories_shape_and_radii():
    from workload import trajectories
    poi = np.array([0.5, 0.4, 0.3])
    p, off = trajectories.horizon_trajectories(poi, 20, 31, 0, r_min=0.3, r_max=0.8, jitter_deg=10.0)
    assert p.shape == (620, 7) and off[0] == 0 and off[-1] == 620 and np.all(np.diff(off) == 31)
    r = np.linalg.norm(p[:, :3] - poi, axis=1)
    assert r.min() >= 0.3 - 1e-5 and r.max() <= 0.8 + 1e-5
    assert np.allclose(np.linalg.norm(p[:, 3:], axis=1), 1.0, atol=1e-6)
