"""Walks that skip uniform bricks, against the oracle (GPU required).

On linear maps with brick skipping on (the default; nbt_map_set_tuning), calls with many rays run
the tile kernel that replaces the walk through a uniform brick (8 to 64 voxels, all unknown or all
free; on probability maps, all gains exactly 1 or exactly 0) by per-axis crossing counts (the same
FP32 crossing parameters as the voxel-by-voxel walk).  Every case here has more than
466,944 rays per call, so that kernel runs, and the voxel steps and unknown counts of every view
must equal the oracle's exactly -- the FP32 gains of probability maps within 1e-5 relative -- with
skipping on and off: maps of every brick class, sides that are not multiples of 8, an origin off
the voxel grid, cameras inside and outside the map, both grid and range modes, all three metrics,
the map updated between calls (the summaries must be rebuilt), and trajectory IG.
"""

import numpy as np
import pytest
import torch

import oracle
import paper_2503_22588_gb300 as nbt
from workload import configs, poses, scenes

pytestmark = pytest.mark.gpu

THREADS = 16


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    nbt.build()
    oracle.build()


def run_case(grid, enc, pz, cam, origin=(0.0, 0.0, 0.0), voxel=0.01):
    """Both walks of the throughput kernel (skipping on and off) against the oracle, exactly."""
    assert len(pz) * cam.width * cam.height > 466944        # the throughput kernel's range
    m = nbt.Map.from_grid(torch.from_numpy(np.ascontiguousarray(grid)).cuda(), voxel, origin, enc)
    om = oracle.Map(np.ascontiguousarray(grid), voxel, origin)
    ocam = oracle.camera(cam.width, cam.height, cam.fov_h, cam.fov_v, cam.max_range,
                         ["corners", "centers"][cam.grid_mode], ["planar", "spherical"][cam.range_mode])
    rig, rst = oracle.views_ig(om, pz, ocam, oracle.params("count"), "f32", THREADS)
    for skip in (True, False):
        m.set_tuning(8, skip=skip)
        ig, st = nbt.views_ig(m, torch.from_numpy(pz).cuda(), cam, nbt.ig_params("count"))
        torch.cuda.synchronize()
        assert np.array_equal(st.cpu().numpy(), rst), skip
        assert np.array_equal(ig.cpu().numpy().astype(np.float64), rig), skip
    m.close()
    return rst


def shell(center, n, r0, r1, seed):
    return poses.shell_views(np.asarray(center, np.float64), n, r0, r1, seed)


@pytest.mark.parametrize("enc", ["u8", "u2"])
def test_boxes_spheres_half_unknown(enc):
    grid = scenes.boxes_spheres(96, 40, 3, half_unknown=True)
    pz = shell((0.48, 0.48, 0.48), 128, 0.3, 0.7, 1)
    cam = nbt.camera(64, 64, 1.0, 0.8, 1.0)
    run_case(grid, enc, pz, cam)


@pytest.mark.parametrize("enc,nx", [("u8", 101), ("u2", 101), ("u8", 96), ("u2", 96)])
def test_room_with_partial_bricks_and_an_offset_origin(enc, nx):
    """Sides nx x 77 x 90, origin off the grid, cameras inside and outside.  nx = 101: no side a
    multiple of 8 (summaries voxel by voxel); nx = 96: whole 8-voxel rows read as one word each,
    bricks cut short along y and z."""
    grid = scenes.room_states(128, 150, 0.4, seed=5)[:90, :77, :nx]
    origin = (-0.0123, 0.0377, 0.0049)
    c = np.array([0.5, 0.38, 0.45])
    pz = np.concatenate([shell(c, 64, 0.05, 0.3, 2), shell(c, 64, 0.6, 1.2, 3)])
    cam = nbt.camera(80, 56, 1.1, 0.9, 1.5)
    run_case(grid, enc, pz, cam, origin)


@pytest.mark.parametrize("fill", [0, 1])
def test_uniform_maps(fill):
    """All unknown (every voxel counts) or all free (none does): whole walks of macro steps."""
    grid = np.full((64, 72, 80), fill, np.uint8)
    pz = shell((0.4, 0.36, 0.32), 128, 0.1, 0.9, 4)
    cam = nbt.camera(64, 64, 1.0, 0.8, 1.2, "centers", "spherical")
    st = run_case(grid, "u2", pz, cam)
    assert st.sum() > 0


def test_occupied_shell_and_thin_walls():
    """Bricks that hold occupied voxels are never skipped: a closed shell of thin walls."""
    n = 96
    grid = np.zeros((n, n, n), np.uint8)
    grid[8:88, 8:88, 8:88] = 1
    grid[8:88, 8:88, 20] = 2
    grid[8:88, 47, 8:88] = 2
    grid[63, 8:88, 8:88] = 2
    grid[30:50, 30:50, 30:50] = 0
    pz = shell((0.48, 0.48, 0.48), 128, 0.2, 0.6, 6)
    cam = nbt.camera(64, 64, 1.2, 1.0, 1.0)
    run_case(grid, "u8", pz, cam)


def test_summaries_follow_uploads_and_inserts():
    """The brick summaries are derived data: rebuilt after an upload and after a depth-scan insert."""
    grid = scenes.room_states(96, 80, 0.4, seed=9)
    pz = shell((0.48, 0.48, 0.48), 128, 0.3, 0.7, 7)
    cam = nbt.camera(64, 64, 1.0, 0.8, 1.0)
    m = nbt.Map.from_grid(torch.from_numpy(grid).cuda(), 0.01, (0.0, 0.0, 0.0), "u2")
    m.set_tuning(8, skip=True)
    ptc = torch.from_numpy(pz).cuda()
    prm = nbt.ig_params("count")
    ocam = oracle.camera(64, 64, 1.0, 0.8, 1.0)
    for step in range(3):
        ig, st = nbt.views_ig(m, ptc, cam, prm)
        torch.cuda.synchronize()
        rig, rst = oracle.views_ig(oracle.Map(grid), pz, ocam, oracle.params("count"), "f32", THREADS)
        assert np.array_equal(st.cpu().numpy(), rst), step
        assert np.array_equal(ig.cpu().numpy().astype(np.float64), rig), step
        if step == 0:
            grid = grid.copy()
            grid[:, :, 40:56] = 0                            # a new unknown slab, uploaded
            m.upload(torch.from_numpy(grid).cuda())
        elif step == 1:
            pts = np.stack(np.meshgrid(np.linspace(0.1, 0.85, 60), np.linspace(0.1, 0.85, 60), [0.7]), -1)
            pts = pts.reshape(-1, 3).astype(np.float32)
            m.insert_points(torch.from_numpy(pts).cuda(), (0.48, 0.48, 0.1))
            grid = m.download().cpu().numpy()
    m.close()


def test_trajectories_on_a_state_map():
    w = configs.traj256(seed=2, n_traj=48, n=128, len_range=(5, 20))
    w.camera = configs.Camera(96, 72)
    m = nbt.Map.from_grid(torch.from_numpy(w.grid).cuda(), w.voxel_size, w.origin, "u2")
    m.set_tuning(8, skip=True)
    cam = nbt.camera(96, 72, w.camera.fov_h, w.camera.fov_v, 1.0)
    assert len(w.poses) * 96 * 72 > 466944
    pose_out = torch.empty(len(w.poses), dtype=torch.float32, device="cuda")
    tig = nbt.traj_ig(m, torch.from_numpy(w.poses).cuda(), torch.from_numpy(w.offsets).cuda(), cam,
                      nbt.ig_params("count"), pose_out=pose_out)
    torch.cuda.synchronize()
    om = oracle.Map(w.grid)
    rig, _ = oracle.traj_ig(om, w.poses, w.offsets, oracle.camera_of(w.camera), oracle.params("count"), "f32",
                            THREADS)
    pig, _ = oracle.views_ig(om, w.poses, oracle.camera_of(w.camera), oracle.params("count"), "f32", THREADS)
    assert np.array_equal(pose_out.cpu().numpy().astype(np.float64), pig)     # counts below 2^24: exact
    assert np.array_equal(tig.cpu().numpy(), rig.astype(np.float32))          # sums returned as FP32
    assert rig.max() > 2 ** 24                                                # (some exceed 2^24)
    m.close()


def test_pyramid_levels_and_their_boundaries():
    """Large uniform regions (bricks of 16, 32 and 64 voxels are uniform) next to mixed ones: free and
    unknown halves split off any brick boundary, an unknown block and a few occupied specks."""
    n = 160
    grid = np.ones((n, n, n), np.uint8)
    grid[:, :, 37:] = 0
    grid[70:133, 5:90, 90:150] = 1
    rng = np.random.default_rng(3)
    for _ in range(40):
        z, y, x = rng.integers(0, n, 3)
        grid[z, y, x] = 2
    pz = shell((0.8, 0.8, 0.8), 96, 0.3, 1.0, 8)
    cam = nbt.camera(80, 72, 1.0, 0.8, 1.6)
    run_case(grid, "u2", pz, cam, (0.003, -0.004, 0.0))


def run_f32_case(grid, pz, cam, prm_name, origin=(0.0, 0.0, 0.0), occ=0.7, free=0.3):
    """FP32 probability map: both walks against the FP64 oracle -- voxel steps exactly, IG within
    1e-5 relative (skipping adds a brick's unit gains at once, so per-ray FP32 sums round differently)."""
    assert len(pz) * cam.width * cam.height > 466944
    m = nbt.Map.from_grid(torch.from_numpy(np.ascontiguousarray(grid)).cuda(), 0.01, origin, "f32")
    om = oracle.Map(np.ascontiguousarray(grid), 0.01, origin)
    ocam = oracle.camera(cam.width, cam.height, cam.fov_h, cam.fov_v, cam.max_range)
    rig, rst = oracle.views_ig(om, pz, ocam, oracle.params(prm_name, occ, free), "f32", THREADS)
    for skip in (True, False):
        m.set_tuning(8, skip=skip)
        ig, st = nbt.views_ig(m, torch.from_numpy(pz).cuda(), cam, nbt.ig_params(prm_name, occ, free))
        torch.cuda.synchronize()
        assert np.array_equal(st.cpu().numpy(), rst), (prm_name, skip)
        rel = np.abs(ig.cpu().numpy().astype(np.float64) - rig) / np.maximum(np.abs(rig), 1e-30)
        assert rel.max() <= 1e-5, (prm_name, skip, rel.max())
    m.close()


@pytest.mark.parametrize("metric", ["entropy", "eq2", "count"])
def test_probability_tabletop_every_metric(metric):
    """The tabletop's unknown half and the unknown space under the table are uniform bricks of gain 1."""
    w = configs.prob256(seed=2, n_views=64, n=128, n_prims=60)
    cam = nbt.camera(96, 96, w.camera.fov_h, w.camera.fov_v, 1.0)
    run_f32_case(w.grid, w.poses, cam, metric)


def test_probability_summaries_follow_metric_thresholds_and_uploads():
    """Gains (and with them the brick summaries) are derived per metric and thresholds and after an
    upload: alternate them on one map and compare every call with the oracle."""
    w = configs.prob256(seed=3, n_views=64, n=96, n_prims=40)
    cam = nbt.camera(96, 96, w.camera.fov_h, w.camera.fov_v, 1.0)
    grid = w.grid.copy()
    m = nbt.Map.from_grid(torch.from_numpy(grid).cuda(), 0.01, (0.0, 0.0, 0.0), "f32")
    m.set_tuning(8, skip=True)
    ocam = oracle.camera(96, 96, w.camera.fov_h, w.camera.fov_v, 1.0)
    pt = torch.from_numpy(w.poses).cuda()
    for step, (metric, occ, free) in enumerate([("entropy", 0.7, 0.3), ("count", 0.7, 0.3), ("eq2", 0.6, 0.45),
                                                ("entropy", 0.7, 0.3), ("count", 0.7, 0.3)]):
        if step == 3:
            grid[:, :, 20:40] = 0.5                          # a new unknown slab, uploaded
            m.upload(torch.from_numpy(grid).cuda())
        ig, st = nbt.views_ig(m, pt, cam, nbt.ig_params(metric, occ, free))
        torch.cuda.synchronize()
        rig, rst = oracle.views_ig(oracle.Map(grid), w.poses, ocam, oracle.params(metric, occ, free), "f32",
                                   THREADS)
        assert np.array_equal(st.cpu().numpy(), rst), step
        rel = np.abs(ig.cpu().numpy().astype(np.float64) - rig) / np.maximum(np.abs(rig), 1e-30)
        assert rel.max() <= 1e-5, (step, rel.max())
    m.close()
