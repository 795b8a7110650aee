"""Parity of the CUDA path with the CPU oracle (GPU required).

Bars: ray segments and voxel sequences bit-exact with the oracle's FP32
reference walk; voxel-step counts exact; unknown-voxel counts exact;
floating-point IG within a relative 1e-5 of the FP64 oracle, both along the
FP32 reference walk and along the exact FP64 walk.
"""

import math
import os

import numpy as np
import pytest
import torch

import oracle
import paper_2503_22588_gb300 as nbt
from gpu_util import RTOL, gpu_camera, gpu_map, oracle_camera, oracle_map, rel_err, views_gpu
from workload import configs, poses, scenes

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    nbt.build()
    oracle.build()


def _segments(rng, dims, n, max_len):
    dims = np.asarray(dims, np.float64)
    o = np.where(rng.random((n, 1)) < 0.5, rng.random((n, 3)) * dims, rng.uniform(-0.5, 1.5, (n, 3)) * dims)
    v = rng.standard_normal((n, 3))
    v /= np.linalg.norm(v, axis=1, keepdims=True)
    return o.astype(np.float32), (v * rng.uniform(0.1, max_len, (n, 1))).astype(np.float32)


def _edge_segments(dims):
    nx, ny, nz = dims
    rows = [
        ([0.5, 0.5, 0.5], [nx + 5.0, 0.0, 0.0]),            # axis-aligned, through the whole map
        ([nx - 0.5, 1.25, 1.75], [-(nx + 3.0), 0.0, 0.0]),  # axis-aligned, negative
        ([1.3, 1.7, 0.2], [0.0, 0.0, nz * 2.0]),             # along z
        ([2.0, 2.0, 2.0], [3.0, 3.0, 3.0]),                  # starts on a corner, exact diagonal
        ([0.0, 0.0, 0.0], [1.0, 0.0, 0.0]),                  # starts on the min corner
        ([1.5, 1.5, 1.5], [0.0, 0.0, 0.0]),                  # zero length
        ([-1.0, -1.0, -1.0], [-2.0, -3.0, -1.0]),            # outside, pointing away
        ([-5.0, 1.5, 1.5], [nx + 10.0, 0.0, 0.0]),           # enters through the x = 0 face
        ([1.5, float(ny), 1.5], [1.0, 0.0, 0.0]),            # on the y = N face (outside)
        ([1.5, 1.0, 1.5], [2.0, 0.0, 0.3]),                  # in the y = 1 plane
        ([float("nan"), 1.0, 1.0], [1.0, 1.0, 1.0]),         # NaN start
        ([1.0, 1.0, 1.0], [float("inf"), 0.0, 0.0]),         # infinite displacement
        ([nx / 2.0, ny / 2.0, nz / 2.0], [1e-30, 1e-30, 1e-30]),  # tiny displacement
        ([0.5, 0.5, 0.5], [3e6, 2e6, 1e6]),                  # huge segment
    ]
    o = np.array([r[0] for r in rows], np.float32)
    d = np.array([r[1] for r in rows], np.float32)
    return o, d


@pytest.mark.parametrize("grid_mode", ["corners", "centers"])
@pytest.mark.parametrize("range_mode", ["planar", "spherical"])
@pytest.mark.parametrize("wh", [(64, 48), (33, 9), (1, 1), (7, 1)])
def test_view_segments_bitexact(grid_mode, range_mode, wh):
    w = configs.exact64(seed=1, n_views=5)
    cam = configs.Camera(wh[0], wh[1], grid_mode=grid_mode, range_mode=range_mode)
    gm = gpu_map(w)
    o, d = nbt.view_segments(gm, torch.from_numpy(w.poses).cuda(), gpu_camera(cam))
    o = o.cpu().numpy()
    d = d.cpu().numpy()
    om = oracle_map(w)
    n = wh[0] * wh[1]
    for v in range(len(w.poses)):
        ro, rd = oracle.view_rays(om, oracle_camera(cam), w.poses[v])
        assert np.array_equal(o[v * n:(v + 1) * n].view(np.uint32), ro.view(np.uint32))
        assert np.array_equal(d[v * n:(v + 1) * n].view(np.uint32), rd.view(np.uint32))


@pytest.mark.parametrize("dims", [(16, 16, 16), (37, 20, 50), (256, 256, 256), (1, 1, 1), (5, 64, 3)])
@pytest.mark.parametrize("brick", [1, 4, 8])
def test_trace_segments_bitexact(dims, brick):
    rng = np.random.default_rng(dims[0] * 7 + brick)
    o, d = _segments(rng, dims, 3000, max_len=1.5 * max(dims))
    eo, ed = _edge_segments(dims)
    o = np.concatenate([o, eo])
    d = np.concatenate([d, ed])
    grid = np.zeros(dims[::-1], np.uint8)
    gm = nbt.Map.from_grid(torch.from_numpy(grid).cuda(), 0.01, (0.0, 0.0, 0.0), "u8", brick)
    idx, cnt = nbt.trace_segments(gm, torch.from_numpy(o).cuda(), torch.from_numpy(d).cuda())
    idx = idx.cpu().numpy()
    cnt = cnt.cpu().numpy()
    for k in range(len(o)):
        ref = oracle.trace(dims, o[k], d[k], "f32")
        assert cnt[k] == len(ref), k
        assert np.array_equal(idx[k, :cnt[k]], ref), k


def test_largest_map_walks_bit_exact():
    """The largest accepted map: 2048 x 2048 x 511 one-byte states, 2,143,289,344 voxels, just under
    the 2^31-element limit, so linear voxel indices reach the top of the int32 range."""
    dims = (2048, 2048, 511)
    with pytest.raises(nbt.NbtError):
        nbt.Map(2049, 4, 4, 0.01)                      # a side above 2048
    with pytest.raises(nbt.NbtError):
        nbt.Map(2048, 2048, 512, 0.01, brick=1)        # exactly 2^31 elements
    with pytest.raises(nbt.NbtError):
        nbt.Map(*dims, 0.01, brick=8)                  # 8^3 bricks pad it to 2^31 elements
    grid = torch.zeros(dims[::-1], dtype=torch.uint8, device="cuda")   # all unknown
    gm = nbt.Map.from_grid(grid, 0.01, (0.0, 0.0, 0.0), "u8", 1)
    del grid
    rng = np.random.default_rng(2048)
    o, d = _segments(rng, dims, 300, max_len=3000.0)
    eo = np.array([[0.5, 0.5, 0.5], [2047.5, 2047.5, 510.5], [2047.9, 0.1, 510.9]], np.float32)
    ed = np.array([[2047.0, 2047.0, 510.0], [-2047.0, -2047.0, -510.0], [-2047.0, 2047.0, -510.0]], np.float32)
    o = np.concatenate([o, eo])
    d = np.concatenate([d, ed])
    idx, cnt = nbt.trace_segments(gm, torch.from_numpy(o).cuda(), torch.from_numpy(d).cuda())
    idx = idx.cpu().numpy()
    cnt = cnt.cpu().numpy()
    assert idx.max() == 2048 * 2048 * 511 - 1                # the last voxel is reached
    for k in range(len(o)):
        ref = oracle.trace(dims, o[k], d[k], "f32")
        assert cnt[k] == len(ref), k
        assert np.array_equal(idx[k, :cnt[k]], ref), k
    # whole perspectives: 48 views of 120 x 90 rays are more rays than two per resident thread, so
    # they take the main tile kernel; on an all-unknown map the count IG of a view is its voxel steps
    # (below 2^24 per view, so exact in FP32)
    xy = [(1.0 + 3.0 * a, 1.0 + 0.75 * b) for a in range(2) for b in range(24)]
    pose = np.array([[x, y, 0.3, 1.0, 0.0, 0.0, 0.0] if k % 2 == 0 else      # looking up the z axis
                     [x + 12.0, y + 0.5, 4.8, 0.0, 1.0, 0.0, 0.0]              # from the top, looking down
                     for k, (x, y) in enumerate(xy)], np.float32)
    cam = configs.Camera(120, 90, max_range=30.0)
    ig, st = views_gpu(gm, pose, gpu_camera(cam), nbt.ig_params("count"))
    om = oracle.Map(np.zeros(dims[::-1], np.uint8), 0.01, (0.0, 0.0, 0.0))
    ig_o, st_o = oracle.views_ig(om, pose, oracle_camera(cam), oracle.params("count"), "f32",
                                 threads=os.cpu_count() or 1)
    assert np.array_equal(st, st_o)
    assert np.array_equal(ig, ig_o) and np.array_equal(ig, st.astype(np.float64))
    assert st.min() > 100 * 120 * 90 and st.max() < 2 ** 24


@pytest.mark.parametrize("encoding", ["u8", "u2"])
@pytest.mark.parametrize("brick", [1, 4, 8])
def test_trace_views_occluded_bitexact(encoding, brick):
    w = configs.exact64(seed=4, n_views=6)
    gm = gpu_map(w, brick, encoding)
    cam = gpu_camera(w.camera)
    o, d = nbt.view_segments(gm, torch.from_numpy(w.poses).cuda(), cam)
    prm = nbt.ig_params("count")
    idx, cnt = nbt.trace_segments(gm, o, d, prm)
    idx = idx.cpu().numpy()
    cnt = cnt.cpu().numpy()
    o = o.cpu().numpy()
    d = d.cpu().numpy()
    om = oracle_map(w)
    op = oracle.params("count")
    for k in range(len(o)):
        ref = oracle.trace_occluded(om, o[k], d[k], op, "f32")
        assert cnt[k] == len(ref) and np.array_equal(idx[k, :cnt[k]], ref), k


@pytest.mark.parametrize("seed", [0, 1, 2])
@pytest.mark.parametrize("encoding,brick", [("u8", 1), ("u8", 8), ("u8", 4), ("u2", 1), ("u2", 8), ("u2", 4)])
def test_views_ig_count_exact(seed, encoding, brick):
    """64^3 states, 64 views, 64 x 48 rays: unknown counts and steps equal the oracle's exactly."""
    w = configs.exact64(seed=seed)
    gm = gpu_map(w, brick, encoding)
    ig, st = views_gpu(gm, w.poses, gpu_camera(w.camera), nbt.ig_params("count"))
    rig, rst = oracle.views_ig(oracle_map(w), w.poses, oracle_camera(w.camera), oracle.params("count"), "f32", 8)
    assert np.array_equal(st, rst)
    assert np.array_equal(ig, rig)
    xig, _ = oracle.views_ig(oracle_map(w), w.poses, oracle_camera(w.camera), oracle.params("count"), "f64", 8)
    assert np.all(rel_err(ig, xig) <= RTOL)


@pytest.mark.parametrize("metric", ["entropy", "eq2", "count"])
@pytest.mark.parametrize("brick", [1, 8, 4])
def test_views_ig_probability_map(metric, brick):
    """Reduced tabletop (96^3 FP32), 24 views of 80 x 60 rays."""
    w = configs.prob256(seed=3, n_views=24, n=96, n_prims=40)
    w.camera = configs.Camera(80, 60)
    gm = gpu_map(w, brick)
    ig, st = views_gpu(gm, w.poses, gpu_camera(w.camera), nbt.ig_params(metric))
    om = oracle_map(w)
    rig, rst = oracle.views_ig(om, w.poses, oracle_camera(w.camera), oracle.params(metric), "f32", 8)
    assert np.array_equal(st, rst)
    assert np.all(rel_err(ig, rig) <= RTOL), rel_err(ig, rig).max()
    xig, xst = oracle.views_ig(om, w.poses, oracle_camera(w.camera), oracle.params(metric), "f64", 8)
    assert np.all(rel_err(ig, xig) <= RTOL), rel_err(ig, xig).max()
    assert np.all(np.abs(st - xst) <= 0.001 * xst + 2)


def test_views_ig_mean_and_include_hit():
    w = configs.prob256(seed=5, n_views=8, n=64, n_prims=20)
    w.camera = configs.Camera(40, 30)
    gm = gpu_map(w)
    om = oracle_map(w)
    for prm_kw in ({"reduce": "mean"}, {"include_hit": False}, {"include_hit": False, "reduce": "mean"},
                   {"occ_threshold": 0.6, "free_threshold": 0.35}):
        ig, st = views_gpu(gm, w.poses, gpu_camera(w.camera), nbt.ig_params("eq2", **prm_kw))
        rig, rst = oracle.views_ig(om, w.poses, oracle_camera(w.camera), oracle.params("eq2", **prm_kw), "f32", 4)
        assert np.array_equal(st, rst), prm_kw
        assert np.all(rel_err(ig, rig) <= RTOL), prm_kw


@pytest.mark.parametrize("wh", [(33, 9), (1, 1), (31, 7), (200, 3)])
def test_views_ig_ragged_tiles(wh):
    w = configs.exact64(seed=6, n_views=9)
    cam = configs.Camera(*wh)
    gm = gpu_map(w)
    ig, st = views_gpu(gm, w.poses, gpu_camera(cam), nbt.ig_params("count"))
    rig, rst = oracle.views_ig(oracle_map(w), w.poses, oracle_camera(cam), oracle.params("count"), "f32", 4)
    assert np.array_equal(st, rst) and np.array_equal(ig, rig)


def test_views_ig_degenerate_maps_and_poses():
    # 1 x 1 x 1 map; non-cubic map; cameras outside looking away; empty view list
    for dims in ((1, 1, 1), (37, 20, 50)):
        grid = scenes.random_states(dims[::-1], 0.4, 0.1, seed=3)
        w = configs.Workload("t", 0, "u8", "count", configs.Camera(16, 12), grid, None, None)
        poi = np.array(dims, np.float64) * 0.005
        pos = poi + np.array([[0.3, 0.0, 0.0], [0.0, -0.25, 0.1], [0.0, 0.0, 0.4], [0.01, 0.02, 0.03]])
        p = poses.look_at_poses(pos, poi)
        away = poses.look_at_poses(poi + np.array([[0.5, 0.5, 0.5]]), poi + np.array([1.0, 1.0, 1.0]))
        w.poses = np.concatenate([p, away])
        gm = gpu_map(w)
        ig, st = views_gpu(gm, w.poses, gpu_camera(w.camera), nbt.ig_params("count"))
        rig, rst = oracle.views_ig(oracle_map(w), w.poses, oracle_camera(w.camera), oracle.params("count"))
        assert np.array_equal(st, rst) and np.array_equal(ig, rig)
        assert ig[-1] == 0 and st[-1] == 0
    out, steps = nbt.views_ig(gm, torch.zeros((0, 7), dtype=torch.float32, device="cuda"), gpu_camera(w.camera),
                              nbt.ig_params("count"))
    assert out.numel() == 0


@pytest.mark.parametrize("encoding,metric", [("u8", "count"), ("u2", "count"), ("f32", "entropy"), ("f32", "eq2")])
def test_latency_and_throughput_kernels_agree(encoding, metric):
    """The call size picks the kernel -- many rays: rolling prefetch; fewer: walk-ahead; a few
    thousand: rays split over 8 or 16 lanes.  Steps and counts are identical; FP32 gains are
    identical except that the split kernel sums a ray lane part by lane part (<= 1e-6)."""
    w = configs.exact64(seed=5, n_views=512)
    grid = w.grid
    if encoding == "f32":
        grid = scenes.probabilities_from_masks(grid == 2, grid == 0, 5)
    gm = nbt.Map.from_grid(torch.from_numpy(np.ascontiguousarray(grid)).cuda(), w.voxel_size, w.origin, encoding)
    cam, prm = gpu_camera(w.camera), nbt.ig_params(metric)
    p = torch.from_numpy(w.poses).cuda()

    def batched(k):
        parts = [nbt.views_ig(gm, p[i:i + k], cam, prm) for i in range(0, 512, k)]
        return torch.cat([a for a, _ in parts]), torch.cat([b for _, b in parts])

    big_ig, big_st = nbt.views_ig(gm, p, cam, prm)     # 1.57M rays: rolling prefetch
    mid_ig, mid_st = batched(32)                        # 98k rays: walk-ahead
    sm_ig, sm_st = batched(4)                           # 12k rays: 8 lanes per ray
    one_ig, one_st = batched(1)                         # 3k rays: 16 lanes per ray
    torch.cuda.synchronize()
    for st in (mid_st, sm_st, one_st):
        assert torch.equal(big_st, st)
    assert torch.equal(big_ig, mid_ig)
    for ig in (sm_ig, one_ig):
        if metric == "count":
            assert torch.equal(big_ig, ig)
        else:
            assert rel_err(ig.cpu().numpy(), big_ig.cpu().numpy().astype(np.float64)).max() <= 1e-6
    rig, rst = oracle.views_ig(oracle.Map(grid, w.voxel_size, w.origin), w.poses[:64], oracle_camera(w.camera),
                               oracle.params(metric), "f32", 8)
    for ig, st in ((big_ig, big_st), (one_ig, one_st)):
        assert np.array_equal(st.cpu().numpy()[:64], rst)
        assert rel_err(ig.cpu().numpy()[:64], rig).max() <= RTOL
    gm.close()


def test_closed_forms_on_gpu():
    """All-free map: IG 0; all-occupied: one step per ray that meets the map."""
    cam = configs.Camera(24, 18)
    poi = np.array([0.16, 0.16, 0.16])
    p = poses.sphere_views(poi, 10, 0.1)  # inside the 32^3 map
    for state, expect_steps in ((1, None), (2, 24 * 18)):
        grid = scenes.uniform_states((32, 32, 32), state)
        gm = nbt.Map.from_grid(torch.from_numpy(grid).cuda(), 0.01)
        ig, st = views_gpu(gm, p, gpu_camera(cam), nbt.ig_params("count"))
        assert np.all(ig == 0)
        if expect_steps:
            assert np.all(st == expect_steps)


def test_traj_ig_matches_oracle():
    w = configs.traj256(seed=2, n_traj=24, n=96, len_range=(1, 9))
    w.camera = configs.Camera(48, 36)
    gm = gpu_map(w)
    off = torch.from_numpy(w.offsets).cuda()
    pz = torch.from_numpy(w.poses).cuda()
    pose_out = torch.empty(len(w.poses), dtype=torch.float32, device="cuda")
    tig = nbt.traj_ig(gm, pz, off, gpu_camera(w.camera), nbt.ig_params("count"), pose_out=pose_out)
    torch.cuda.synchronize()
    rig, _ = oracle.traj_ig(oracle_map(w), w.poses, w.offsets, oracle_camera(w.camera), oracle.params("count"),
                            "f32", 8)
    assert np.array_equal(tig.cpu().numpy().astype(np.float64), rig)
    vig, _ = oracle.views_ig(oracle_map(w), w.poses, oracle_camera(w.camera), oracle.params("count"), "f32", 8)
    assert np.array_equal(pose_out.cpu().numpy().astype(np.float64), vig)


def test_traj_ig_empty_and_uneven():
    w = configs.exact64(seed=8, n_views=10)
    gm = gpu_map(w)
    offsets = np.array([0, 0, 4, 4, 5, 10, 10], np.int32)
    tig = nbt.traj_ig(gm, torch.from_numpy(w.poses).cuda(), torch.from_numpy(offsets).cuda(),
                      gpu_camera(w.camera), nbt.ig_params("count", reduce="mean"))
    rig, _ = oracle.traj_ig(oracle_map(w), w.poses, offsets, oracle_camera(w.camera),
                            oracle.params("count", reduce="mean"))
    assert np.all(rel_err(tig.cpu().numpy(), rig) <= 1e-6)
    assert tig[0].item() == 0 and tig[2].item() == 0 and tig[5].item() == 0


def test_deterministic_results():
    w = configs.prob256(seed=1, n_views=32, n=64, n_prims=20)
    w.camera = configs.Camera(64, 48)
    gm = gpu_map(w)
    a = views_gpu(gm, w.poses, gpu_camera(w.camera), nbt.ig_params("entropy"))
    b = views_gpu(gm, w.poses, gpu_camera(w.camera), nbt.ig_params("entropy"))
    assert np.array_equal(a[0], b[0]) and np.array_equal(a[1], b[1])


def test_invalid_arguments_are_rejected():
    w = configs.exact64(seed=0, n_views=2)
    gm = gpu_map(w)
    p = torch.from_numpy(w.poses).cuda()
    with pytest.raises(nbt.NbtError) as e:
        nbt.views_ig(gm, p, gpu_camera(w.camera), nbt.ig_params("entropy"))   # entropy on a state map
    assert e.value.status == -5
    with pytest.raises(nbt.NbtError) as e:
        nbt.views_ig(gm, p, nbt.camera(0, 4, 1.0, 1.0, 1.0), nbt.ig_params("count"))
    assert e.value.status == -1
    with pytest.raises(nbt.NbtError) as e:
        nbt.views_ig(gm, p, nbt.camera(8, 4, 4.0, 1.0, 1.0), nbt.ig_params("count"))  # fov >= pi
    assert e.value.status == -1
    small = torch.empty(8, dtype=torch.uint8, device="cuda")
    with pytest.raises(nbt.NbtError) as e:
        nbt.views_ig(gm, p, gpu_camera(w.camera), nbt.ig_params("count"), ws=small)
    assert e.value.status == -6
    with pytest.raises(nbt.NbtError):
        nbt.Map(0, 4, 4, 0.01)
    with pytest.raises(nbt.NbtError):
        nbt.Map(4, 4, 4, 0.01, brick=5)
    with pytest.raises(nbt.NbtError):
        nbt.Map(4, 4, 4, -1.0)
    with pytest.raises(TypeError):
        gm.upload(np.zeros((64, 64, 64), np.float32))


def test_host_upload_matches_device_upload():
    w = configs.prob256(seed=2, n_views=6, n=64, n_prims=10)
    w.camera = configs.Camera(32, 24)
    a = nbt.Map.from_grid(w.grid, w.voxel_size)                       # host numpy source
    b = nbt.Map.from_grid(torch.from_numpy(w.grid).cuda(), w.voxel_size)  # device source
    ra = views_gpu(a, w.poses, gpu_camera(w.camera), nbt.ig_params("entropy"))
    rb = views_gpu(b, w.poses, gpu_camera(w.camera), nbt.ig_params("entropy"))
    assert np.array_equal(ra[0], rb[0]) and np.array_equal(ra[1], rb[1])
    # re-upload invalidates the derived gains
    g2 = w.grid.copy()
    g2[:, :, :32] = 0.5
    a.upload(g2)
    rc = views_gpu(a, w.poses, gpu_camera(w.camera), nbt.ig_params("entropy"))
    rig, _ = oracle.views_ig(oracle.Map(g2), w.poses, oracle_camera(w.camera), oracle.params("entropy"))
    assert np.all(rel_err(rc[0], rig) <= RTOL)


@pytest.mark.parametrize("brick", [1, 4, 8])
def test_odd_dims_two_bit_upload_and_walk(brick):
    """Non-multiple-of-4 dims: 2-bit bytes straddle rows in the linear layout."""
    dims = (37, 21, 19)
    grid = scenes.random_states(dims[::-1], 0.35, 0.08, seed=11)
    w = configs.Workload("t", 0, "u2", "count", configs.Camera(40, 30), grid, None, None)
    poi = np.array(dims, np.float64) * 0.005
    w.poses = poses.sphere_views(poi, 12, 0.25)
    for src in ("host", "device"):
        g = grid if src == "host" else torch.from_numpy(grid).cuda()
        gm = nbt.Map.from_grid(g, 0.01, (0.0, 0.0, 0.0), "u2", brick)
        ig, st = views_gpu(gm, w.poses, gpu_camera(w.camera), nbt.ig_params("count"))
        rig, rst = oracle.views_ig(oracle_map(w), w.poses, oracle_camera(w.camera), oracle.params("count"))
        assert np.array_equal(st, rst) and np.array_equal(ig, rig), (src, brick)


@pytest.mark.parametrize("packet_w", [4, 8, 16, 32])
def test_packet_shapes_same_results(packet_w):
    w = configs.exact64(seed=9, n_views=16)
    gm = gpu_map(w)
    gm.set_tuning(packet_w)
    assert gm.tuning() == {"packet_w": packet_w, "brick": 1, "skip": 1}
    ig, st = views_gpu(gm, w.poses, gpu_camera(w.camera), nbt.ig_params("count"))
    rig, rst = oracle.views_ig(oracle_map(w), w.poses, oracle_camera(w.camera), oracle.params("count"))
    assert np.array_equal(st, rst) and np.array_equal(ig, rig)
    with pytest.raises(nbt.NbtError):
        gm.set_tuning(6)


def test_large_host_upload_in_slabs():
    """A host upload larger than the 64 MiB staging buffer goes through several slabs."""
    n = 416  # 416^3 bytes = 72 MB of uint8 states
    grid = scenes.random_states((n, n, n), 0.3, 0.02, seed=4)
    for enc, brick in (("u8", 1), ("u2", 1), ("u2", 8)):
        a = nbt.Map.from_grid(grid, 0.01, (0.0, 0.0, 0.0), enc, brick)
        b = nbt.Map.from_grid(torch.from_numpy(grid).cuda(), 0.01, (0.0, 0.0, 0.0), enc, brick)
        poi = np.full(3, n * 0.005)
        p = poses.sphere_views(poi, 8, 0.6)
        cam = nbt.camera(32, 24, 1.0, 0.8, 1.2)
        ra = views_gpu(a, p, cam, nbt.ig_params("count"))
        rb = views_gpu(b, p, cam, nbt.ig_params("count"))
        assert np.array_equal(ra[0], rb[0]) and np.array_equal(ra[1], rb[1]), (enc, brick)
        a.close()
        b.close()


def test_traj_plan_graph_replays_match_direct_calls():
    w = configs.traj256(seed=4, n_traj=20, n=96, len_range=(2, 9))
    w.camera = configs.Camera(40, 30)
    gm = gpu_map(w)
    cam = gpu_camera(w.camera)
    prm = nbt.ig_params("count")
    pz = torch.from_numpy(w.poses).cuda()
    off = torch.from_numpy(w.offsets).cuda()
    plan = nbt.TrajPlan(gm, pz, off, cam, prm)
    for it in range(3):
        if it:
            # next planner cycle: new candidate poses, same shapes, refilled in place
            w2 = configs.traj256(seed=10 + it, n_traj=20, n=96, len_range=(2, 9))
            k = min(len(w2.poses), len(w.poses))
            pz[:k] = torch.from_numpy(w2.poses[:k]).cuda()
        got = plan.launch().clone()
        ref = nbt.traj_ig(gm, pz, off, cam, prm)
        torch.cuda.synchronize()
        assert torch.equal(got, ref), it
        rig, _ = oracle.traj_ig(oracle_map(w), pz.cpu().numpy(), w.offsets, oracle_camera(w.camera),
                                oracle.params("count"))
        assert np.array_equal(got.cpu().numpy().astype(np.float64), rig), it
    plan.close()


def test_autotune_returns_a_valid_fastest_config():
    w = configs.exact64(seed=3, n_views=32)
    cam = gpu_camera(w.camera)
    prm = nbt.ig_params("count")
    pz = torch.from_numpy(w.poses).cuda()
    m, cfg, timings = nbt.autotune(torch.from_numpy(w.grid).cuda(), w.voxel_size, w.origin, "u8", pz, cam, prm,
                                   layouts=(1, 8), packets=(8, 16), skips=(0, 1), reps=2)
    assert set(timings) == {(1, 8, 0), (1, 8, 1), (1, 16, 0), (1, 16, 1), (8, 8, 0), (8, 16, 0)}
    assert cfg["ms"] == min(timings.values())
    assert m.tuning() == {"packet_w": cfg["packet_w"], "brick": cfg["brick"], "skip": cfg["skip"]}
    ig, st = views_gpu(m, w.poses, cam, prm)
    rig, rst = oracle.views_ig(oracle_map(w), w.poses, oracle_camera(w.camera), oracle.params("count"))
    assert np.array_equal(st, rst) and np.array_equal(ig, rig)


def test_plan_launch_after_its_map_was_destroyed_is_refused():
    """A plan keeps its map's handle and creation id; once the map is destroyed the launch returns
    NBT_EINVAL and enqueues nothing, also when a new map was created in the meantime."""
    w = configs.traj256(seed=5, n_traj=4, n=48, len_range=(2, 4))
    w.camera = configs.Camera(16, 12)
    gm = gpu_map(w)
    cam = gpu_camera(w.camera)
    pz = torch.from_numpy(w.poses).cuda()
    off = torch.from_numpy(w.offsets).cuda()
    plan = nbt.TrajPlan(gm, pz, off, cam, nbt.ig_params("count"))
    plan.launch()
    torch.cuda.synchronize()
    gm.close()
    others = [gpu_map(w) for _ in range(3)]    # may reuse the freed address
    from paper_2503_22588_gb300 import _lib
    assert _lib.lib().nbt_plan_launch(plan._h, None) == -1
    plan.close()
    for m in others:
        m.close()
