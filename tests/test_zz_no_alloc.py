"""nbt_views_ig_noalloc against nbt_views_ig (GPU required).

The allocation-free entry point serves callers that may not allocate device
memory, such as a real-time planning loop or a process whose device memory
belongs to another allocator: it keeps its scratch in a fixed device array
of the library instead of a caller workspace.  Its results must match the
regular entry point's on two calls in a row, it must leave the device's
free memory unchanged, and it must refuse requests larger than its array.
This file is collected last so that a failure here comes after every other
test has run; it also passes on its own in a fresh process.
"""

import ctypes as C

import numpy as np
import pytest
import torch

import paper_2503_22588_gb300 as nbt
from paper_2503_22588_gb300 import _lib
from workload import configs

pytestmark = pytest.mark.gpu

RTOL = 1e-5  # the floating-point IG tolerance of the parity tests


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    nbt.build()


def _camera(w):
    c = w.camera
    return nbt.camera(c.width, c.height, c.fov_h, c.fov_v, c.max_range)


def _noalloc_call(m, poses, cam, prm, out, steps):
    """Call the entry point through the C ABI directly."""
    return _lib.lib().nbt_views_ig_noalloc(m.handle, poses.data_ptr(), poses.shape[0], C.byref(cam), C.byref(prm),
                                           out.data_ptr(), steps.data_ptr(),
                                           torch.cuda.current_stream().cuda_stream)


@pytest.mark.parametrize("which", ["exact64", "prob64"])
def test_noalloc_matches_views_ig_twice(which):
    if which == "exact64":
        w = configs.exact64(seed=5)
        prm = nbt.ig_params("count")
    else:
        w = configs.prob256(seed=5, n_views=48, n=64, n_prims=20)
        w.camera = configs.Camera(64, 48)
        prm = nbt.ig_params("entropy")
    cam = _camera(w)
    m = nbt.Map.from_grid(torch.from_numpy(w.grid).cuda(), w.voxel_size)
    poses = torch.from_numpy(w.poses).cuda()
    ref_ig, ref_steps = nbt.views_ig(m, poses, cam, prm)
    torch.cuda.synchronize()
    ref_ig = ref_ig.cpu().numpy().astype(np.float64)
    ref_steps = ref_steps.cpu().numpy()
    for _ in range(2):
        out = torch.full((len(w.poses),), -1.0, dtype=torch.float32, device="cuda")
        steps = torch.zeros(len(w.poses), dtype=torch.int64, device="cuda")
        assert _noalloc_call(m, poses, cam, prm, out, steps) == 0
        torch.cuda.synchronize()
        got = out.cpu().numpy().astype(np.float64)
        assert np.array_equal(steps.cpu().numpy(), ref_steps)
        assert np.all(np.abs(got - ref_ig) <= RTOL * np.maximum(np.abs(ref_ig), 1e-30))
    m.close()


def test_noalloc_allocates_no_device_memory():
    w = configs.exact64(seed=6)
    cam = _camera(w)
    prm = nbt.ig_params("count")
    m = nbt.Map.from_grid(torch.from_numpy(w.grid).cuda(), w.voxel_size)
    poses = torch.from_numpy(w.poses).cuda()
    out = torch.empty(len(w.poses), dtype=torch.float32, device="cuda")
    steps = torch.empty(len(w.poses), dtype=torch.int64, device="cuda")
    assert _noalloc_call(m, poses, cam, prm, out, steps) == 0  # first call: per-device set-up
    torch.cuda.synchronize()
    free_before, _ = torch.cuda.mem_get_info()
    for _ in range(2):
        assert _noalloc_call(m, poses, cam, prm, out, steps) == 0
    torch.cuda.synchronize()
    free_after, _ = torch.cuda.mem_get_info()
    assert free_after == free_before
    m.close()


def test_noalloc_rejects_requests_beyond_its_scratch():
    w = configs.exact64(seed=7, n_views=2)
    cam = nbt.camera(320, 240, 1.0, 0.8, 1.0)            # 300 tiles per view
    n = (4 << 20) // (16 * 300) + 1                       # one view more than fits
    m = nbt.Map.from_grid(torch.from_numpy(w.grid).cuda(), w.voxel_size)
    poses = torch.zeros((n, 7), dtype=torch.float32, device="cuda")
    poses[:, 3] = 1.0
    out = torch.empty(n, dtype=torch.float32, device="cuda")
    steps = torch.empty(n, dtype=torch.int64, device="cuda")
    assert _noalloc_call(m, poses, cam, nbt.ig_params("count"), out, steps) == -7
    assert _lib.lib().nbt_status_string(-7).startswith(b"NBT_ESCRATCH")
    assert _noalloc_call(m, poses[: n - 2], cam, nbt.ig_params("count"), out, steps) == 0
    torch.cuda.synchronize()
    # a view count whose byte size would wrap around int64 is refused as well (bounded before any
    # product), and nothing is enqueued: the last good results stay in place
    before = out.clone()
    for huge in (2 ** 31, 2 ** 60, 2 ** 63 - 1):
        rc = _lib.lib().nbt_views_ig_noalloc(m.handle, poses.data_ptr(), huge, C.byref(cam),
                                             C.byref(nbt.ig_params("count")), out.data_ptr(), steps.data_ptr(),
                                             torch.cuda.current_stream().cuda_stream)
        assert rc == -7, huge
    torch.cuda.synchronize()
    assert torch.equal(out, before)
    m.close()
