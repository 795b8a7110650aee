"""The C ABI library loads and exports every symbol include/nbt.h declares (no GPU)."""

import ctypes as C
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    text = open(os.path.join(ROOT, "include", "nbt.h")).read()
    return sorted(set(re.findall(r"^\s*(?:int|const char \*)\s*(nbt_\w+)\s*\(", text, re.M)))


@pytest.fixture(scope="module")
def libnbt():
    import paper_2503_22588_gb300 as nbt
    try:
        nbt.build()
    except (RuntimeError, FileNotFoundError) as e:  # no nvcc on this machine
        if not os.path.exists(nbt.LIB_PATH):
            pytest.skip(f"cannot build libnbt.so here: {e}")
    return nbt


def test_every_declared_symbol_is_exported_and_bound(libnbt):
    from paper_2503_22588_gb300 import _lib
    names = declared_functions()
    assert len(names) >= 11
    raw = C.CDLL(libnbt.LIB_PATH)
    for n in names:
        assert hasattr(raw, n), n
        assert n in _lib.SIGNATURES, n
    assert set(_lib.SIGNATURES) == set(names)


def test_host_only_entry_points(libnbt):
    from paper_2503_22588_gb300 import _lib
    L = _lib.lib()
    v = C.c_int32()
    assert L.nbt_get_version(C.byref(v)) == 0 and v.value == 1
    assert L.nbt_get_version(None) == -1
    assert L.nbt_status_string(-6).startswith(b"NBT_EWORKSPACE")
    assert L.nbt_map_create(None, None) == -1
    assert L.nbt_map_destroy(None) == 0
    cam = libnbt.camera(160, 120, 1.0, 0.8, 1.0)
    b = C.c_int64()
    assert L.nbt_workspace_size(1024, C.byref(cam), C.byref(b)) == 0
    assert b.value == 256 + 1024 * 5 * 15 * 16
    assert L.nbt_workspace_size(-1, C.byref(cam), C.byref(b)) == -1
    bad = libnbt.camera(0, 120, 1.0, 0.8, 1.0)
    assert L.nbt_workspace_size(4, C.byref(bad), C.byref(b)) == -1
    h = C.c_void_p()
    assert L.nbt_id_buffer_create(0, 10, C.byref(h)) == -1        # N_B out of range
    assert L.nbt_id_buffer_create(33, 10, C.byref(h)) == -1
    assert L.nbt_id_buffer_create(10, 0, C.byref(h)) == -1        # no perspectives
    assert L.nbt_id_buffer_create(10, 10, None) == -1
    assert L.nbt_id_buffer_destroy(None) == 0
    assert L.nbt_id_buffer_clear(None) == -1
    assert L.nbt_id_buffer_count(None, None) == -1
    assert L.nbt_idw_gain(None, None, 0, 2.0, None, None) == -1
    prm = _lib.CostParams(2.0, 1.0, 1e-7)
    poi = (C.c_float * 3)(0.0, 0.0, 0.0)
    assert L.nbt_ig_cost(None, None, 0, None, 0, poi, 1.0, 1.0, C.byref(prm), None, None, None, None, None) == -1


def test_structs_match_header_sizes():
    from paper_2503_22588_gb300 import _lib
    assert C.sizeof(_lib.MapDesc) == 36
    assert C.sizeof(_lib.Camera) == 28
    assert C.sizeof(_lib.IgParams) == 20
    assert C.sizeof(_lib.Tuning) == 12
    assert C.sizeof(_lib.CostParams) == 12


def test_product_package_does_not_touch_the_oracle():
    pkg = os.path.join(ROOT, "paper_2503_22588_gb300")
    for dirpath, _, files in os.walk(pkg):
        for f in files:
            if f.endswith((".py", ".cu", ".cuh", ".h", ".cpp")):
                text = open(os.path.join(dirpath, f)).read()
                for bad in ("import oracle", "from oracle", "liborc", "nbt_oracle"):
                    assert bad not in text, (f, bad)


def test_grid_scale_camera_matches_the_oracle(libnbt):
    """Host-only entry point: the paper's s_G endpoint grid, against oracle/endpoints.py."""
    import math
    import numpy as np
    from oracle import endpoints as E
    rng = np.random.default_rng(1)
    cases = [(math.radians(60), math.radians(45), 1.0, 0.01, g) for g in (1, 5, 10, 20, 50, 100, 200)]
    cases += [tuple(rng.uniform(0.2, 2.5, 2)) + (rng.uniform(0.2, 5.0), 0.01, rng.uniform(1.0, 300.0))
              for _ in range(200)]
    for fh, fv, d, sv, sg in cases:
        cam = libnbt.camera_from_grid_scale(fh, fv, d, sv, sg)
        assert (cam.width, cam.height) == E.grid_size(fh, fv, d, sv, sg), (fh, fv, d, sv, sg)
        assert cam.grid_mode == 0 and cam.range_mode == 0
        assert abs(cam.fov_h - fh) <= 1e-6 * fh and cam.max_range == np.float32(d)
    from paper_2503_22588_gb300 import NbtError
    import pytest as _pt
    for bad in ((0.0, 1.0, 1.0, 0.01, 5.0), (1.0, 3.2, 1.0, 0.01, 5.0), (1.0, 1.0, 1.0, 0.01, -1.0),
                (1.0, 1.0, float("nan"), 0.01, 5.0), (3.0, 1.0, 100.0, 0.0001, 0.01)):
        with _pt.raises(NbtError):
            libnbt.camera_from_grid_scale(*bad)


def test_surrogate_parameter_layout_matches_the_oracle_network(libnbt):
    """The library's parameter count, and the binding's layout of them (the order
    nbt_surrogate_set_params documents), equal the oracle network's shapes."""
    import numpy as np

    from oracle import surrogate as S
    from paper_2503_22588_gb300 import surrogate as gs
    p = S.init_params(0)
    assert gs.param_count() == sum(v.size for v in p.values())
    assert [k for k, _ in gs.SHAPES] == list(p.keys())
    assert all(tuple(p[k].shape) == tuple(shp) for k, shp in gs.SHAPES)
    back = gs.unpack(gs.pack(p))
    assert all(np.array_equal(back[k], p[k]) for k in p)


def test_map_create_rejects_bad_descriptions_before_any_cuda_call(libnbt):
    """Map descriptions are validated on the host first, so these fail with NBT_EINVAL (-1) on a
    machine without a GPU as well: sides outside [1, 2048], 2^31 or more voxels, a brick other than
    1, 4 or 8, a non-positive or non-finite voxel size, a non-finite origin, an unknown encoding."""
    from paper_2503_22588_gb300 import _lib
    L = _lib.lib()

    def create(nx=8, ny=8, nz=8, voxel=0.01, origin=(0.0, 0.0, 0.0), enc=0, brick=1):
        d = _lib.MapDesc(nx, ny, nz, voxel, (C.c_float * 3)(*origin), enc, brick)
        h = C.c_void_p()
        rc = L.nbt_map_create(C.byref(d), C.byref(h))
        assert h.value is None
        return rc

    bad = [dict(nx=0), dict(ny=-3), dict(nz=2049), dict(nx=2048, ny=2048, nz=512), dict(brick=5),
           dict(brick=2), dict(voxel=0.0), dict(voxel=-0.01), dict(voxel=float("nan")), dict(voxel=float("inf")),
           dict(origin=(0.0, float("nan"), 0.0)), dict(origin=(float("inf"), 0.0, 0.0)), dict(enc=3), dict(enc=-1)]
    for kw in bad:
        assert create(**kw) == -1, kw


def test_surrogate_create_rejects_batch_sizes_outside_1_to_4096(libnbt):
    from paper_2503_22588_gb300 import _lib
    L = _lib.lib()
    h = C.c_void_p()
    for mb in (0, -1, 4097):
        assert L.nbt_surrogate_create(mb, C.byref(h)) == -1 and h.value is None
    assert L.nbt_surrogate_create(16, None) == -1


def test_null_handles_are_rejected_on_the_host(libnbt):
    """Every entry point that takes a map, plan, surrogate or ID-buffer handle answers NBT_EINVAL to a
    NULL handle without touching the GPU; destroying NULL is a no-op (NBT_OK)."""
    from paper_2503_22588_gb300 import _lib
    L = _lib.lib()
    cam = libnbt.camera(8, 8, 1.0, 0.8, 1.0)
    prm = libnbt.ig_params("count")
    calls = {
        "nbt_map_upload": (None, None, 0, 0, None),
        "nbt_map_info": (None, None, None),
        "nbt_map_download": (None, None, 0, None),
        "nbt_views_ig": (None, None, 1, C.byref(cam), C.byref(prm), None, None, None, 0, None),
        "nbt_views_ig_noalloc": (None, None, 1, C.byref(cam), C.byref(prm), None, None, None),
        "nbt_traj_ig": (None, None, 1, None, 1, C.byref(cam), C.byref(prm), None, None, None, 0, None),
        "nbt_trace_segments": (None, None, None, 1, None, None, 0, None, None),
        "nbt_view_segments": (None, None, 1, C.byref(cam), None, None, None),
        "nbt_plan_launch": (None, None),
        "nbt_map_set_tuning": (None, None),
        "nbt_map_get_tuning": (None, None),
        "nbt_surrogate_set_params": (None, None, 0),
        "nbt_surrogate_get_params": (None, None, 0),
        "nbt_surrogate_forward": (None, None, None, 1, None, None),
        "nbt_id_buffer_push": (None, None, None, 1, None),
        "nbt_id_buffer_count": (None, None),
    }
    for name, args in calls.items():
        assert getattr(L, name)(*args) == -1, name
    for name in ("nbt_map_destroy", "nbt_plan_destroy", "nbt_surrogate_destroy", "nbt_id_buffer_destroy"):
        assert getattr(L, name)(None) == 0, name


def test_sizes_are_bounded_before_they_are_multiplied(libnbt):
    """nbt_workspace_size takes n_poses in [0, INT32_MAX]: a huge count (whose byte size would wrap
    around int64) is refused on the host instead of returning a wrapped, small size."""
    from paper_2503_22588_gb300 import _lib
    L = _lib.lib()
    cam = libnbt.camera(1, 1, 1.0, 0.8, 1.0)
    b = C.c_int64(-5)
    for n in (2 ** 31, 2 ** 60, 2 ** 63 - 1):
        assert L.nbt_workspace_size(n, C.byref(cam), C.byref(b)) == -1, n
    assert b.value == -5
    assert L.nbt_workspace_size(2 ** 31 - 1, C.byref(cam), C.byref(b)) == 0
    assert b.value == 256 + (2 ** 31 - 1) * 16


def test_handles_that_name_no_live_map_are_rejected_without_reading_them(libnbt):
    """A map handle that was never created (or was destroyed) is checked against the live-map
    registry before it is read: NBT_EINVAL, no GPU needed, no memory behind the pointer touched."""
    from paper_2503_22588_gb300 import _lib
    L = _lib.lib()
    bogus = C.c_void_p(0x10)          # not a valid address: reading it would crash the test
    cam = libnbt.camera(8, 8, 1.0, 0.8, 1.0)
    prm = libnbt.ig_params("count")
    assert L.nbt_map_destroy(bogus) == -1
    assert L.nbt_map_info(bogus, None, None) == -1
    assert L.nbt_views_ig(bogus, None, 1, C.byref(cam), C.byref(prm), None, None, None, 0, None) == -1
    assert L.nbt_views_ig_noalloc(bogus, None, 1, C.byref(cam), C.byref(prm), None, None, None) == -1
    assert L.nbt_map_upload(bogus, None, 0, 0, None) == -1
    t = _lib.Tuning(8, 0, 0)
    assert L.nbt_map_set_tuning(bogus, C.byref(t)) == -1
    assert L.nbt_map_get_tuning(bogus, C.byref(t)) == -1


def test_surrogate_checkpoint_file_round_trip_is_bitwise(tmp_path):
    """save_checkpoint / load_checkpoint keep every bit of the parameters and Adam moments, the step
    count and the target scale; a file of the wrong size is refused (no GPU needed)."""
    import numpy as np
    from paper_2503_22588_gb300 import surrogate as gs
    n = gs.param_count()
    rng = np.random.default_rng(0)
    state = {"params": rng.standard_normal(n).astype(np.float32),
             "adam_m": rng.standard_normal(n).astype(np.float32) * 1e-3,
             "adam_v": np.abs(rng.standard_normal(n)).astype(np.float32) * 1e-6,
             "step": 123456789012, "target_scale": 0.01}
    state["params"][:3] = [np.float32(-0.0), np.float32(1e-45), np.float32(3.4e38)]
    gs.save_checkpoint(state, tmp_path / "ck.npz")
    got = gs.load_checkpoint(tmp_path / "ck.npz")
    for k in ("params", "adam_m", "adam_v"):
        assert got[k].dtype == np.float32 and got[k].tobytes() == state[k].tobytes(), k
    assert got["step"] == state["step"] and got["target_scale"] == state["target_scale"]
    with pytest.raises(ValueError):
        gs.save_checkpoint({**state, "params": state["params"][:-1]}, tmp_path / "bad.npz")
    np.savez(tmp_path / "short.npz", params=state["params"][:-1], adam_m=state["adam_m"],
             adam_v=state["adam_v"], step=np.int64(1), target_scale=np.float64(1.0))
    with pytest.raises(ValueError):
        gs.load_checkpoint(tmp_path / "short.npz")
