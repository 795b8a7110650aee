"""Python binding of the IG raycasting library (same names as the C ABI).

Argument marshalling only: every step of the computation runs in the CUDA
kernels of libnbt.so.  PyTorch provides device memory and streams; device
arguments are CUDA tensors, host arguments numpy arrays or CPU tensors.
"""

from __future__ import annotations

import ctypes as C

import numpy as np
import torch

from ._lib import ENCODINGS, GRID, METRICS, RANGE, REDUCE, Camera, IgParams, InsertParams, MapDesc, Tuning, check, lib


def _stream(stream) -> int:
    if stream is None:
        return torch.cuda.current_stream().cuda_stream
    return stream.cuda_stream if hasattr(stream, "cuda_stream") else int(stream)


def _dev(t: torch.Tensor, dtype, name: str, shape_tail=None) -> int:
    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise TypeError(f"{name} must be a CUDA tensor")
    if t.dtype != dtype:
        raise TypeError(f"{name} must be {dtype}, got {t.dtype}")
    if not t.is_contiguous():
        raise ValueError(f"{name} must be contiguous")
    if shape_tail is not None and tuple(t.shape[1:]) != tuple(shape_tail):
        raise ValueError(f"{name} must have shape (n, {', '.join(map(str, shape_tail))})")
    return t.data_ptr()


def camera(width: int, height: int, fov_h: float, fov_v: float, max_range: float, grid_mode: str = "corners",
           range_mode: str = "planar") -> Camera:
    """nbt_camera: W x H rays, full opening angles in radians, range d_Cam in metres."""
    return Camera(int(width), int(height), float(fov_h), float(fov_v), float(max_range), GRID[grid_mode],
                  RANGE[range_mode])


def camera_from_grid_scale(fov_h: float, fov_v: float, max_range: float, voxel_size: float,
                           grid_scale: float) -> Camera:
    """nbt_camera_from_grid_scale: the paper's corner-to-corner endpoint grid with spacing s_G * s_Vox."""
    cam = Camera()
    check(lib().nbt_camera_from_grid_scale(float(fov_h), float(fov_v), float(max_range), float(voxel_size),
                                           float(grid_scale), C.byref(cam)), "nbt_camera_from_grid_scale")
    return cam


def ig_params(metric: str = "count", occ_threshold: float = 0.7, free_threshold: float = 0.3,
              include_hit: bool = True, reduce: str = "sum") -> IgParams:
    """nbt_ig_params: metric 'count' | 'eq2' | 'entropy', reduce 'sum' | 'mean'."""
    return IgParams(METRICS[metric], float(occ_threshold), float(free_threshold), int(bool(include_hit)),
                    REDUCE[reduce])


class Map:
    """nbt_map: a voxel map held on the current CUDA device."""

    def __init__(self, nx: int, ny: int, nz: int, voxel_size: float, origin=(0.0, 0.0, 0.0), encoding: str = "u8",
                 brick: int = 0):
        desc = MapDesc(int(nx), int(ny), int(nz), float(voxel_size), (C.c_float * 3)(*origin), ENCODINGS[encoding],
                       int(brick))
        h = C.c_void_p()
        check(lib().nbt_map_create(C.byref(desc), C.byref(h)), "nbt_map_create")
        self._h = h
        self.encoding = encoding
        self.dims = (int(nx), int(ny), int(nz))
        self.voxel_size = float(voxel_size)
        self.origin = tuple(float(v) for v in origin)

    @classmethod
    def from_grid(cls, grid, voxel_size: float, origin=(0.0, 0.0, 0.0), encoding: str | None = None,
                  brick: int = 0, stream=None) -> "Map":
        """Create a map from a dense (nz, ny, nx) grid and upload it."""
        nz, ny, nx = grid.shape
        if encoding is None:
            is_f32 = (grid.dtype == np.float32) if isinstance(grid, np.ndarray) else (grid.dtype == torch.float32)
            encoding = "f32" if is_f32 else "u8"
        m = cls(nx, ny, nz, voxel_size, origin, encoding, brick)
        m.upload(grid, stream)
        return m

    @property
    def handle(self) -> int:
        if self._h is None:
            raise ValueError("map is closed")
        return self._h.value

    def upload(self, grid, stream=None) -> None:
        """nbt_map_upload from a CUDA tensor, a CPU tensor or a numpy array (dense, x fastest).

        The copy is asynchronous on ``stream``: a pinned (page-locked) host grid is read when the
        stream reaches the copy, so keep it alive until then; pageable memory is read before the
        call returns.
        """
        want = np.float32 if self.encoding == "f32" else np.uint8
        if isinstance(grid, torch.Tensor) and grid.is_cuda:
            tdt = torch.float32 if want == np.float32 else torch.uint8
            ptr = _dev(grid, tdt, "grid")
            nbytes = grid.numel() * grid.element_size()
            check(lib().nbt_map_upload(self.handle, ptr, nbytes, 1, _stream(stream)), "nbt_map_upload")
            return
        arr = grid.numpy() if isinstance(grid, torch.Tensor) else grid
        arr = np.ascontiguousarray(arr)
        if arr.dtype != want:
            raise TypeError(f"grid must be {np.dtype(want)} for a {self.encoding} map")
        check(lib().nbt_map_upload(self.handle, arr.ctypes.data, arr.nbytes, 0, _stream(stream)), "nbt_map_upload")

    def info(self):
        desc = MapDesc()
        nbytes = C.c_int64()
        check(lib().nbt_map_info(self.handle, C.byref(desc), C.byref(nbytes)), "nbt_map_info")
        return desc, nbytes.value

    def download(self, stream=None) -> torch.Tensor:
        """nbt_map_download: the dense (nz, ny, nx) grid (uint8 states or float32 P) on the map's device."""
        d, _ = self.info()
        dt = torch.float32 if self.encoding == "f32" else torch.uint8
        out = torch.empty((d.nz, d.ny, d.nx), dtype=dt, device=torch.device("cuda", torch.cuda.current_device()))
        check(lib().nbt_map_download(self.handle, out.data_ptr(), out.numel() * out.element_size(), _stream(stream)),
              "nbt_map_download")
        return out

    def insert_points(self, points: torch.Tensor, sensor, prob_hit: float = 0.7, prob_miss: float = 0.4,
                      clamp_min: float = 0.1192, clamp_max: float = 0.971, max_range: float = 0.0,
                      stats: torch.Tensor | None = None, stream=None) -> None:
        """nbt_map_insert_points: one depth scan, points (n, 3) float32 world metres on the device.

        ``stats``: optional device int64 tensor of 3, written with (distinct
        endpoint voxels inside the map, rays cast, voxel steps walked).
        """
        n = points.shape[0]
        prm = InsertParams(float(prob_hit), float(prob_miss), float(clamp_min), float(clamp_max), float(max_range))
        s = (C.c_float * 3)(*[float(v) for v in sensor])
        st = _dev(stats, torch.int64, "stats") if stats is not None else None
        check(lib().nbt_map_insert_points(self.handle, _dev(points, torch.float32, "points", (3,)) if n else None, n,
                                          s, C.byref(prm), st, _stream(stream)), "nbt_map_insert_points")

    def set_tuning(self, packet_w: int = 8, skip: bool | None = None) -> None:
        """nbt_map_set_tuning: warp ray-packet width (4, 8, 16 or 32 pixels); ``skip``: count walks on
        linear state maps skip uniform 8^3 bricks (None keeps the current setting)."""
        sk = self.tuning()["skip"] if skip is None else int(bool(skip))
        check(lib().nbt_map_set_tuning(self.handle, C.byref(Tuning(int(packet_w), 0, sk))), "nbt_map_set_tuning")

    def tuning(self) -> dict:
        t = Tuning()
        check(lib().nbt_map_get_tuning(self.handle, C.byref(t)), "nbt_map_get_tuning")
        return {"packet_w": t.packet_w, "brick": t.brick, "skip": t.skip}

    def close(self) -> None:
        if getattr(self, "_h", None) is not None:
            lib().nbt_map_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def workspace_size(n_poses: int, cam: Camera) -> int:
    b = C.c_int64()
    check(lib().nbt_workspace_size(int(n_poses), C.byref(cam), C.byref(b)), "nbt_workspace_size")
    return b.value


def workspace(n_poses: int, cam: Camera, device=None) -> torch.Tensor:
    """A device workspace tensor large enough for n_poses perspectives."""
    return torch.empty(max(workspace_size(n_poses, cam), 16), dtype=torch.uint8,
                       device=device if device is not None else torch.device("cuda"))


def views_ig(m: Map, poses: torch.Tensor, cam: Camera, params: IgParams, out: torch.Tensor | None = None,
             steps: torch.Tensor | None = None, ws: torch.Tensor | None = None, stream=None, want_steps: bool = True):
    """nbt_views_ig: per-perspective IG of poses (n, 7) float32 on the device."""
    n = poses.shape[0]
    pp = _dev(poses, torch.float32, "poses", (7,))
    if out is None:
        out = torch.empty(n, dtype=torch.float32, device=poses.device)
    if steps is None and want_steps:
        steps = torch.empty(n, dtype=torch.int64, device=poses.device)
    if ws is None:
        ws = workspace(n, cam, poses.device)
    sp = _dev(steps, torch.int64, "steps") if steps is not None else None
    check(lib().nbt_views_ig(m.handle, pp, n, C.byref(cam), C.byref(params), _dev(out, torch.float32, "out"), sp,
                             _dev(ws, torch.uint8, "workspace"), ws.numel(), _stream(stream)), "nbt_views_ig")
    return out, steps


def traj_ig(m: Map, poses: torch.Tensor, offsets: torch.Tensor, cam: Camera, params: IgParams,
            out: torch.Tensor | None = None, pose_out: torch.Tensor | None = None, ws: torch.Tensor | None = None,
            stream=None):
    """nbt_traj_ig: per-trajectory IG over CSR offsets (n_traj + 1,) int32 on the device."""
    n = poses.shape[0]
    nt = offsets.shape[0] - 1
    pp = _dev(poses, torch.float32, "poses", (7,)) if n else 0
    if out is None:
        out = torch.empty(max(nt, 0), dtype=torch.float32, device=offsets.device)
    if ws is None:
        ws = workspace(n, cam, offsets.device)
    po = _dev(pose_out, torch.float32, "pose_out") if pose_out is not None else None
    check(lib().nbt_traj_ig(m.handle, pp, n, _dev(offsets, torch.int32, "offsets"), nt, C.byref(cam),
                            C.byref(params), _dev(out, torch.float32, "out") if nt > 0 else None, po,
                            _dev(ws, torch.uint8, "workspace"), ws.numel(), _stream(stream)), "nbt_traj_ig")
    return out


def trace_segments(m: Map, o: torch.Tensor, d: torch.Tensor, params: IgParams | None = None,
                   cap: int | None = None, stream=None):
    """nbt_trace_segments: visited voxel indices per segment (int32 (n, cap)) and counts (n,)."""
    n = o.shape[0]
    cap = sum(m.dims) + 3 if cap is None else cap
    idx = torch.full((n, cap), -1, dtype=torch.int32, device=o.device)
    cnt = torch.zeros(n, dtype=torch.int32, device=o.device)
    prm = C.byref(params) if params is not None else None
    check(lib().nbt_trace_segments(m.handle, _dev(o, torch.float32, "o", (3,)), _dev(d, torch.float32, "d", (3,)), n,
                                   prm, idx.data_ptr(), cap, cnt.data_ptr(), _stream(stream)), "nbt_trace_segments")
    return idx, cnt


def view_segments(m: Map, poses: torch.Tensor, cam: Camera, stream=None):
    """nbt_view_segments: the FP32 ray segments (voxel units) the kernels generate."""
    n = poses.shape[0] * cam.width * cam.height
    o = torch.empty((n, 3), dtype=torch.float32, device=poses.device)
    d = torch.empty((n, 3), dtype=torch.float32, device=poses.device)
    check(lib().nbt_view_segments(m.handle, _dev(poses, torch.float32, "poses", (7,)), poses.shape[0],
                                  C.byref(cam), o.data_ptr(), d.data_ptr(), _stream(stream)), "nbt_view_segments")
    return o, d


def views_ig_noalloc(m: Map, poses: torch.Tensor, cam: Camera, params: IgParams, out: torch.Tensor,
                     steps: torch.Tensor | None = None, stream=None):
    """nbt_views_ig_noalloc: nbt_views_ig with its scratch in the library's fixed device array.

    For callers that must not allocate device memory (a real-time planning
    loop, a process whose device memory belongs to another allocator): the
    outputs are preallocated by the caller and the call allocates nothing.
    Calls that overlap on the GPU race on the shared array.
    """
    n = poses.shape[0]
    sp = _dev(steps, torch.int64, "steps") if steps is not None else None
    check(lib().nbt_views_ig_noalloc(m.handle, _dev(poses, torch.float32, "poses", (7,)), n, C.byref(cam),
                                     C.byref(params), _dev(out, torch.float32, "out"), sp, _stream(stream)),
          "nbt_views_ig_noalloc")
    return out, steps


class TrajPlan:
    """nbt_plan: one nbt_traj_ig call captured in a CUDA graph, replayed per planning cycle.

    The tensors passed here are kept alive by the plan; refill ``poses`` and
    ``offsets`` in place between launches.
    """

    def __init__(self, m: Map, poses: torch.Tensor, offsets: torch.Tensor, cam: Camera, params: IgParams,
                 out: torch.Tensor | None = None, pose_out: torch.Tensor | None = None):
        n = poses.shape[0]
        nt = offsets.shape[0] - 1
        self.map, self.poses, self.offsets = m, poses, offsets
        self.out = out if out is not None else torch.empty(max(nt, 0), dtype=torch.float32, device=offsets.device)
        self.pose_out = pose_out
        self.ws = workspace(n, cam, offsets.device)
        self._cam, self._params = cam, params
        h = C.c_void_p()
        po = _dev(pose_out, torch.float32, "pose_out") if pose_out is not None else None
        check(lib().nbt_plan_create_traj(m.handle, _dev(poses, torch.float32, "poses", (7,)) if n else None, n,
                                         _dev(offsets, torch.int32, "offsets"), nt, C.byref(cam), C.byref(params),
                                         _dev(self.out, torch.float32, "out") if nt > 0 else None, po,
                                         _dev(self.ws, torch.uint8, "workspace"), self.ws.numel(), C.byref(h)),
              "nbt_plan_create_traj")
        self._h = h

    def launch(self, stream=None) -> torch.Tensor:
        if self.map._h is None:
            raise ValueError("the plan's map is closed")
        check(lib().nbt_plan_launch(self._h, _stream(stream)), "nbt_plan_launch")
        return self.out

    def close(self) -> None:
        if getattr(self, "_h", None) is not None:
            lib().nbt_plan_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
