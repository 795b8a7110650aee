"""Named synthetic workloads (inputs only).

Each workload stands in for the paper's replayed Azure Kinect stream (not
available here) with a seeded scene of the stated size.  Voxel size is 1 cm
everywhere (Section V), the map origin is the world origin, and the camera
looks at its PoI.  Field of view 60 x 45 degrees and range 1.0 m are used for
all workloads (the tabletop and room workloads do not state them; the same
camera as the 64^3 workload is assumed).

Names (sizes in the name, as the workloads are referred to everywhere):

* ``exact64``  : 64^3 uint8 states, 20 boxes/spheres, half unknown; 64 views on a
  0.5 m sphere; 64 x 48 rays; IG = unknown voxels before the first occupied one.
* ``prob256``  : 256^3 FP32 probabilities, tabletop of 200 primitives; 1024 views on
  a Fibonacci shell of radii 0.3-0.8 m; 160 x 120 rays; IG = binary entropy
  summed until p > 0.7.
* ``traj256``  : 256^3 uint8 tabletop; 512 trajectories of 5-40 poses around 4 PoIs;
  128 x 96 rays; per-trajectory IG = sum of per-pose IG.
* ``room512``  : 512^3 2-bit states, room of 2000 primitives, 40 % unknown;
  8 PoIs x 4096 views; 320 x 240 rays.
"""

from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

from . import poses as _poses
from . import scenes as _scenes
from . import trajectories as _traj

VOXEL = 0.01


@dataclass
class Camera:
    width: int
    height: int
    fov_h_deg: float = 60.0
    fov_v_deg: float = 45.0
    max_range: float = 1.0
    grid_mode: str = "corners"      # "corners" (paper: border rays included) | "centers"
    range_mode: str = "planar"      # "planar" (far plane at d_Cam) | "spherical"

    @property
    def fov_h(self) -> float:
        return float(np.float32(math.radians(self.fov_h_deg)))

    @property
    def fov_v(self) -> float:
        return float(np.float32(math.radians(self.fov_v_deg)))


@dataclass
class Workload:
    name: str
    n: int
    encoding: str                     # "u8" | "f32" | "u2"
    metric: str                       # "count" | "entropy" | "eq2"
    camera: Camera
    grid: np.ndarray                  # (n, n, n) uint8 states or float32 probabilities
    poses: np.ndarray                 # (n_poses, 7) float32
    pois: np.ndarray                  # (k, 3) float64 world metres
    offsets: np.ndarray | None = None # int32 CSR offsets for trajectory workloads
    voxel_size: float = VOXEL
    origin: tuple = (0.0, 0.0, 0.0)
    meta: dict = field(default_factory=dict)

    @property
    def n_poses(self) -> int:
        return int(self.poses.shape[0])

    @property
    def rays_per_pose(self) -> int:
        return self.camera.width * self.camera.height


def exact64(seed: int = 0, n_views: int = 64) -> Workload:
    n = 64
    grid = _scenes.boxes_spheres(n, 20, seed, half_unknown=True)
    poi = np.full(3, n * VOXEL / 2)
    poses = _poses.sphere_views(poi, n_views, 0.5)
    return Workload("exact64", n, "u8", "count", Camera(64, 48), grid, poses, poi[None, :])


def prob256(seed: int = 0, n_views: int = 1024, n: int = 256, n_prims: int = 200) -> Workload:
    grid = _scenes.tabletop_probabilities(n, n_prims, seed)
    poi = np.full(3, n * VOXEL / 2)
    poses = _poses.shell_views(poi, n_views, 0.3, 0.8, seed)
    return Workload("prob256", n, "f32", "entropy", Camera(160, 120), grid, poses, poi[None, :])


def _tabletop_pois(n: int) -> np.ndarray:
    c = n / 2.0
    zt = c - min(12.0, 0.05 * n)
    pts = [(c - 0.15 * n, c - 0.08 * n, zt + 8.0), (c + 0.15 * n, c - 0.08 * n, zt + 8.0),
           (c - 0.15 * n, c + 0.08 * n, zt + 8.0), (c + 0.15 * n, c + 0.08 * n, zt + 8.0)]
    return np.array(pts) * VOXEL


def traj256(seed: int = 0, n_traj: int = 512, n: int = 256, len_range=(5, 40)) -> Workload:
    grid = _scenes.tabletop_states(n, 200, seed)
    pois = _tabletop_pois(n)
    poses, offsets = _traj.random_trajectories(pois, n_traj, seed, len_range=len_range)
    return Workload("traj256", n, "u8", "count", Camera(128, 96), grid, poses, pois, offsets=offsets)


def room512(seed: int = 0, n_pois: int = 8, views_per_poi: int = 4096, n: int = 512,
            n_prims: int = 2000) -> Workload:
    grid = _scenes.room_states(n, n_prims, 0.4, seed)
    rng = np.random.default_rng(seed + 77)
    pois = rng.uniform(1.0, n * VOXEL - 1.0, size=(n_pois, 3))
    poses = np.concatenate([_poses.shell_views(p, views_per_poi, 0.3, 0.8, seed + 1 + k)
                            for k, p in enumerate(pois)])
    return Workload("room512", n, "u2", "count", Camera(320, 240), grid, poses, pois)


WORKLOADS = {"exact64": exact64, "prob256": prob256, "traj256": traj256, "room512": room512}
