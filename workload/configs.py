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
* ``fig3`` (``fig3_scene``): the paper-exact ID on the prob256 tabletop --
  N_P perspectives from Eq. 1 in a ball of r_S = 1 m around the PoI, the
  endpoint grid of grid factor s_G (Section III), Eq. 2, mean per
  perspective -- swept over s_G x N_P like the paper's Fig. 3.
* ``insert`` (``insert_scans``): the map update -- 640 x 576 depth scans
  (Azure Kinect NFOV geometry) of an analytic tabletop inserted into a 256^3
  FP32 probability map of 1 cm voxels.
* ``idw_cost`` : IG cost of candidate trajectories (no map): a buffer of
  N_B = 10 IDs of N_P = 500 perspectives each (Eq. 1 in a ball of r_S = 1 m
  around the PoI; the paper's Section IV settings), and 16,384 candidate
  trajectories of 31 states (a 3 s horizon at 0.1 s steps), camera
  orientation jittered up to 40 degrees off the PoI.
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


FIG3_GRID_SCALES = (1, 5, 10, 20, 50, 100, 200)
FIG3_VIEW_COUNTS = (100, 250, 500, 1000)


def fig3_scene(seed: int = 0, n: int = 256, n_prims: int = 200):
    """The paper-exact ID setting on the tabletop: (grid, PoI, perspectives for N_P = 1000).

    FP32 probability tabletop (the ``prob256`` scene), PoI at the map centre,
    perspectives drawn with Eq. 1 in the ball of r_S = 1 m around it and
    looking at it (the first N_P rows are the N_P-perspective ID).
    """
    grid = _scenes.tabletop_probabilities(n, n_prims, seed)
    poi = np.full(3, n * VOXEL / 2)
    poses = _poses.ball_views(poi, max(FIG3_VIEW_COUNTS), 1.0, seed)
    return grid, poi, poses


def insert_scans(seed: int = 0, n_scans: int = 8, width: int = 640, height: int = 576):
    """Depth scans for the map update: (scans [(sensor pose, points)], map size n, voxel size).

    Azure Kinect NFOV geometry (640 x 576 pixels, 75 x 65 degrees, range
    3.86 m, 2 mm range noise) looking at the analytic tabletop from 0.6-1.2 m
    above it; the map is the 256^3 cube of 1 cm voxels around the table.
    """
    from . import sensor as _sensor
    scene = _sensor.tabletop_scene(seed)
    poi = np.array([1.28, 1.28, 0.8])
    scans = []
    for k, pose in enumerate(_sensor.scan_poses(poi, n_scans, seed)):
        pts = _sensor.depth_points(scene, pose, width, height, math.radians(75.0), math.radians(65.0), 3.86,
                                   0.002, seed * 100 + k)
        scans.append((pose, pts))
    return scans, 256, VOXEL


@dataclass
class CostWorkload:
    name: str
    ids: list                          # [(poses (N_P, 7) float32, g (N_P,) float32)], oldest first
    n_b: int
    poses: np.ndarray                  # (n_traj * horizon, 7) float32 candidate states
    offsets: np.ndarray                # (n_traj + 1,) int32
    poi: np.ndarray                    # (3,) float32
    fov_h_deg: float = 60.0
    fov_v_deg: float = 45.0
    power: float = 2.0
    w_info: float = 1.0
    eps: float = 1e-7
    meta: dict = field(default_factory=dict)

    @property
    def fov_h(self) -> float:
        return float(np.float32(math.radians(self.fov_h_deg)))

    @property
    def fov_v(self) -> float:
        return float(np.float32(math.radians(self.fov_v_deg)))


def id_gains(pos: np.ndarray, poi, seed: int, scale: float = 1.0) -> np.ndarray:
    """Synthetic mean ray IGs of perspectives at ``pos``: highest on a shell
    around the PoI, varying with azimuth, plus uniform noise (all >= 0)."""
    rng = np.random.default_rng(seed)
    v = pos - np.asarray(poi, np.float64)[None, :]
    r = np.linalg.norm(v, axis=1)
    phi = np.arctan2(v[:, 1], v[:, 0])
    g = 30.0 * np.exp(-((r - 0.6) / 0.3) ** 2) * (0.75 + 0.25 * np.cos(2.0 * phi)) + rng.uniform(0.0, 2.0, len(r))
    return (scale * g).astype(np.float32)


def idw_cost(seed: int = 0, n_traj: int = 16384, horizon: int = 31, n_ids: int = 10, n_p: int = 500,
             n_b: int = 10, jitter_deg: float = 40.0) -> CostWorkload:
    poi = np.array([0.8, 0.7, 0.5], np.float32)
    ids = []
    for m in range(n_ids):
        pz = _poses.ball_views(poi.astype(np.float64), n_p, 1.0, seed * 1000 + m)
        ids.append((pz, id_gains(pz[:, :3].astype(np.float64), poi, seed * 1000 + 500 + m, 0.7 + 0.03 * m)))
    poses, offsets = _traj.horizon_trajectories(poi, n_traj, horizon, seed, jitter_deg=jitter_deg)
    return CostWorkload("idw_cost", ids, n_b, poses, offsets, poi, meta={"horizon": horizon, "n_p": n_p})


WORKLOADS = {"exact64": exact64, "prob256": prob256, "traj256": traj256, "room512": room512}
