"""Autotuner for the IG kernels: map layout (brick) and warp ray-packet shape.

For one workload shape it builds the map in each candidate layout, times
``nbt_traj_ig`` (or ``nbt_views_ig`` when no offsets are given) for each
packet width with CUDA events, and returns the fastest map, its tuning and
all timings.  Every candidate visits the same voxels (the parity tests check
all layouts and packet shapes), so tuning changes speed only.
"""

from __future__ import annotations

import torch

from .api import Camera, IgParams, Map, traj_ig, views_ig, workspace

LAYOUTS = (1, 4, 8)          # linear, 4^3 and 8^3 Morton bricks
PACKETS = (4, 8, 16, 32)     # warp packet width in pixels (height 32 / width)


def _time(fn, reps: int, stream) -> float:
    for _ in range(2):
        fn()
    start = torch.cuda.Event(enable_timing=True)
    stop = torch.cuda.Event(enable_timing=True)
    start.record(stream)
    for _ in range(reps):
        fn()
    stop.record(stream)
    stop.synchronize()
    return start.elapsed_time(stop) / reps


def autotune(grid, voxel_size: float, origin, encoding: str, poses: torch.Tensor, cam: Camera, params: IgParams,
             offsets: torch.Tensor | None = None, layouts=LAYOUTS, packets=PACKETS, skips=(0,), reps: int = 5):
    """Return (best Map, {"brick", "packet_w", "skip", "ms"}, {(brick, packet_w, skip): ms}).

    ``grid`` is the dense (nz, ny, nx) map (CUDA tensor or numpy).  ``skips``:
    brick skipping off / on (it applies to linear state maps only).  The maps
    built for the other layouts are closed before returning.
    """
    stream = torch.cuda.current_stream()
    n = poses.shape[0]
    ws = workspace(n, cam, poses.device)
    out = torch.empty(n if offsets is None else offsets.shape[0] - 1, dtype=torch.float32, device=poses.device)
    maps = {brick: Map.from_grid(grid, voxel_size, origin, encoding, brick) for brick in layouts}
    timings = {}
    state_map = encoding != "f32"
    for brick, m in maps.items():
        for pw in packets:
            for sk in (skips if state_map and brick == 1 else (0,)):
                m.set_tuning(pw, sk)
                if offsets is None:
                    fn = lambda: views_ig(m, poses, cam, params, out, None, ws, stream, want_steps=False)  # noqa: E731
                else:
                    fn = lambda: traj_ig(m, poses, offsets, cam, params, out, None, ws, stream)  # noqa: E731
                timings[(brick, pw, sk)] = _time(fn, reps, stream)
    (brick, pw, sk), ms = min(timings.items(), key=lambda kv: kv[1])
    for b, m in maps.items():
        if b != brick:
            m.close()
    best = maps[brick]
    best.set_tuning(pw, sk)
    return best, {"brick": brick, "packet_w": pw, "skip": sk, "ms": ms}, timings
