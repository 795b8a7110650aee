"""Shared helpers of the GPU tests (CUDA path vs. the CPU oracle)."""

from __future__ import annotations

import numpy as np
import torch

import oracle
import paper_2503_22588_gb300 as nbt

RTOL = 1e-5  # per-perspective IG vs the FP64 oracle (relative)


def gpu_camera(cam):
    return nbt.camera(cam.width, cam.height, cam.fov_h, cam.fov_v, cam.max_range, cam.grid_mode, cam.range_mode)


def oracle_camera(cam):
    return oracle.camera_of(cam)


def gpu_map(w, brick: int = 0, encoding: str | None = None):
    enc = encoding or w.encoding
    grid = torch.from_numpy(np.ascontiguousarray(w.grid)).cuda()
    return nbt.Map.from_grid(grid, w.voxel_size, w.origin, enc, brick)


def oracle_map(w):
    return oracle.Map(w.grid, w.voxel_size, w.origin)


def rel_err(a, b):
    a = np.asarray(a, np.float64)
    b = np.asarray(b, np.float64)
    return np.abs(a - b) / np.maximum(np.abs(b), 1e-30)


def views_gpu(m, poses: np.ndarray, cam, prm):
    p = torch.from_numpy(np.ascontiguousarray(poses)).cuda()
    ig, st = nbt.views_ig(m, p, cam, prm)
    torch.cuda.synchronize()
    return ig.cpu().numpy().astype(np.float64), st.cpu().numpy()
