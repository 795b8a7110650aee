"""Seeded voxel scenes (inputs only).

Every generator is deterministic in its ``seed`` and returns dense grids of
shape ``(nz, ny, nx)`` (x fastest).  A voxel belongs to a primitive when its
centre ``(i + 0.5)`` lies inside the primitive (coordinates in voxel units).
"""

from __future__ import annotations

import math

import numpy as np

UNKNOWN, FREE, OCCUPIED = 0, 1, 2


def _centre_range(lo: float, hi: float, n: int) -> tuple[int, int]:
    """Index range [a, b) of voxels whose centres lie in [lo, hi)."""
    a = max(0, math.ceil(lo - 0.5))
    b = min(n, math.ceil(hi - 0.5))
    return a, max(a, b)


def fill_box(mask: np.ndarray, lo, hi) -> None:
    """Mark voxels whose centres lie in the axis-aligned box [lo, hi) (x, y, z)."""
    nz, ny, nx = mask.shape
    x0, x1 = _centre_range(lo[0], hi[0], nx)
    y0, y1 = _centre_range(lo[1], hi[1], ny)
    z0, z1 = _centre_range(lo[2], hi[2], nz)
    mask[z0:z1, y0:y1, x0:x1] = True


def fill_sphere(mask: np.ndarray, c, r: float) -> None:
    """Mark voxels whose centres lie in the closed ball of radius r around c."""
    nz, ny, nx = mask.shape
    x0, x1 = _centre_range(c[0] - r, c[0] + r + 1e-9, nx)
    y0, y1 = _centre_range(c[1] - r, c[1] + r + 1e-9, ny)
    z0, z1 = _centre_range(c[2] - r, c[2] + r + 1e-9, nz)
    if x0 >= x1 or y0 >= y1 or z0 >= z1:
        return
    zz, yy, xx = np.meshgrid(np.arange(z0, z1) + 0.5 - c[2],
                             np.arange(y0, y1) + 0.5 - c[1],
                             np.arange(x0, x1) + 0.5 - c[0], indexing="ij")
    inside = xx * xx + yy * yy + zz * zz <= r * r
    mask[z0:z1, y0:y1, x0:x1] |= inside


def fill_cylinder_z(mask: np.ndarray, c_xy, r: float, z_lo: float, z_hi: float) -> None:
    """Mark voxels inside a vertical cylinder (axis parallel to z)."""
    nz, ny, nx = mask.shape
    x0, x1 = _centre_range(c_xy[0] - r, c_xy[0] + r + 1e-9, nx)
    y0, y1 = _centre_range(c_xy[1] - r, c_xy[1] + r + 1e-9, ny)
    z0, z1 = _centre_range(z_lo, z_hi, nz)
    if x0 >= x1 or y0 >= y1 or z0 >= z1:
        return
    yy, xx = np.meshgrid(np.arange(y0, y1) + 0.5 - c_xy[1],
                         np.arange(x0, x1) + 0.5 - c_xy[0], indexing="ij")
    disk = xx * xx + yy * yy <= r * r
    mask[z0:z1, y0:y1, x0:x1] |= disk[None, :, :]


def states_from_masks(occupied: np.ndarray, unknown: np.ndarray) -> np.ndarray:
    """uint8 states: unknown overrides occupied, everything else is free."""
    st = np.where(occupied, OCCUPIED, FREE).astype(np.uint8)
    st[unknown] = UNKNOWN
    return st


def uniform_states(shape, state: int) -> np.ndarray:
    """A grid holding one state everywhere."""
    return np.full(shape, state, dtype=np.uint8)


def random_states(shape, p_unknown: float, p_occupied: float, seed: int) -> np.ndarray:
    """I.i.d. voxel states (for tests): unknown / occupied / free by probability."""
    rng = np.random.default_rng(seed)
    u = rng.random(shape)
    st = np.full(shape, FREE, dtype=np.uint8)
    st[u < p_unknown + p_occupied] = OCCUPIED
    st[u < p_unknown] = UNKNOWN
    return st


def boxes_spheres(n: int = 64, n_prims: int = 20, seed: int = 0,
                  size_range=(2.0, 12.0), half_unknown: bool = True) -> np.ndarray:
    """n^3 state grid with random axis-aligned boxes and spheres.

    Primitive sizes (box edge, sphere diameter) are uniform in ``size_range``
    voxels, centres uniform in the grid.  With ``half_unknown`` the half
    ``x >= n/2`` is set to unknown, overriding free and occupied.
    """
    rng = np.random.default_rng(seed)
    occ = np.zeros((n, n, n), dtype=bool)
    for _ in range(n_prims):
        c = rng.uniform(0.0, n, size=3)
        if rng.integers(2) == 0:
            half = rng.uniform(size_range[0], size_range[1], size=3) / 2.0
            fill_box(occ, c - half, c + half)
        else:
            r = rng.uniform(size_range[0], size_range[1]) / 2.0
            fill_sphere(occ, c, r)
    unk = np.zeros_like(occ)
    if half_unknown:
        unk[:, :, n // 2:] = True
    return states_from_masks(occ, unk)


def tabletop_masks(n: int = 256, n_prims: int = 200, seed: int = 0):
    """Cluttered tabletop: (occupied, unknown) boolean masks.

    A 3-voxel-thick table top whose upper face is 12 voxels below the grid
    centre, covering 160 x 100 voxels around the centre, four legs, and
    ``n_prims`` boxes / spheres / vertical cylinders (2-16 voxels) standing on
    the table.  Unknown: the space under the table top inside its footprint,
    and the slab ``x >= n/2 + n/16`` (overriding objects there).
    """
    rng = np.random.default_rng(seed)
    occ = np.zeros((n, n, n), dtype=bool)
    c = n / 2.0
    hx, hy = min(80.0, 0.31 * n), min(50.0, 0.2 * n)
    zt = c - min(12.0, 0.05 * n)
    fill_box(occ, (c - hx, c - hy, zt - 3.0), (c + hx, c + hy, zt))
    for sx in (-1, 1):
        for sy in (-1, 1):
            lx, ly = c + sx * (hx - 3.0), c + sy * (hy - 3.0)
            fill_box(occ, (lx - 2.0, ly - 2.0, 0.0), (lx + 2.0, ly + 2.0, zt - 3.0))
    for _ in range(n_prims):
        px = rng.uniform(c - hx + 2.0, c + hx - 2.0)
        py = rng.uniform(c - hy + 2.0, c + hy - 2.0)
        size = rng.uniform(2.0, 16.0, size=3)
        kind = rng.integers(3)
        if kind == 0:
            fill_box(occ, (px - size[0] / 2, py - size[1] / 2, zt), (px + size[0] / 2, py + size[1] / 2, zt + size[2]))
        elif kind == 1:
            r = size[0] / 2
            fill_sphere(occ, (px, py, zt + r), r)
        else:
            fill_cylinder_z(occ, (px, py), size[0] / 2, zt, zt + size[2])
    unk = np.zeros_like(occ)
    fill_box(unk, (c - hx, c - hy, 0.0), (c + hx, c + hy, zt - 3.0))
    unk &= ~occ
    unk[:, :, int(c + n / 16):] = True
    return occ, unk


def tabletop_states(n: int = 256, n_prims: int = 200, seed: int = 0) -> np.ndarray:
    """uint8 state grid of :func:`tabletop_masks`."""
    occ, unk = tabletop_masks(n, n_prims, seed)
    return states_from_masks(occ, unk)


def probabilities_from_masks(occupied: np.ndarray, unknown: np.ndarray, seed: int) -> np.ndarray:
    """FP32 occupancy probabilities: unknown 0.5, free ~ Beta(2, 8), occupied ~ Beta(8, 2).

    Draws are made in FP64 and stored as FP32.
    """
    rng = np.random.default_rng(seed + 0x5EED)
    p = np.empty(occupied.shape, dtype=np.float64)
    free = ~occupied
    p[free] = rng.beta(2.0, 8.0, size=int(free.sum()))
    p[occupied] = rng.beta(8.0, 2.0, size=int(occupied.sum()))
    p[unknown] = 0.5
    return p.astype(np.float32)


def tabletop_probabilities(n: int = 256, n_prims: int = 200, seed: int = 0) -> np.ndarray:
    """FP32 probability grid of the cluttered tabletop."""
    occ, unk = tabletop_masks(n, n_prims, seed)
    return probabilities_from_masks(occ, unk, seed)


def room_states(n: int = 512, n_prims: int = 2000, unknown_frac: float = 0.4, seed: int = 0) -> np.ndarray:
    """Room: floor, four walls, ``n_prims`` furniture primitives, ~``unknown_frac`` unknown.

    Primitives (boxes, spheres, vertical cylinders, 4-40 voxels) stand on the
    floor or float (shelves).  Unknown space is a union of random boxes (edges
    n/16 .. n/3) added until the unknown fraction reaches ``unknown_frac``; it
    overrides free and occupied.
    """
    rng = np.random.default_rng(seed)
    occ = np.zeros((n, n, n), dtype=bool)
    w = max(2, n // 128)
    occ[:w] = True
    occ[:, :w] = True
    occ[:, -w:] = True
    occ[:, :, :w] = True
    occ[:, :, -w:] = True
    for _ in range(n_prims):
        size = rng.uniform(4.0, 40.0, size=3)
        px, py = rng.uniform(w, n - w, size=2)
        base = w if rng.random() < 0.6 else rng.uniform(w, n * 0.7)
        kind = rng.integers(3)
        if kind == 0:
            fill_box(occ, (px - size[0] / 2, py - size[1] / 2, base), (px + size[0] / 2, py + size[1] / 2, base + size[2]))
        elif kind == 1:
            r = size[0] / 2
            fill_sphere(occ, (px, py, base + r), r)
        else:
            fill_cylinder_z(occ, (px, py), size[0] / 2, base, base + size[2])
    unk = np.zeros_like(occ)
    total = float(n) ** 3
    covered = 0
    while covered < unknown_frac * total:
        e = rng.uniform(n / 16.0, n / 3.0, size=3)
        lo = rng.uniform(0.0, n, size=3) - e / 2
        x0, x1 = _centre_range(lo[0], lo[0] + e[0], n)
        y0, y1 = _centre_range(lo[1], lo[1] + e[1], n)
        z0, z1 = _centre_range(lo[2], lo[2] + e[2], n)
        sub = unk[z0:z1, y0:y1, x0:x1]
        covered += int(sub.size - np.count_nonzero(sub))
        sub[...] = True
    return states_from_masks(occ, unk)
