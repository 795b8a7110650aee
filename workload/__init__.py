"""Seeded synthetic inputs for the IG raycasting path.

This package only *generates inputs*: voxel scenes (dense, x-fastest grids),
camera poses and trajectories.  It holds none of the information-gain
arithmetic (no ray generation, traversal or gain).  Both the CPU oracle and
the CUDA library consume what it produces, so that the two sides see the
same bytes.

Layout convention for every grid returned here: a C-contiguous numpy array of
shape ``(nz, ny, nx)``; the linear voxel index is ``(z * ny + y) * nx + x``
(x fastest).  Voxel ``(x, y, z)`` covers ``[origin + x*s, origin + (x+1)*s)``
along x, and likewise for y and z.  State grids use ``0 = unknown``,
``1 = free``, ``2 = occupied``.
"""

from . import scenes, poses, trajectories, configs  # noqa: F401

UNKNOWN, FREE, OCCUPIED = 0, 1, 2
