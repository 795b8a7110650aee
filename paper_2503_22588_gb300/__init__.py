"""GB300-native information-gain raycasting for Next-Best-Trajectory planning.

The hot path of the paper's Section III (Online Local Information
Distribution) as hand-written sm_103a CUDA kernels behind a C ABI
(``include/nbt.h``, ``libnbt.so``); this package is the Python binding.
"""

from ._lib import LibraryMissing, NbtError, lib  # noqa: F401
from .api import (Map, TrajPlan, camera, camera_from_grid_scale, ig_params, trace_segments, traj_ig, view_segments,  # noqa: F401
                  views_ig, views_ig_noalloc, workspace, workspace_size)
from .autotune import autotune  # noqa: F401
from . import surrogate  # noqa: F401
from .idw import IdBuffer, idw_gain, ig_cost  # noqa: F401
from .build import LIB_PATH, build  # noqa: F401
