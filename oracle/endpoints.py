"""CPU oracle of the paper's endpoint-grid density -- TEST INFRASTRUCTURE, NOT PRODUCT CODE.

Section III "Endpoint Calculation": the far plane at d_Cam spans
[-d_h, d_h] x [-d_v, d_v], d_h = d_Cam tan(FoV_h / 2), d_v = d_Cam tan(FoV_v / 2);
the four border rays bound the endpoint grid, and the grid spacing is the
voxel size s_Vox scaled by the grid factor s_G.

Reading (the paper gives the spacing, not the count): the grid keeps its
corner rays and spaces W points evenly from -d_h to d_h, with W the largest
count whose spacing 2 d_h / (W - 1) is not finer than s_G s_Vox, i.e.
W = floor(2 d_h / (s_G s_Vox)) + 1, and at least 2 (the corners); H likewise
with d_v.  N_E = W H.  Evaluated in FP64 from the FP32 parameters, as
(2 d_h) / (s_G s_Vox), so both sides take the integer decision alike.
"""

from __future__ import annotations

import math

import numpy as np


def grid_size(fov_h, fov_v, d_cam, s_vox, s_g):
    """(W, H) of the endpoint grid for grid factor s_G."""
    f = lambda v: float(np.float32(v))  # noqa: E731  (the parameters arrive as FP32)
    step = f(s_g) * f(s_vox)
    out = []
    for fov in (fov_h, fov_v):
        half = f(d_cam) * math.tan(f(fov) * 0.5)
        out.append(max(2, int(math.floor((2.0 * half) / step)) + 1))
    return tuple(out)
