"""Pins of the endpoint-grid density oracle (no GPU): hand-computed grids and
a brute-force search for the densest grid not finer than s_G s_Vox."""

import math

import numpy as np

from oracle import endpoints as E


def test_hand_computed_grids():
    fh, fv = math.radians(60), math.radians(45)
    # 2 tan(30 deg) = 1.1547 m, 2 tan(22.5 deg) = 0.8284 m at d_Cam = 1 m
    assert E.grid_size(fh, fv, 1.0, 0.01, 5) == (24, 17)       # 5 cm: floor(23.09) + 1, floor(16.57) + 1
    assert E.grid_size(fh, fv, 1.0, 0.01, 1) == (116, 83)      # 1 cm: floor(115.47) + 1, floor(82.84) + 1
    assert E.grid_size(fh, fv, 1.0, 0.01, 100) == (2, 2)       # 1 m: only the corner rays
    assert E.grid_size(fh, fv, 1.0, 0.01, 50) == (3, 2)        # 0.5 m: floor(2.31) + 1, floor(1.66) + 1
    assert E.grid_size(fh, fv, 3.0, 0.01, 20) == (18, 13)      # 3.464 m / 0.2 m, 2.485 m / 0.2 m


def test_densest_grid_not_finer_than_the_step_by_search():
    rng = np.random.default_rng(0)
    for _ in range(300):
        fh, fv = rng.uniform(0.2, 2.5, 2)
        d = rng.uniform(0.2, 5.0)
        sv = rng.choice([0.005, 0.01, 0.02])
        sg = rng.uniform(1.0, 300.0)
        w, h = E.grid_size(fh, fv, d, sv, sg)
        step = float(np.float32(sg)) * float(np.float32(sv))
        for n, fov in ((w, fh), (h, fv)):
            span = 2.0 * float(np.float32(d)) * math.tan(float(np.float32(fov)) * 0.5)
            best = 2
            k = 2
            while span / (k - 1) >= step:       # spacing of k points not finer than the step
                best = k
                k += 1
            assert n == best, (fh, fv, d, sv, sg, n, best)
