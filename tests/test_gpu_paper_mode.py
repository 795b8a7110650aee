"""The paper-exact perspective mode on the GPU against the oracle: Eq. 1
perspectives in a ball around the PoI, the endpoint grid of grid factor s_G
(Section III), Eq. 2 on a probability map, mean per perspective (GPU required)."""

import math

import numpy as np
import pytest
import torch

import oracle
import paper_2503_22588_gb300 as nbt
from oracle.endpoints import grid_size
from workload import poses, scenes

from gpu_util import RTOL, rel_err, views_gpu

pytestmark = pytest.mark.gpu
TIE = 1e-6   # parameter gap below which the FP32 and exact walks may order two crossings differently


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    nbt.build()


@pytest.mark.parametrize("s_g", [1, 5, 20, 100])
def test_grid_scale_ids_match_the_oracle(s_g):
    n, vs = 64, 0.01
    grid = scenes.tabletop_probabilities(n, 20, 3)
    poi = np.full(3, n * vs / 2)
    ps = poses.ball_views(poi, 40, 0.3, 7)                     # Eq. 1, r_S = 0.3 m
    fh, fv, d = math.radians(60), math.radians(45), 0.5
    cam = nbt.camera_from_grid_scale(fh, fv, d, vs, s_g)
    assert (cam.width, cam.height) == grid_size(fh, fv, d, vs, s_g)
    m = nbt.Map.from_grid(torch.from_numpy(grid).cuda(), vs)
    ig, st = views_gpu(m, ps, cam, nbt.ig_params("eq2", reduce="mean"))
    ocam = oracle.camera(cam.width, cam.height, fh, fv, d)
    om = oracle.Map(grid, vs, (0.0, 0.0, 0.0))
    rig, rst = oracle.views_ig(om, ps, ocam, oracle.params("eq2", reduce="mean"), "f32", 4)
    xig, _ = oracle.views_ig(om, ps, ocam, oracle.params("eq2", reduce="mean"), "f64", 4)
    assert np.array_equal(st, rst)
    assert rel_err(ig, rig).max() <= RTOL
    # Against the exact FP64 walk: with few rays per view one FP32 tie flip
    # (a ray within ~1 ulp of a voxel edge or corner) moves the mean past the
    # bar; such a view is accepted only where the oracle shows that tie.
    bad = np.nonzero(rel_err(ig, xig) > RTOL)[0]
    assert len(bad) <= 0.1 * len(ps)
    dims = (n, n, n)
    for v in bad:
        o, dd = oracle.view_rays(om, ocam, ps[v])
        diff = [k for k in range(len(o))
                if not np.array_equal(oracle.trace(dims, o[k], dd[k], "f32"), oracle.trace(dims, o[k], dd[k], "f64"))]
        assert diff, v
        assert all(oracle.min_tie_gap(dims, o[k], dd[k]) < TIE for k in diff), v
    assert np.all(ig > 0)
    m.close()
