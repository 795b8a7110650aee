"""Full-size workloads in the benchmark's launch configuration, checked on
sampled outputs the oracle computes one by one (GPU required)."""

import numpy as np
import pytest
import torch

import oracle
import paper_2503_22588_gb300 as nbt
from gpu_util import RTOL, gpu_camera, gpu_map, oracle_camera, oracle_map, rel_err
from workload import configs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    nbt.build()
    oracle.build()


def _check_sample(w, ig, st, sample, walk="f32"):
    om = oracle_map(w)
    rig, rst = oracle.views_ig(om, w.poses[sample], oracle_camera(w.camera), oracle.params(w.metric), walk, 16)
    if walk == "f32":
        assert np.array_equal(st[sample], rst)
    if w.metric == "count" and walk == "f32":
        assert np.array_equal(ig[sample], rig)
    assert np.all(rel_err(ig[sample], rig) <= RTOL), rel_err(ig[sample], rig).max()


def test_prob256_full_size_sampled():
    """256^3 FP32 tabletop, 1024 views x 160 x 120 rays, entropy: 16 sampled views."""
    w = configs.prob256(seed=0)
    gm = gpu_map(w)
    p = torch.from_numpy(w.poses).cuda()
    ig, st = nbt.views_ig(gm, p, gpu_camera(w.camera), nbt.ig_params("entropy"))
    ig = ig.cpu().numpy().astype(np.float64)
    st = st.cpu().numpy()
    assert np.all(np.isfinite(ig)) and np.all(ig >= 0) and st.min() > 0
    sample = np.random.default_rng(0).choice(len(w.poses), 16, replace=False)
    _check_sample(w, ig, st, sample, "f32")
    _check_sample(w, ig, st, sample[:6], "f64")


def test_room512_full_size_sampled():
    """512^3 2-bit room, 8 PoIs x 4096 views x 320 x 240 rays: 6 sampled views."""
    w = configs.room512(seed=0)
    gm = gpu_map(w)
    p = torch.from_numpy(w.poses).cuda()
    ig, st = nbt.views_ig(gm, p, gpu_camera(w.camera), nbt.ig_params("count"))
    ig = ig.cpu().numpy().astype(np.float64)
    st = st.cpu().numpy()
    sample = np.random.default_rng(1).choice(len(w.poses), 6, replace=False)
    _check_sample(w, ig, st, sample, "f32")


def test_traj256_full_size_sampled():
    """512 trajectories (5-40 poses) x 128 x 96 rays on a 256^3 map: 12 sampled trajectories."""
    w = configs.traj256(seed=0)
    gm = gpu_map(w)
    tig = nbt.traj_ig(gm, torch.from_numpy(w.poses).cuda(), torch.from_numpy(w.offsets).cuda(),
                      gpu_camera(w.camera), nbt.ig_params("count"))
    tig = tig.cpu().numpy().astype(np.float64)
    om = oracle_map(w)
    for t in np.random.default_rng(2).choice(len(w.offsets) - 1, 12, replace=False):
        b, e = w.offsets[t], w.offsets[t + 1]
        rig, _ = oracle.views_ig(om, w.poses[b:e], oracle_camera(w.camera), oracle.params("count"), "f32", 16)
        assert rel_err(tig[t], rig.sum()) <= 1e-6, t


def test_room512_pruned_selection_full_size_sampled():
    """The headline selection in the benchmark's configuration: nbt_plan_pruned over one 512^3 2-bit room,
    8 PoIs x 4096 candidates of 320 x 240 rays, the top 205 per PoI re-scored exactly (8 network batches of
    4096, crops beside the forward).  Kept indices = the per-PoI top 205 of the network's scores; each PoI's
    reported IG = the oracle's exact IG of the reported view and the largest exact IG among its kept views;
    3 more kept views per PoI against the oracle."""
    from paper_2503_22588_gb300 import planning as P
    from paper_2503_22588_gb300 import surrogate as gs
    w = configs.room512(seed=0)
    gm = gpu_map(w)
    pz = torch.from_numpy(w.poses).cuda()
    cam = gpu_camera(w.camera)
    prm = nbt.ig_params("count")
    net = gs.Surrogate(max_batch=4096, params=gs.he_init(0), target_scale=P.TARGET_SCALE)
    seg, keep = 4096, 205
    best, val, kept = P.pruned_best(net, gm, pz, seg, keep, cam, prm)
    scores = P.surrogate_scores(net, gm, pz, cam, prm)
    idx, _ = P.segment_topk(scores, seg, keep)
    assert torch.equal(kept, idx)
    kept_np = kept.cpu().numpy()
    best_np = best.cpu().numpy()
    val_np = val.cpu().numpy().astype(np.float64)
    ig_k, _ = nbt.views_ig(gm, pz[kept.reshape(-1).long()].contiguous(), cam, prm)
    ig_k = ig_k.cpu().numpy().astype(np.float64).reshape(kept_np.shape)
    for s in range(len(best_np)):
        assert best_np[s] in kept_np[s] and s * seg <= best_np[s] < (s + 1) * seg
        assert val_np[s] == ig_k[s].max()
    om = oracle_map(w)
    rig, _ = oracle.views_ig(om, w.poses[best_np], oracle_camera(w.camera), oracle.params("count"), "f32", 16)
    assert np.array_equal(val_np, rig)
    rng = np.random.default_rng(3)
    cols = rng.choice(keep, 3, replace=False)
    sample = kept_np[:, cols].reshape(-1)
    rig2, _ = oracle.views_ig(om, w.poses[sample], oracle_camera(w.camera), oracle.params("count"), "f32", 16)
    assert np.array_equal(ig_k[:, cols].reshape(-1), rig2)
    net.close()
    gm.close()
