"""What the trained surrogate gains over the method without it (GPU required).

The pruned planner raycasts only the surrogate's top candidates per PoI and takes the best of them.
At the same exact budget (the same number of raycast views per PoI) it is compared with three ways
of choosing which candidates to raycast without the trained network:

* Eq. 3 (paper Section IV): half of the budget raycast at random candidates and pushed as one
  information distribution, G(x) evaluated at the other candidates, its top half raycast;
* the same network before training (He-initialised weights);
* random candidates.

The network is trained here with the library's own kernels on exact labels of seeded rooms and
evaluated on held-out rooms.  The trained network must find the exact best view more often than
each alternative, and lose less IG when it misses (mean regret 1 - chosen IG / best IG).  With
keep = all candidates the pruned planner must reproduce exact scoring.
"""

import math

import numpy as np
import pytest
import torch

import paper_2503_22588_gb300 as nbt
from paper_2503_22588_gb300 import planning as P, surrogate as gs
from workload import poses as wp, scenes

pytestmark = pytest.mark.gpu

N, VIEWS, KEEP = 128, 1024, 51           # 128^3 rooms, 1024 candidates per PoI, keep 5 %


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    nbt.build()


def room(seed):
    g = scenes.room_states(N, 120, 0.4, seed=seed)
    rng = np.random.default_rng(seed + 1)
    pois = rng.uniform(0.35, N * 0.01 - 0.35, size=(4, 3))
    pz = np.concatenate([wp.shell_views(p, VIEWS, 0.3, 0.8, seed * 10 + k) for k, p in enumerate(pois)])
    m = nbt.Map.from_grid(torch.from_numpy(g).cuda(), 0.01, (0.0, 0.0, 0.0), "u2")
    return m, torch.from_numpy(pz).cuda()


def test_trained_surrogate_beats_eq3_untrained_and_random_at_the_same_exact_budget():
    cam = nbt.camera(64, 48, math.radians(60), math.radians(45), 1.0)
    prm = nbt.ig_params("count")
    train = [room(100 + s) for s in range(10)]
    targets = [P.label_views(m, pz, cam, prm) for m, pz in train]
    net = gs.Surrogate(max_batch=1024, params=gs.he_init(0), target_scale=P.TARGET_SCALE)
    losses = P.train(net, [m for m, _ in train], [pz for _, pz in train], targets, cam, prm, epochs=8, lr=1e-3,
                     batch=256)
    assert losses[-1] < 0.5 * losses[0], losses
    for m, _ in train:
        m.close()
    net0 = gs.Surrogate(max_batch=1024, params=gs.he_init(0))
    k1 = KEEP // 2
    k2 = KEEP - k1
    buf = nbt.IdBuffer(n_b=1, max_views=k1)
    agree = {"trained": 0, "eq3": 0, "untrained": 0, "random": 0}
    regret = {k: [] for k in agree}
    cases = 0
    for s in range(8):
        m, pz = room(500 + s)
        ig, _ = nbt.views_ig(m, pz, cam, prm, want_steps=False)
        bx, vx = P.segment_argmax(ig, VIEWS)
        # keep = all: exactly the exact choice
        ba, va, _ = P.pruned_best(net, m, pz, VIEWS, VIEWS, cam, prm)
        assert torch.equal(ba, bx) and torch.equal(va, vx)
        picks = {}
        picks["trained"], _, _ = P.pruned_best(net, m, pz, VIEWS, KEEP, cam, prm)
        picks["untrained"], _, _ = P.pruned_best(net0, m, pz, VIEWS, KEEP, cam, prm)
        rs = torch.from_numpy(np.random.default_rng(700 + s).random(len(pz), dtype=np.float32)).cuda()
        idx_r, kept_r = P.segment_topk(rs, VIEWS, KEEP, pz)
        ig_r, _ = nbt.views_ig(m, kept_r, cam, prm, want_steps=False)
        picks["random"], _ = P.segment_argmax(ig_r, KEEP, idx_r.reshape(-1).contiguous())
        idx_1, kept_1 = P.segment_topk(rs, VIEWS, k1, pz)
        ig_1, _ = nbt.views_ig(m, kept_1, cam, prm, want_steps=False)
        g = torch.empty(len(pz), dtype=torch.float32, device="cuda")
        for q in range(len(pz) // VIEWS):
            buf.push(kept_1[q * k1:(q + 1) * k1], ig_1[q * k1:(q + 1) * k1])
            nbt.idw_gain(buf, pz[q * VIEWS:(q + 1) * VIEWS], 2.0, g[q * VIEWS:(q + 1) * VIEWS])
        g.index_fill_(0, idx_1.reshape(-1).long(), float("-inf"))
        idx_2, kept_2 = P.segment_topk(g, VIEWS, k2, pz)
        ig_2, _ = nbt.views_ig(m, kept_2, cam, prm, want_steps=False)
        nq = len(pz) // VIEWS
        vals = torch.cat([ig_1.view(nq, k1), ig_2.view(nq, k2)], 1).reshape(-1).contiguous()
        idxs = torch.cat([idx_1, idx_2], 1).reshape(-1).contiguous()
        picks["eq3"], _ = P.segment_argmax(vals, KEEP, idxs)
        best = vx.cpu().numpy().astype(np.float64)
        igh = ig.cpu().numpy().astype(np.float64)
        for k, b in picks.items():
            agree[k] += int((b == bx).sum().item())
            regret[k].extend(list(1.0 - igh[b.cpu().numpy()] / np.maximum(best, 1.0)))
        cases += len(bx)
        m.close()
    buf.close()
    net0.close()
    net.close()
    mean_regret = {k: float(np.mean(v)) for k, v in regret.items()}
    print("same best view:", {k: f"{v}/{cases}" for k, v in agree.items()}, "mean regret:", mean_regret)
    for k in ("eq3", "untrained", "random"):
        assert agree["trained"] > agree[k], (agree, mean_regret)
        assert mean_regret["trained"] < mean_regret[k], (agree, mean_regret)
