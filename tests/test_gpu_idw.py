"""IG interpolation (Eq. 3), orientation factor and c_I on the GPU against the
FP64 oracle (GPU required).

Bars (derived in the design notes from the arithmetic): G and the cost
terms within 1e-5 relative for p = 2 (2e-5 for other p); O within 2e-6
relative, and zero exactly where the oracle's FP32 field-of-view decision
says outside.
"""

import math

import numpy as np
import pytest
import torch

import paper_2503_22588_gb300 as nbt
from oracle import idw as I
from workload import configs, poses

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    nbt.build()


def make_id(n, seed, poi=(0.5, 0.4, 0.3)):
    pz = poses.ball_views(np.asarray(poi), n, 1.0, seed) if n else np.zeros((0, 7), np.float32)
    g = configs.id_gains(pz[:, :3].astype(np.float64), poi, seed + 7) if n else np.zeros(0, np.float32)
    return pz, g


def push_all(buf, ids):
    for pz, g in ids:
        buf.push(torch.from_numpy(pz).cuda(), torch.from_numpy(g).cuda())


def oracle_ids(ids):
    return [(pz[:, :3].astype(np.float64), g.astype(np.float64)) for pz, g in ids]


def rel(a, b):
    return np.abs(np.asarray(a, np.float64) - b) / np.maximum(np.abs(b), 1e-30)


def queries(n, seed, poi=(0.5, 0.4, 0.3)):
    return poses.ball_views(np.asarray(poi), n, 1.2, seed)


@pytest.mark.parametrize("sizes", [[1], [63, 64, 65], [500, 0, 1000, 7], [130] * 12])
def test_idw_gain_matches_oracle(sizes):
    ids = [make_id(n, 100 + k) for k, n in enumerate(sizes)]
    buf = nbt.IdBuffer(10, 1024)
    push_all(buf, ids)
    assert len(buf) == min(len(sizes), 10)
    q = queries(257, 5)
    got = nbt.idw_gain(buf, torch.from_numpy(q).cuda()).cpu().numpy()
    kept = oracle_ids(ids)[-10:]
    want = np.array([I.id_buffer_gain(x[:3].astype(np.float64), kept, 10) for x in q])
    assert rel(got, want).max() <= 1e-5, rel(got, want).max()
    buf.close()


@pytest.mark.parametrize("p", [1.0, 3.0, 0.5])
def test_idw_gain_other_powers(p):
    ids = [make_id(n, 200 + n) for n in (300, 77)]
    buf = nbt.IdBuffer(4, 512)
    push_all(buf, ids)
    q = queries(129, 6)
    got = nbt.idw_gain(buf, torch.from_numpy(q).cuda(), power=p).cpu().numpy()
    want = np.array([I.id_buffer_gain(x[:3].astype(np.float64), oracle_ids(ids), 4, p) for x in q])
    assert rel(got, want).max() <= 2e-5, rel(got, want).max()
    buf.close()


def test_coincident_queries_take_the_mean():
    pz, g = make_id(200, 11)
    pz = np.concatenate([pz, pz[:3]])          # perspectives 200..202 repeat 0..2 with other gains
    g = np.concatenate([g, np.array([1.0, 2.0, 3.0], np.float32)])
    buf = nbt.IdBuffer(3, 256)
    push_all(buf, [(pz, g)])
    q = np.concatenate([pz[[0, 1, 2, 50]], queries(4, 3)]).astype(np.float32)
    got = nbt.idw_gain(buf, torch.from_numpy(q).cuda()).cpu().numpy()
    want = np.array([I.id_buffer_gain(x[:3].astype(np.float64), oracle_ids([(pz, g)]), 3) for x in q])
    assert abs(got[0] - (g[0] + 1.0) / 2) <= 1e-6 * abs(got[0])
    assert got[3] == g[50]
    assert rel(got, want).max() <= 1e-5
    buf.close()


def test_large_power_near_points_use_the_fp64_path():
    pz, g = make_id(100, 12)
    q = pz[:8].copy()
    q[:, 0] += np.float32(1e-5)                 # 10 um from a start point: d^-8 = 1e40 overflows FP32
    buf = nbt.IdBuffer(2, 128)
    push_all(buf, [(pz, g)])
    got = nbt.idw_gain(buf, torch.from_numpy(q).cuda(), power=8.0).cpu().numpy()
    want = np.array([I.id_buffer_gain(x[:3].astype(np.float64), oracle_ids([(pz, g)]), 2, 8.0) for x in q])
    assert np.all(np.isfinite(got))
    assert rel(got, want).max() <= 2e-5, (got, want)
    buf.close()


def test_ring_drops_the_oldest_and_clear_empties():
    ids = [make_id(50 + 10 * k, 300 + k) for k in range(7)]
    buf = nbt.IdBuffer(3, 128)
    q = torch.from_numpy(queries(33, 9)).cuda()
    for k in range(7):
        push_all(buf, [ids[k]])
        got = nbt.idw_gain(buf, q).cpu().numpy()
        kept = oracle_ids(ids[max(0, k - 2):k + 1])
        want = np.array([I.id_buffer_gain(x[:3].astype(np.float64), kept, 3) for x in q.cpu().numpy()])
        assert rel(got, want).max() <= 1e-5, k
    buf.clear()
    assert len(buf) == 0
    assert np.all(nbt.idw_gain(buf, q).cpu().numpy() == 0.0)
    buf.close()


def _cost_case(n_traj, horizon, seed, n_ids=4, n_p=300):
    poi = np.array([0.5, 0.4, 0.3], np.float32)
    ids = [make_id(n_p + 13 * k, 400 + k, poi) for k in range(n_ids)]
    from workload import trajectories
    ps, off = trajectories.horizon_trajectories(poi, n_traj, horizon, seed, jitter_deg=40.0)
    return poi, ids, ps, off


@pytest.mark.parametrize("w_info", [1.0, 0.25])
def test_ig_cost_matches_oracle(w_info):
    poi, ids, ps, off = _cost_case(40, 31, 1)
    fh, fv = float(np.float32(math.radians(60))), float(np.float32(math.radians(45)))
    buf = nbt.IdBuffer(10, 512)
    push_all(buf, ids)
    cost, g, o, term = nbt.ig_cost(buf, torch.from_numpy(ps).cuda(), torch.from_numpy(off).cuda(), poi, fh, fv,
                                   w_info=w_info, want_parts=True)
    G, O, C = I.ig_cost(ps, off, poi.astype(np.float64), fh, fv, oracle_ids(ids), 10, 2.0, w_info)
    g, o, term, cost = (x.cpu().numpy() for x in (g, o, term, cost))
    assert rel(g, G).max() <= 1e-5
    outside = O == 0.0
    assert outside.any() and (~outside).any()
    assert np.all(o[outside] == 0.0)
    assert rel(o[~outside], O[~outside]).max() <= 2e-6
    T = w_info / (O * G + 1e-7)
    assert rel(term, T).max() <= 1e-5
    assert rel(cost, C).max() <= 1e-5
    buf.close()


def test_ig_cost_ragged_offsets_and_empty_trajectories():
    poi, ids, ps, off = _cost_case(12, 9, 2)
    off = np.array([0, 0, 5, 5, 40, 108, 108], np.int32)   # empty, short, empty, long trajectories
    fh, fv = math.radians(60), math.radians(45)
    buf = nbt.IdBuffer(4, 512)
    push_all(buf, ids)
    cost = nbt.ig_cost(buf, torch.from_numpy(ps).cuda(), torch.from_numpy(off).cuda(), poi, fh, fv).cpu().numpy()
    _, _, C = I.ig_cost(ps, off, poi.astype(np.float64), float(np.float32(fh)), float(np.float32(fv)),
                        oracle_ids(ids), 4)
    assert cost[0] == 0.0 and cost[2] == 0.0 and cost[5] == 0.0
    assert rel(cost, C)[[1, 3, 4]].max() <= 1e-5
    buf.close()


def test_fullsize_cost_workload_sampled():
    """The benchmark's workload (10 IDs x 500, 16,384 x 31 states) in the benchmark's launch; sampled checks."""
    w = configs.idw_cost()
    buf = nbt.IdBuffer(w.n_b, 512)
    push_all(buf, w.ids)
    pz = torch.from_numpy(w.poses).cuda()
    cost, g, o, term = nbt.ig_cost(buf, pz, torch.from_numpy(w.offsets).cuda(), w.poi, w.fov_h, w.fov_v,
                                   want_parts=True)
    torch.cuda.synchronize()
    rng = np.random.default_rng(0)
    trajs = rng.choice(len(w.offsets) - 1, 24, replace=False)
    kept = oracle_ids(w.ids)
    for t in trajs:
        a, b = w.offsets[t], w.offsets[t + 1]
        G, O, C = I.ig_cost(w.poses[a:b], [0, b - a], w.poi.astype(np.float64), w.fov_h, w.fov_v, kept, w.n_b)
        assert rel(g[a:b].cpu().numpy(), G).max() <= 1e-5
        assert np.all((o[a:b].cpu().numpy() == 0.0) == (O == 0.0))
        assert rel(cost[t].item(), C[0]) <= 1e-5
    # properties over every state: G within the gain range times the buffer's harmonic weight sum
    gmax = max(float(x[1].max()) for x in w.ids)
    h = sum(1.0 / k for k in range(1, w.n_b + 1))
    gg = g.cpu().numpy()
    assert np.all(gg >= 0.0) and np.all(gg <= gmax * h * (1 + 1e-5))
    assert np.all(np.isfinite(cost.cpu().numpy()))
    buf.close()


def test_invalid_arguments():
    from paper_2503_22588_gb300 import NbtError
    with pytest.raises(NbtError):
        nbt.IdBuffer(0, 10)
    with pytest.raises(NbtError):
        nbt.IdBuffer(33, 10)
    buf = nbt.IdBuffer(2, 16)
    pz, g = make_id(17, 1)
    with pytest.raises(NbtError):
        push_all(buf, [(pz, g)])                    # more than max_views
    q = torch.from_numpy(queries(4, 1)).cuda()
    for p in (0.0, -1.0, 9.0, float("nan")):
        with pytest.raises(NbtError):
            nbt.idw_gain(buf, q, power=p)
    off = torch.tensor([0, 4], dtype=torch.int32, device="cuda")
    with pytest.raises(NbtError):
        nbt.ig_cost(buf, q, off, (0, 0, 0), 0.0, 1.0)
    with pytest.raises(NbtError):
        nbt.ig_cost(buf, q, off, (0, 0, 0), 1.0, 1.0, eps=0.0)
    with pytest.raises(NbtError):
        nbt.ig_cost(buf, q, off, (0, 0, 0), 1.0, 1.0, w_info=-1.0)
    assert nbt.idw_gain(buf, q[:0]).numel() == 0
    buf.close()
