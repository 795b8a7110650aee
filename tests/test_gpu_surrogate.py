"""The learned surrogate's CUDA kernels against the FP64 oracle (GPU required).

Crops: the class codes byte-exact (the oracle's one-hot crops, coded).

Exact arithmetic: with parameters and inputs chosen so that every value the GPU stores in BF16 is
exactly representable and every FP32 sum is exact (integer weights in {-1, 0, 1}, integer biases,
dyadic loss residuals; the premise is checked with the oracle), the forward predictions, the loss
and every element of every gradient equal the FP64 oracle bit for bit.  A wrong tap, index,
transpose, mask or dropped term anywhere in the tcgen05 kernels fails this test, whatever its size.

Realistic parameters (He initialisation): the oracle is evaluated with the same BF16 roundings as
the GPU (weights, forward activations, and in the backward pass the hidden gradient and every
masked input gradient), so the remaining differences come from FP32-vs-FP64 accumulation and the
rare BF16 rounding flips it causes.  Forward: per element within one BF16 rounding unit (2^-8) of
the sum of the absolute terms of the output layer's dot product.  Gradients: relative L2 error per
tensor <= 1e-2.  Adam: the update the oracle computes from the GPU's gradients, to FP32 precision.
"""

import ctypes as C
import math

import numpy as np
import pytest
import torch

import paper_2503_22588_gb300 as nbt
from oracle import surrogate as S
from paper_2503_22588_gb300 import _lib
from paper_2503_22588_gb300 import surrogate as gs
from workload import configs, poses, scenes

pytestmark = pytest.mark.gpu

BF16_WEIGHTS = ("w0", "w1", "w2", "w3", "f1")


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    nbt.build()


def no_device_timeout():
    f = C.c_int32()
    assert _lib.lib().nbt_tc_error(C.byref(f)) == 0
    return f.value == 0


def as_used_by_gpu(p):
    """The parameters as the GPU uses them: BF16 weights, FP32 biases and f2."""
    q = {k: np.asarray(v, np.float64) for k, v in p.items()}
    for k in BF16_WEIGHTS:
        q[k] = S._bf16(p[k])
    return q


def small_scene(enc, seed=0, n=48):
    grid = scenes.boxes_spheres(n, 30, seed, size_range=(2.0, 10.0), half_unknown=True)
    if enc == "f32":
        occ = grid == 2
        unk = grid == 0
        grid = scenes.probabilities_from_masks(occ, unk, seed)
    poi = np.full(3, n * 0.005)
    p = poses.shell_views(poi, 8, 0.1, 0.3, seed)
    return grid, p


def rel_l2(a, b):
    a = np.asarray(a, np.float64).ravel()
    b = np.asarray(b, np.float64).ravel()
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-30))


@pytest.mark.parametrize("enc,brick", [(e, b) for e in ("u8", "u2", "f32") for b in (1, 8)])
def test_crops_bitexact(enc, brick):
    """Linear layout (offsets computed) and 8^3 bricks (offsets from the tables)."""
    grid, p = small_scene(enc, seed=3)
    cam = nbt.camera(64, 48, math.radians(60), math.radians(45), 0.5)
    prm = nbt.ig_params("count" if enc != "f32" else "entropy")
    m = nbt.Map.from_grid(torch.from_numpy(grid).cuda(), 0.01, (0.0, 0.0, 0.0), enc, brick)
    cr, ft = gs.crops(m, torch.from_numpy(p).cuda(), cam, prm)
    assert cr.dtype == torch.uint8 and cr.shape == (len(p), 32, 32, 32)
    cr = cr.cpu().numpy()
    ft = ft.float().cpu().numpy()
    cc = S.crop_consts(math.radians(60), math.radians(45), 0.5)
    for v in range(3):
        oc, of = S.frustum_crop(grid, 0.01, (0, 0, 0), p[v], cc)
        assert np.array_equal(cr[v], S.crop_codes(oc)), v
        assert np.array_equal(ft[v], S._bf16(of).astype(np.float32)), v
        assert oc[..., 0].any() and oc[..., 1].any() and (cr[v] == 0).any()


def _batch(n_views=6, seed=2):
    grid, p = small_scene("u8", seed=seed)
    cam = nbt.camera(64, 48, math.radians(60), math.radians(45), 0.5)
    m = nbt.Map.from_grid(torch.from_numpy(grid).cuda(), 0.01)
    pz = torch.from_numpy(np.concatenate([p, p])[:n_views]).cuda()
    return gs.crops(m, pz, cam, nbt.ig_params("count"))


def forward_bar(q, cache):
    """Per-prediction bar: one BF16 rounding unit (2^-8) of sum_j |h1_j f2_j| (the output layer's
    absolute terms, h1 as the GPU stores it), plus FP32 accumulation of the 128 terms."""
    terms = np.abs(cache["h"]) @ np.abs(np.asarray(q["f2"], np.float64))
    return 2.0 ** -8 * terms + 128 * 2.0 ** -24 * (terms + abs(float(q["g2"][0])))


def check_forward(pred, q, cr, ft):
    y, cache = S.forward(q, S.codes_to_onehot(cr), ft, bf16_activations=True)
    bar = forward_bar(q, cache)
    err = np.abs(pred - y)
    assert np.all(err <= bar), (err, bar)
    return float((err / bar).max())


def test_forward_matches_oracle():
    cr, ft = _batch(6)
    params = S.init_params(1)
    params["b0"] += 0.05
    params["g1"] += 0.02
    net = gs.Surrogate(max_batch=4, params=params)   # 6 samples: two passes
    pred = net.forward(cr, ft).cpu().numpy().astype(np.float64)
    assert no_device_timeout()
    check_forward(pred, as_used_by_gpu(params), cr.cpu().numpy(), ft.float().cpu().numpy())
    net.close()


def test_forward_many_views_matches_oracle_on_a_sample():
    """160 views: more crops than SMs, so the persistent layer-0/1 kernel takes a second crop
    on some CTAs; a sample of first- and second-pass views against the oracle."""
    cr, ft = _batch(4, seed=3)
    cr = cr.repeat(40, 1, 1, 1)                       # 160 crops: 4 scenes' crops, rolled per copy
    for k in range(40):
        cr[4 * k:4 * k + 4] = torch.roll(cr[4 * k:4 * k + 4], shifts=(k % 5, 3 * k % 7, k % 3), dims=(1, 2, 3))
    ft = ft.repeat(40, 1)
    params = S.init_params(4)
    params["b0"] += 0.03
    params["b1"] += 0.03
    net = gs.Surrogate(max_batch=160, params=params)
    pred = net.forward(cr, ft).cpu().numpy().astype(np.float64)
    sample = [0, 1, 77, 151, 152, 155, 159]
    assert no_device_timeout()
    check_forward(pred[sample], as_used_by_gpu(params), cr[sample].cpu().numpy(), ft[sample].float().cpu().numpy())
    assert len(np.unique(np.round(pred, 6))) > 20          # the rolled crops really differ
    net.close()


def test_forward_odd_batch_matches_oracle():
    """7 views in one batch: the last two-crop tile of layers 2-3 has no second crop."""
    cr, ft = _batch(7, seed=11)
    params = S.init_params(6)
    params["b2"] += 0.02
    params["b3"] += 0.02
    net = gs.Surrogate(max_batch=8, params=params)
    pred = net.forward(cr, ft).cpu().numpy().astype(np.float64)
    assert no_device_timeout()
    assert pred.shape == (7,)
    check_forward(pred, as_used_by_gpu(params), cr.cpu().numpy(), ft.float().cpu().numpy())
    net.close()


def test_backward_matches_oracle_gradients():
    """Targets two units below the oracle's predictions, so the residuals y - t carry no
    cancellation: every gradient tensor within 1e-2 relative L2 of the BF16-modelled oracle."""
    cr, ft = _batch(8, seed=5)
    cr = torch.cat([cr, torch.flip(cr, dims=(1,)), torch.flip(cr, dims=(2,)), torch.flip(cr, dims=(3,))])
    ft = ft.repeat(4, 1)
    params = S.init_params(4)
    params["g1"] += 0.05
    q = as_used_by_gpu(params)
    x = S.codes_to_onehot(cr.cpu().numpy())
    y, _ = S.forward(q, x, ft.float().cpu().numpy(), bf16_activations=True)
    t_np = (y - 2.0 - 0.25 * np.arange(len(y)) / len(y)).astype(np.float32)
    net = gs.Surrogate(max_batch=32, params=params)
    t = torch.from_numpy(t_np).cuda()
    loss, grads = net.backward(cr, ft, t)
    torch.cuda.synchronize()
    assert no_device_timeout()
    g = gs.unpack(grads.cpu().numpy())
    oloss, og = S.loss_and_grads(q, x, ft.float().cpu().numpy(), t_np, bf16_activations=True)
    assert abs(loss.item() - oloss) <= 1e-3 * abs(oloss)
    errs = {k: rel_l2(g[k], og[k]) for k in og}
    print("gradient rel. L2 errors:", {k: f"{v:.1e}" for k, v in errs.items()})
    assert max(errs.values()) <= 1e-2, errs
    net.close()


def exact_params(seed, nnz=(0, 5, 4, 3), nnz_f1=5):
    """Parameters in exact arithmetic: weights in {-1, 0, 1} (layer 0: the three live one-hot channels;
    layers 1-3 and fc1: nnz nonzeros per output row), small integer biases, f2 in {-1, 0, 1}."""
    rng = np.random.default_rng(seed)
    p = {}
    w0 = np.zeros((16, 27, 8), np.float32)
    w0[:, :, :3] = rng.choice([-1.0, 0.0, 0.0, 1.0], size=(16, 27, 3))
    p["w0"] = w0.reshape(16, 216)
    p["b0"] = rng.integers(0, 4, 16).astype(np.float32)
    for i, (cin, cout, _) in enumerate(S.LAYERS[1:], 1):
        w = np.zeros((cout, 27 * cin), np.float32)
        for o in range(cout):
            w[o, rng.choice(27 * cin, size=nnz[i], replace=False)] = rng.choice([-1.0, 1.0], size=nnz[i])
        p[f"w{i}"] = w
        p[f"b{i}"] = rng.integers(0, 3, cout).astype(np.float32)
    f1 = np.zeros((128, 4104), np.float32)
    for j in range(128):
        f1[j, rng.choice(4104, size=nnz_f1, replace=False)] = rng.choice([-1.0, 1.0], size=nnz_f1)
    p["f1"] = f1
    p["g1"] = rng.integers(0, 3, 128).astype(np.float32)
    p["f2"] = rng.choice([-1.0, 0.0, 1.0], size=128).astype(np.float32)
    p["g2"] = np.array([float(rng.integers(-3, 4))], np.float32)
    return p


def bf16_exact(a):
    a = np.asarray(a, np.float64)
    return np.array_equal(S._bf16(a), a)


@pytest.mark.parametrize("seed", [0, 3])
def test_exact_arithmetic_forward_loss_and_gradients_are_bitwise(seed):
    cr, _ = _batch(8, seed=5 + seed)
    ft = torch.ones((8, 8), dtype=torch.bfloat16, device="cuda")
    params = exact_params(seed)
    x = S.codes_to_onehot(cr.cpu().numpy())
    q = {k: np.asarray(v, np.float64) for k, v in params.items()}
    y, cache = S.forward(q, x, np.ones((8, 8)))
    # premise: every value the GPU stores in BF16 is exact, the activations are alive
    assert all(bf16_exact(a) for a in cache["acts"]) and bf16_exact(cache["h"])
    assert all(0.2 < float((a > 0).mean()) < 0.9 for a in cache["acts"][1:])
    residual = np.random.default_rng(seed).choice([-2.0, -1.0, 1.0, 2.0], size=8)
    t = y - residual                                     # dy = 2 residual / 8: dyadic
    oloss, og = S.loss_and_grads(q, x, np.ones((8, 8)), t)
    _, og16 = S.loss_and_grads(q, x, np.ones((8, 8)), t, bf16_activations=True)
    assert all(np.array_equal(og[k], og16[k]) for k in og)   # the backward BF16 stores are exact too
    net = gs.Surrogate(max_batch=8, params=params)
    pred = net.forward(cr, ft).cpu().numpy().astype(np.float64)         # fused inference kernels
    loss, grads = net.backward(cr, ft, torch.from_numpy(t.astype(np.float32)).cuda())   # training kernels
    torch.cuda.synchronize()
    assert no_device_timeout()
    assert np.array_equal(pred, y), (pred, y)
    assert loss.item() == oloss
    g = gs.unpack(grads.cpu().numpy())
    for k in og:
        bad = np.flatnonzero(g[k].astype(np.float64).ravel() != og[k].ravel())
        assert bad.size == 0, (k, bad[:8], g[k].ravel()[bad[:8]], og[k].ravel()[bad[:8]])
        assert np.abs(og[k]).max() > 0, k                  # every gradient tensor is exercised
    net.close()


def test_adam_step_matches_oracle_update():
    cr, ft = _batch(8, seed=6)
    params = S.init_params(7)
    net = gs.Surrogate(max_batch=8, params=params)
    t = torch.rand(8, device="cuda", generator=torch.Generator(device="cuda").manual_seed(0))
    _, grads = net.backward(cr, ft, t)
    g = gs.unpack(grads.cpu().numpy())
    net.train_step(cr, ft, t, lr=1e-3)
    got = net.get_params()
    zeros = {k: np.zeros_like(v, np.float64) for k, v in params.items()}
    want, _, _ = S.adam(params, g, zeros, zeros, 1, lr=1e-3)
    for k in params:
        assert np.allclose(got[k], want[k], rtol=1e-5, atol=1e-7), k
    net.close()


def test_training_reduces_the_loss():
    cr, ft = _batch(32, seed=8)
    net = gs.Surrogate(max_batch=32, params=S.init_params(9))
    t = torch.rand(32, device="cuda", generator=torch.Generator(device="cuda").manual_seed(1))
    first = net.backward(cr, ft, t)[0].item()
    for _ in range(60):
        net.train_step(cr, ft, t, lr=1e-3)
    last = net.backward(cr, ft, t)[0].item()
    assert no_device_timeout()
    assert last < 0.5 * first, (first, last)
    net.close()


def test_segment_topk_and_argmax_match_numpy():
    from paper_2503_22588_gb300 import planning as P
    g = torch.Generator(device="cuda").manual_seed(3)
    for seg, keep in ((4096, 205), (100, 7), (33, 33), (1, 1)):
        n = seg * 5
        scores = torch.rand(n, device="cuda", generator=g)
        if seg > 5:
            scores[3] = scores[5]  # a tie inside the first segment
        pz = torch.rand((n, 7), device="cuda", generator=g)
        idx, kept = P.segment_topk(scores, seg, keep, pz)
        s = scores.cpu().numpy().reshape(-1, seg)
        for k in range(5):
            order = sorted(range(seg), key=lambda i: (-s[k, i], i))[:keep]
            assert list(idx[k].cpu().numpy() - k * seg) == order, (seg, k)
        assert torch.equal(kept, pz[idx.reshape(-1).long()])
        best, val = P.segment_argmax(scores, seg)
        assert np.array_equal(best.cpu().numpy(), s.argmax(1) + np.arange(5) * seg)
        assert np.array_equal(val.cpu().numpy(), s.max(1))


def test_pruned_selection_keeps_the_exact_best_when_everything_is_kept():
    """keep = seg: pruning changes nothing, so the pruned choice equals the exact one."""
    from paper_2503_22588_gb300 import planning as P
    w = configs.exact64(seed=4, n_views=64)
    cam = nbt.camera(32, 24, w.camera.fov_h, w.camera.fov_v, 1.0)
    prm = nbt.ig_params("count")
    m = nbt.Map.from_grid(torch.from_numpy(w.grid).cuda(), 0.01)
    pz = torch.from_numpy(w.poses).cuda()
    net = gs.Surrogate(max_batch=32, params=S.init_params(2))
    bx, vx, _ = P.exact_best(m, pz, 16, cam, prm)
    bp, vp, kept = P.pruned_best(net, m, pz, 16, 16, cam, prm)
    assert torch.equal(bx, bp) and torch.equal(vx, vp)
    bp2, vp2, kept2 = P.pruned_best(net, m, pz, 16, 3, cam, prm)
    assert kept2.shape == (4, 3) and torch.all(vp2 <= vx)
    net.close()


def test_plan_pruned_kept_indices_are_the_top_scores_and_best_is_their_exact_argmax():
    """nbt_plan_pruned in one call equals its steps run one by one: the kept indices are the per-segment
    top-k of the network's scores of the crops, and the best view is the exact argmax among them."""
    from paper_2503_22588_gb300 import planning as P
    w = configs.exact64(seed=6, n_views=64)
    cam = nbt.camera(32, 24, w.camera.fov_h, w.camera.fov_v, 1.0)
    prm = nbt.ig_params("count")
    m = nbt.Map.from_grid(torch.from_numpy(w.grid).cuda(), 0.01)
    pz = torch.from_numpy(w.poses).cuda()
    net = gs.Surrogate(max_batch=24, params=S.init_params(3))      # 64 candidates: three batches
    best, val, kept = P.pruned_best(net, m, pz, 16, 5, cam, prm)
    scores = P.surrogate_scores(net, m, pz, cam, prm)
    idx, kp = P.segment_topk(scores, 16, 5, pz)
    assert torch.equal(kept, idx)
    ig, _ = nbt.views_ig(m, kp, cam, prm)
    b2, v2 = P.segment_argmax(ig, 5, idx.reshape(-1).contiguous())
    assert torch.equal(best, b2) and torch.equal(val, v2)
    exact, _ = nbt.views_ig(m, pz, cam, prm)
    assert torch.equal(val, exact[best.long()])                   # the reported IG is the exact one
    assert no_device_timeout()
    net.close()
    m.close()


def test_plan_pruned_over_many_batches_equals_its_steps_every_time():
    """The crops of batch b + 1 run on the network's side stream while the forward of batch b runs, in
    two alternating buffers: over 24 batches, repeated, the kept indices and the best views equal
    those of the steps run one by one on one stream."""
    from paper_2503_22588_gb300 import planning as P
    w = configs.exact64(seed=7, n_views=192)
    cam = nbt.camera(32, 24, w.camera.fov_h, w.camera.fov_v, 1.0)
    prm = nbt.ig_params("count")
    m = nbt.Map.from_grid(torch.from_numpy(w.grid).cuda(), 0.01)
    pz = torch.from_numpy(w.poses).cuda()
    net = gs.Surrogate(max_batch=8, params=S.init_params(5))       # 192 candidates: 24 batches
    scores = P.surrogate_scores(net, m, pz, cam, prm)
    idx, kp = P.segment_topk(scores, 32, 4, pz)
    ig, _ = nbt.views_ig(m, kp, cam, prm)
    b_ref, v_ref = P.segment_argmax(ig, 4, idx.reshape(-1).contiguous())
    ws = P.pruned_workspace(net, 192, 32, 4, cam)
    for _ in range(5):
        best, val, kept = P.pruned_best(net, m, pz, 32, 4, cam, prm, ws)
        assert torch.equal(kept, idx)
        assert torch.equal(best, b_ref) and torch.equal(val, v_ref)
    assert no_device_timeout()
    net.close()
    m.close()


def test_plan_pruned_refuses_bad_arguments_before_enqueueing():
    from paper_2503_22588_gb300 import planning as P
    w = configs.exact64(seed=6, n_views=32)
    cam = nbt.camera(16, 12, w.camera.fov_h, w.camera.fov_v, 1.0)
    m = nbt.Map.from_grid(torch.from_numpy(w.grid).cuda(), 0.01)
    pz = torch.from_numpy(w.poses).cuda()
    net = gs.Surrogate(max_batch=8, params=S.init_params(3))
    ws = P.pruned_workspace(net, 32, 16, 4, cam)
    best = torch.full((2,), -5, dtype=torch.int32, device="cuda")
    L = _lib.lib()

    def call(n=32, seg=16, keep=4, prm=nbt.ig_params("count"), ws_bytes=None, wsp=None):
        return L.nbt_plan_pruned(m.handle, net.handle, pz.data_ptr(), n, seg, keep, C.byref(cam), C.byref(prm),
                                 best.data_ptr(), None, None, wsp if wsp is not None else ws.data_ptr(),
                                 ws.numel() if ws_bytes is None else ws_bytes, None)

    assert call(n=30) == -1                 # not a multiple of seg
    assert call(keep=17) == -1 and call(keep=0) == -1
    assert call(seg=9000, n=9000) == -1
    assert call(prm=nbt.ig_params("entropy")) == -5     # entropy on a state map: unsupported
    assert call(ws_bytes=ws.numel() - 1) == -6          # workspace too small
    assert call(wsp=ws.data_ptr() + 16) == -6          # not 256-byte aligned
    torch.cuda.synchronize()
    assert torch.all(best == -5)                        # nothing was enqueued
    assert call() == 0
    torch.cuda.synchronize()
    assert torch.all(best >= 0)
    net.close()
    m.close()


def test_crop_arrays_that_are_not_16_byte_aligned_are_refused_before_enqueueing():
    """Crops are written in 4-byte and read in 16-byte vectors: every call that takes a crop array
    refuses one that does not start on a 16-byte boundary, on the host, before any launch."""
    grid, p = small_scene("u8", seed=1)
    cam = nbt.camera(64, 48, math.radians(60), math.radians(45), 0.5)
    prm = nbt.ig_params("count")
    m = nbt.Map.from_grid(torch.from_numpy(grid).cuda(), 0.01)
    pz = torch.from_numpy(p[:2]).cuda()
    raw = torch.full((2 * 32768 + 64,), 7, dtype=torch.uint8, device="cuda")
    ft = torch.zeros((2, 8), dtype=torch.bfloat16, device="cuda")
    net = gs.Surrogate(max_batch=8, params=S.init_params(2))
    pred = torch.zeros(2, dtype=torch.float32, device="cuda")
    tgt = torch.zeros(2, dtype=torch.float32, device="cuda")
    L = _lib.lib()
    for off in (1, 4, 8):
        ptr = raw.data_ptr() + off
        assert L.nbt_surrogate_crops(m.handle, pz.data_ptr(), 2, C.byref(cam), C.byref(prm), ptr, ft.data_ptr(),
                                     None) == -1
        assert L.nbt_surrogate_forward(net.handle, ptr, ft.data_ptr(), 2, pred.data_ptr(), None) == -1
        assert L.nbt_surrogate_backward(net.handle, ptr, ft.data_ptr(), tgt.data_ptr(), 2, None, None, None) == -1
    torch.cuda.synchronize()
    assert torch.all(raw == 7)                          # nothing was written
    assert L.nbt_surrogate_crops(m.handle, pz.data_ptr(), 2, C.byref(cam), C.byref(prm), raw.data_ptr() + 16,
                                 ft.data_ptr(), None) == 0
    torch.cuda.synchronize()
    ref, _ = gs.crops(m, pz, cam, prm)
    assert torch.equal(raw[16:16 + 2 * 32768].view(2, 32, 32, 32), ref)
    net.close()
    m.close()


def test_target_scale_equals_prescaled_targets_bitwise():
    """nbt_surrogate_set_target_scale: loss and gradients with scale c and targets t equal those with
    scale 1 and targets c t rounded to FP32, bit for bit."""
    cr, ft = _batch(8, seed=7)
    params = S.init_params(5)
    t = torch.linspace(10.0, 80.0, 8, device="cuda")
    a = gs.Surrogate(max_batch=8, params=params, target_scale=0.01)
    b = gs.Surrogate(max_batch=8, params=params)
    la, ga = a.backward(cr, ft, t)
    lb, gb = b.backward(cr, ft, (t * 0.01).contiguous())
    torch.cuda.synchronize()
    assert torch.equal(la, lb) and torch.equal(ga, gb)
    a.close()
    b.close()


def test_checkpoint_resume_is_bitwise(tmp_path):
    """N Adam steps in one go equal k steps, a checkpoint written to a file and loaded into a fresh
    network, and N - k more steps: parameters, Adam moments and step count bit for bit."""
    cr, ft = _batch(16, seed=9)
    t = torch.rand(16, device="cuda", generator=torch.Generator(device="cuda").manual_seed(2))
    params = S.init_params(10)
    ref = gs.Surrogate(max_batch=16, params=params, target_scale=0.5)
    for i in range(7):
        ref.train_step(cr, ft, t, lr=1e-3 * (1 + i % 3))
    a = gs.Surrogate(max_batch=16, params=params, target_scale=0.5)
    for i in range(3):
        a.train_step(cr, ft, t, lr=1e-3 * (1 + i % 3))
    state = a.checkpoint()
    assert state["step"] == 3
    a.save(tmp_path / "surrogate.npz")
    a.close()
    b = gs.Surrogate(max_batch=16)
    b.load(tmp_path / "surrogate.npz")
    assert b.target_scale == 0.5
    for i in range(3, 7):
        b.train_step(cr, ft, t, lr=1e-3 * (1 + i % 3))
    want, got = ref.checkpoint(), b.checkpoint()
    assert got["step"] == want["step"] == 7
    for k in ("params", "adam_m", "adam_v"):
        assert np.array_equal(got[k], want[k]), k
    # and the next predictions agree too
    assert torch.equal(ref.forward(cr, ft), b.forward(cr, ft))
    assert no_device_timeout()
    ref.close()
    b.close()
