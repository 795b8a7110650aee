"""Exact and surrogate-pruned next-best-view selection, and surrogate training.

Candidates come in segments of ``seg`` perspectives (typically the views
around one PoI).  Exact selection raycasts every candidate (Section III) and
takes the best per segment.  Pruned selection (``nbt_plan_pruned``, one C
call) scores every candidate with the learned surrogate, keeps the ``keep``
best per segment, raycasts only those exactly, and takes the best of them;
exact raycasting judges the kept candidates, so a pruning mistake can only
lose the best view, never report a wrong IG.  All arithmetic runs in the
library's kernels; this module only sequences the calls.
"""

from __future__ import annotations

import ctypes as C

import numpy as np
import torch

from ._lib import check, lib
from .api import Camera, IgParams, Map, _dev, _stream, views_ig, workspace
from .surrogate import Surrogate, crops as make_crops

TARGET_SCALE = 0.01  # the network predicts g_P x 0.01 (applied to the targets in the loss kernel)


def segment_argmax(values: torch.Tensor, seg: int, idx: torch.Tensor | None = None, stream=None):
    """nbt_segment_argmax: (best index, best value) per segment."""
    n = values.shape[0]
    best = torch.empty(n // seg, dtype=torch.int32, device=values.device)
    val = torch.empty(n // seg, dtype=torch.float32, device=values.device)
    check(lib().nbt_segment_argmax(_dev(values, torch.float32, "values"),
                                   _dev(idx, torch.int32, "idx") if idx is not None else None, n, int(seg),
                                   best.data_ptr(), val.data_ptr(), _stream(stream)), "nbt_segment_argmax")
    return best, val


def segment_topk(scores: torch.Tensor, seg: int, keep: int, poses: torch.Tensor | None = None, stream=None):
    """nbt_segment_topk: kept global indices [n/seg, keep] (and kept poses)."""
    n = scores.shape[0]
    idx = torch.empty((n // seg, keep), dtype=torch.int32, device=scores.device)
    kept = torch.empty((n // seg * keep, 7), dtype=torch.float32, device=scores.device) if poses is not None else None
    check(lib().nbt_segment_topk(_dev(scores, torch.float32, "scores"), n, int(seg), int(keep), idx.data_ptr(),
                                 _dev(poses, torch.float32, "poses", (7,)) if poses is not None else None,
                                 kept.data_ptr() if kept is not None else None, _stream(stream)), "nbt_segment_topk")
    return idx, kept


def exact_best(m: Map, poses: torch.Tensor, seg: int, cam: Camera, params: IgParams, ws=None, stream=None):
    """Raycast every candidate; (best index, best IG, all IGs) per segment."""
    ig, _ = views_ig(m, poses, cam, params, ws=ws, stream=stream, want_steps=False)
    best, val = segment_argmax(ig, seg, stream=stream)
    return best, val, ig


def surrogate_scores(net: Surrogate, m: Map, poses: torch.Tensor, cam: Camera, params: IgParams, chunk: int | None = None,
                     stream=None) -> torch.Tensor:
    """Predicted mean ray IG (x 1/100) of every candidate, crops built chunk by chunk."""
    n = poses.shape[0]
    chunk = chunk or net.max_batch
    out = torch.empty(n, dtype=torch.float32, device=poses.device)
    for c0 in range(0, n, chunk):
        cr, ft = make_crops(m, poses[c0:c0 + chunk], cam, params, stream)
        net.forward(cr, ft, out[c0:c0 + chunk], stream)
    return out


def pruned_workspace(net: Surrogate, n: int, seg: int, keep: int, cam: Camera, device=None) -> torch.Tensor:
    """A device workspace for nbt_plan_pruned (crops of up to two batches, scores, kept views, raycast scratch)."""
    b = C.c_int64()
    check(lib().nbt_pruned_workspace_size(net.handle, int(n), int(seg), int(keep), C.byref(cam), C.byref(b)),
          "nbt_pruned_workspace_size")
    return torch.empty(max(b.value, 256), dtype=torch.uint8,
                       device=device if device is not None else torch.device("cuda"))


def pruned_best(net: Surrogate, m: Map, poses: torch.Tensor, seg: int, keep: int, cam: Camera, params: IgParams,
                ws: torch.Tensor | None = None, stream=None, out=None, want_kept: bool = True):
    """nbt_plan_pruned: (best index, its exact IG, kept indices [n/seg, keep] or None) per segment.

    ``ws``: a workspace from ``pruned_workspace`` (allocated here if not given);
    ``out``: optional preallocated (best int32 [n/seg], best IG float32 [n/seg]).
    """
    n = poses.shape[0]
    nseg = n // seg if seg > 0 else 0
    if ws is None:
        ws = pruned_workspace(net, n, seg, keep, cam, poses.device)
    if out is None:
        best = torch.empty(nseg, dtype=torch.int32, device=poses.device)
        val = torch.empty(nseg, dtype=torch.float32, device=poses.device)
    else:
        best, val = out
    kept = torch.empty((nseg, keep), dtype=torch.int32, device=poses.device) if want_kept else None
    if ws.data_ptr() % 256:
        raise ValueError("workspace must be 256-byte aligned")
    check(lib().nbt_plan_pruned(m.handle, net.handle, _dev(poses, torch.float32, "poses", (7,)), n, int(seg),
                                int(keep), C.byref(cam), C.byref(params), _dev(best, torch.int32, "best"),
                                _dev(val, torch.float32, "best_ig"), kept.data_ptr() if kept is not None else None,
                                _dev(ws, torch.uint8, "workspace"), ws.numel(), _stream(stream)), "nbt_plan_pruned")
    return best, val, kept


def label_views(m: Map, poses: torch.Tensor, cam: Camera, params: IgParams, stream=None) -> torch.Tensor:
    """Training targets: exact mean ray IG (Section III's g_P); the net scales them (TARGET_SCALE)."""
    prm = IgParams(params.metric, params.occ_threshold, params.free_threshold, params.include_hit, 1)  # mean
    ig, _ = views_ig(m, poses, cam, prm, stream=stream, want_steps=False)
    return ig


def train(net: Surrogate, maps: list, poses: list, targets: list, cam: Camera, params: IgParams, epochs: int,
          lr: float = 1e-3, batch: int | None = None, seed: int = 0, lr_decay: float = 0.5, log=None):
    """Adam over (map i, pose, target) samples; batches are drawn from one map at a time."""
    batch = batch or net.max_batch
    rng = np.random.default_rng(seed)
    losses = []
    order = [(i, b0) for i in range(len(maps)) for b0 in range(0, poses[i].shape[0] - batch + 1, batch)]
    step_losses = torch.zeros(len(order), dtype=torch.float32, device=poses[0].device)
    for ep in range(epochs):
        rate = lr * (lr_decay ** (ep / max(1, epochs - 1)) if lr_decay else 1.0)
        perm = [rng.permutation(poses[i].shape[0]) for i in range(len(maps))]
        perm_t = [torch.from_numpy(p).to(poses[0].device) for p in perm]
        for k, j in enumerate(rng.permutation(len(order))):
            i, b0 = order[j]
            sel = perm_t[i][b0:b0 + batch]
            cr, ft = make_crops(maps[i], poses[i][sel].contiguous(), cam, params)
            net.train_step(cr, ft, targets[i][sel].contiguous(), rate, step_losses[k:k + 1])
        losses.append(float(step_losses.cpu().numpy().mean()))
        if log:
            log(f"epoch {ep}: loss {losses[-1]:.5f} lr {rate:.2e}")
    return losses
