"""Python binding of the learned IG surrogate (argument marshalling only).

Parameters travel as a dict of FP32 arrays named like the network layers:
``w0..w3`` ([C_out, 27 C_in], tap (dz*3+dy)*3+dx then C_in), ``b0..b3``,
``f1`` ([128, 4104]), ``g1`` ([128]), ``f2`` ([128]), ``g2`` ([1]); they
are packed into the library's flat FP32 vector in that order.
"""

from __future__ import annotations

import ctypes as C

import numpy as np
import torch

from ._lib import check, lib
from .api import Camera, IgParams, Map, _dev, _stream

LAYERS = ((8, 16, 2), (16, 32, 2), (32, 64, 2), (64, 64, 1))
CROP, C0, FEATS, HIDDEN, FC_IN = 32, 8, 8, 128, 4104
SHAPES = ([item for i, (ci, co, _) in enumerate(LAYERS) for item in ((f"w{i}", (co, 27 * ci)), (f"b{i}", (co,)))]
          + [("f1", (HIDDEN, FC_IN)), ("g1", (HIDDEN,)), ("f2", (HIDDEN,)), ("g2", (1,))])


def he_init(seed: int) -> dict:
    """Seeded starting parameters: He-normal weights (std sqrt(2 / fan_in)), zero biases."""
    rng = np.random.default_rng(seed)
    out = {}
    for k, shp in SHAPES:
        if len(shp) == 2:
            out[k] = (rng.standard_normal(shp) * np.sqrt(2.0 / shp[1])).astype(np.float32)
        elif k == "f2":
            out[k] = (rng.standard_normal(shp) * np.sqrt(1.0 / shp[0])).astype(np.float32)
        else:
            out[k] = np.zeros(shp, np.float32)
    return out


def param_count() -> int:
    n = C.c_int64()
    check(lib().nbt_surrogate_param_count(C.byref(n)), "nbt_surrogate_param_count")
    return n.value


def pack(params: dict) -> np.ndarray:
    flat = np.concatenate([np.asarray(params[k], np.float32).reshape(-1) for k, _ in SHAPES])
    if flat.size != param_count():
        raise ValueError("parameter count mismatch")
    return np.ascontiguousarray(flat)


def unpack(flat: np.ndarray) -> dict:
    out, o = {}, 0
    for k, shp in SHAPES:
        n = int(np.prod(shp))
        out[k] = np.asarray(flat[o:o + n], np.float32).reshape(shp).copy()
        o += n
    return out


def crops(m: Map, poses: torch.Tensor, cam: Camera, params: IgParams, stream=None, out=None):
    """nbt_surrogate_crops: (crop codes uint8 [n, 32, 32, 32], feats bf16 [n, 8]) on the poses' device.

    Code 0: outside the map; 1 unknown, 2 free, 3 occupied (one-hot channel code - 1).

    ``out``: optional preallocated (crops, feats) with room for at least n
    rows; the first n rows are written and returned.
    """
    n = poses.shape[0]
    if out is None:
        cr = torch.empty((n, CROP, CROP, CROP), dtype=torch.uint8, device=poses.device)
        ft = torch.empty((n, FEATS), dtype=torch.bfloat16, device=poses.device)
    else:
        cr, ft = out[0][:n], out[1][:n]
        _dev(cr, torch.uint8, "crops")
        _dev(ft, torch.bfloat16, "feats")
    if n:
        check(lib().nbt_surrogate_crops(m.handle, _dev(poses, torch.float32, "poses", (7,)), n, C.byref(cam),
                                        C.byref(params), cr.data_ptr(), ft.data_ptr(), _stream(stream)),
              "nbt_surrogate_crops")
    return cr, ft


def save_checkpoint(state: dict, path) -> None:
    """Write a ``Surrogate.checkpoint()`` to ``path`` (numpy ``.npz``): the flat FP32 parameters in the
    nbt_surrogate layout, both Adam moments, the Adam step count and the target scale."""
    params = np.ascontiguousarray(state["params"], np.float32)
    if params.size != param_count():
        raise ValueError(f"checkpoint holds {params.size} parameters, the network has {param_count()}")
    np.savez(path, params=params, adam_m=np.ascontiguousarray(state["adam_m"], np.float32),
             adam_v=np.ascontiguousarray(state["adam_v"], np.float32), step=np.int64(state["step"]),
             target_scale=np.float64(state["target_scale"]))


def load_checkpoint(path) -> dict:
    """Read a checkpoint written by ``save_checkpoint`` (the dict ``Surrogate.restore`` takes)."""
    with np.load(path) as z:
        state = {"params": z["params"].astype(np.float32), "adam_m": z["adam_m"].astype(np.float32),
                 "adam_v": z["adam_v"].astype(np.float32), "step": int(z["step"]),
                 "target_scale": float(z["target_scale"])}
    n = param_count()
    if any(state[k].size != n for k in ("params", "adam_m", "adam_v")):
        raise ValueError(f"checkpoint does not hold {n} parameters per tensor")
    return state


class Surrogate:
    """nbt_surrogate: network, Adam state and activation buffers on the current device."""

    def __init__(self, max_batch: int = 256, params: dict | None = None, target_scale: float = 1.0):
        h = C.c_void_p()
        check(lib().nbt_surrogate_create(int(max_batch), C.byref(h)), "nbt_surrogate_create")
        self._h = h
        self.max_batch = int(max_batch)
        self.n_params = param_count()
        self.target_scale = 1.0
        if params is not None:
            self.set_params(params)
        if target_scale != 1.0:
            self.set_target_scale(target_scale)

    def set_target_scale(self, scale: float) -> None:
        """nbt_surrogate_set_target_scale: training targets are multiplied by ``scale`` in the loss."""
        check(lib().nbt_surrogate_set_target_scale(self.handle, float(scale)), "nbt_surrogate_set_target_scale")
        self.target_scale = float(scale)

    def checkpoint(self) -> dict:
        """The whole training state: parameters, Adam moments, Adam step count and target scale."""
        m = np.empty(self.n_params, np.float32)
        v = np.empty(self.n_params, np.float32)
        step = C.c_int64()
        check(lib().nbt_surrogate_get_adam(self.handle, m.ctypes.data, v.ctypes.data, m.size, C.byref(step)),
              "nbt_surrogate_get_adam")
        return {"params": pack(self.get_params()), "adam_m": m, "adam_v": v, "step": int(step.value),
                "target_scale": self.target_scale}

    def restore(self, state: dict) -> None:
        """Load a ``checkpoint()``: training continues from it bit for bit."""
        flat = np.ascontiguousarray(state["params"], np.float32)
        check(lib().nbt_surrogate_set_params(self.handle, flat.ctypes.data, flat.size), "nbt_surrogate_set_params")
        m = np.ascontiguousarray(state["adam_m"], np.float32)
        v = np.ascontiguousarray(state["adam_v"], np.float32)
        check(lib().nbt_surrogate_set_adam(self.handle, m.ctypes.data, v.ctypes.data, m.size, int(state["step"])),
              "nbt_surrogate_set_adam")
        self.set_target_scale(state["target_scale"])

    def save(self, path) -> None:
        """``checkpoint()`` written to a file (``save_checkpoint``)."""
        save_checkpoint(self.checkpoint(), path)

    def load(self, path) -> None:
        """``restore()`` from a file written by ``save``: training continues from it bit for bit."""
        self.restore(load_checkpoint(path))

    @property
    def handle(self) -> int:
        return self._h.value

    def set_params(self, params: dict) -> None:
        flat = pack(params)
        check(lib().nbt_surrogate_set_params(self.handle, flat.ctypes.data, flat.size), "nbt_surrogate_set_params")

    def get_params(self) -> dict:
        flat = np.empty(self.n_params, np.float32)
        check(lib().nbt_surrogate_get_params(self.handle, flat.ctypes.data, flat.size), "nbt_surrogate_get_params")
        return unpack(flat)

    def forward(self, crops_t: torch.Tensor, feats: torch.Tensor, out: torch.Tensor | None = None, stream=None):
        n = crops_t.shape[0]
        out = out if out is not None else torch.empty(n, dtype=torch.float32, device=crops_t.device)
        if n:
            check(lib().nbt_surrogate_forward(self.handle, _dev(crops_t, torch.uint8, "crops"),
                                              _dev(feats, torch.bfloat16, "feats"), n,
                                              _dev(out, torch.float32, "pred"), _stream(stream)),
                  "nbt_surrogate_forward")
        return out

    def backward(self, crops_t, feats, targets, stream=None):
        """(loss tensor [1], flat gradient tensor [n_params]) for one batch, no update."""
        n = crops_t.shape[0]
        grads = torch.empty(self.n_params, dtype=torch.float32, device=crops_t.device)
        loss = torch.empty(1, dtype=torch.float32, device=crops_t.device)
        check(lib().nbt_surrogate_backward(self.handle, _dev(crops_t, torch.uint8, "crops"),
                                           _dev(feats, torch.bfloat16, "feats"),
                                           _dev(targets, torch.float32, "targets"), n, grads.data_ptr(),
                                           loss.data_ptr(), _stream(stream)), "nbt_surrogate_backward")
        return loss, grads

    def train_step(self, crops_t, feats, targets, lr: float, loss: torch.Tensor | None = None, stream=None):
        n = crops_t.shape[0]
        loss = loss if loss is not None else torch.empty(1, dtype=torch.float32, device=crops_t.device)
        check(lib().nbt_surrogate_train_step(self.handle, _dev(crops_t, torch.uint8, "crops"),
                                             _dev(feats, torch.bfloat16, "feats"),
                                             _dev(targets, torch.float32, "targets"), n, float(lr),
                                             loss.data_ptr(), _stream(stream)), "nbt_surrogate_train_step")
        return loss

    def close(self) -> None:
        if getattr(self, "_h", None) is not None:
            lib().nbt_surrogate_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
