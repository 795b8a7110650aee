"""Binding of the IG-between-perspectives entry points (Section IV, Eq. 3,
orientation factor, c_I): the ID buffer, G(x) and the trajectory IG cost.

Argument marshalling only; the arithmetic runs in libnbt.so.
"""

from __future__ import annotations

import ctypes as C

import torch

from ._lib import CostParams, check, lib
from .api import _dev, _stream

PAPER_EPS = 1e-7     # the epsilon of c_I
PAPER_POWER = 2.0    # IDW distance power p of the paper's experiments
PAPER_N_B = 10       # buffered IDs N_B of the paper's experiments


class IdBuffer:
    """nbt_id_buffer: the N_B most recent information distributions on the current device."""

    def __init__(self, n_b: int = PAPER_N_B, max_views: int = 4096):
        h = C.c_void_p()
        check(lib().nbt_id_buffer_create(int(n_b), int(max_views), C.byref(h)), "nbt_id_buffer_create")
        self._h = h
        self.n_b = int(n_b)
        self.max_views = int(max_views)

    @property
    def handle(self) -> int:
        if self._h is None:
            raise ValueError("the ID buffer is closed")
        return self._h

    def push(self, poses: torch.Tensor, ig: torch.Tensor, stream=None) -> None:
        """nbt_id_buffer_push: one ID of n perspectives (poses (n, 7), IGs (n,) FP32, on the device)."""
        n = poses.shape[0]
        if ig.shape != (n,):
            raise ValueError("ig must have shape (n,)")
        check(lib().nbt_id_buffer_push(self.handle, _dev(poses, torch.float32, "poses", (7,)) if n else None,
                                       _dev(ig, torch.float32, "ig") if n else None, n, _stream(stream)),
              "nbt_id_buffer_push")

    def clear(self) -> None:
        check(lib().nbt_id_buffer_clear(self.handle), "nbt_id_buffer_clear")

    def __len__(self) -> int:
        n = C.c_int32()
        check(lib().nbt_id_buffer_count(self.handle, C.byref(n)), "nbt_id_buffer_count")
        return n.value

    def close(self) -> None:
        if getattr(self, "_h", None) is not None:
            lib().nbt_id_buffer_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def idw_gain(buf: IdBuffer, poses: torch.Tensor, power: float = PAPER_POWER, out: torch.Tensor | None = None,
             stream=None) -> torch.Tensor:
    """nbt_idw_gain: G(x) of Eq. 3 at the positions of poses (n, 7)."""
    n = poses.shape[0]
    if out is None:
        out = torch.empty(n, dtype=torch.float32, device=poses.device)
    check(lib().nbt_idw_gain(buf.handle, _dev(poses, torch.float32, "poses", (7,)) if n else None, n, float(power),
                             _dev(out, torch.float32, "out") if n else None, _stream(stream)), "nbt_idw_gain")
    return out


def ig_cost(buf: IdBuffer, poses: torch.Tensor, offsets: torch.Tensor, poi, fov_h: float, fov_v: float,
            w_info: float = 1.0, power: float = PAPER_POWER, eps: float = PAPER_EPS, want_parts: bool = False,
            stream=None):
    """nbt_ig_cost: c_I per trajectory (CSR offsets (n_traj + 1,) int32 on the device).

    Returns cost (n_traj,), and with want_parts also (G, O, term) per pose.
    """
    n = poses.shape[0]
    nt = offsets.shape[0] - 1
    dev = poses.device
    term = torch.empty(n, dtype=torch.float32, device=dev)
    cost = torch.empty(max(nt, 0), dtype=torch.float32, device=dev)
    g = torch.empty(n, dtype=torch.float32, device=dev) if want_parts else None
    o = torch.empty(n, dtype=torch.float32, device=dev) if want_parts else None
    poi_c = (C.c_float * 3)(*[float(v) for v in poi])
    prm = CostParams(float(power), float(w_info), float(eps))
    check(lib().nbt_ig_cost(buf.handle, _dev(poses, torch.float32, "poses", (7,)) if n else None, n,
                            _dev(offsets, torch.int32, "offsets") if nt > 0 else None, nt, poi_c, float(fov_h),
                            float(fov_v), C.byref(prm), g.data_ptr() if g is not None and n else None,
                            o.data_ptr() if o is not None and n else None, term.data_ptr() if n else None,
                            cost.data_ptr() if nt > 0 else None, _stream(stream)), "nbt_ig_cost")
    return (cost, g, o, term) if want_parts else cost
