"""n-body with collision merge and the checkpointed adjoint
(smmo_nbody_* in include/smmo.h): argument marshalling and the
torch.autograd.Function around the hand-written adjoint kernels."""
from __future__ import annotations

import ctypes

import numpy as np
import torch

from . import smmo

FIELDS = ("x", "y", "z", "vx", "vy", "vz", "m")


class NBodyParams(ctypes.Structure):
    _fields_ = [("G", ctypes.c_float), ("eps", ctypes.c_float), ("dt", ctypes.c_float),
                ("merge_r", ctypes.c_float), ("merge", ctypes.c_int)]


class NBody:
    """Bodies in an SMMO heap; state given as a dict of 7 float arrays
    (numpy or CUDA tensors) indexed by body id."""

    def __init__(self, state: dict, G=1.0, eps=1e-2, dt=1e-3, merge_r=5e-3, merge=True,
                 config: smmo.HeapConfig | None = None, stream=None):
        self.stream = stream
        cols = [torch.as_tensor(np.asarray(state[k], np.float32)).cuda() if not isinstance(state[k], torch.Tensor)
                else state[k].to("cuda", torch.float32).contiguous() for k in FIELDS]
        self.n = int(cols[0].numel())
        nbytes = int((self.n / 64 + 64) * 4096) + (16 << 20)
        self.heap = smmo.Heap(nbytes, config, stream=stream)
        self.params = NBodyParams(G, eps, dt, merge_r, 1 if merge else 0)
        ptrs = (ctypes.c_void_p * 7)(*[c.data_ptr() for c in cols])
        self._w = ctypes.c_void_p()
        smmo.check(smmo.lib().smmo_nbody_create(self.heap.handle, ctypes.c_int64(self.n), ptrs,
                                                ctypes.byref(self.params), smmo._stream(stream),
                                                ctypes.byref(self._w)), "nbody_create")

    def pairs(self) -> int:
        """Pair terms computed by the force passes so far."""
        v = ctypes.c_int64()
        smmo.check(smmo.lib().smmo_nbody_pairs(self._w, ctypes.byref(v), smmo._stream(self.stream)), "nbody_pairs")
        return v.value

    def step(self, n: int = 1):
        smmo.check(smmo.lib().smmo_nbody_step(self._w, n, smmo._stream(self.stream)), "nbody_step")

    def read(self):
        out = torch.empty(7 * self.n, dtype=torch.float32, device="cuda")
        live = torch.empty(self.n, dtype=torch.uint8, device="cuda")
        m = ctypes.c_int64()
        smmo.check(smmo.lib().smmo_nbody_export(self._w, ctypes.c_void_p(out.data_ptr()),
                                                ctypes.c_void_p(live.data_ptr()), ctypes.byref(m),
                                                smmo._stream(self.stream)), "nbody_export")
        o = out.view(7, self.n).cpu().numpy()
        st = {k: o[i].copy() for i, k in enumerate(FIELDS)}
        st["live"] = live.cpu().numpy()
        return st, m.value

    def forward_ckpt(self, steps: int, ckpt: int = 10) -> float:
        loss = ctypes.c_double()
        smmo.check(smmo.lib().smmo_nbody_forward_ckpt(self._w, steps, ckpt, ctypes.byref(loss),
                                                      smmo._stream(self.stream)), "nbody_forward_ckpt")
        return loss.value

    def backward(self) -> torch.Tensor:
        g = torch.empty(self.n, 3, dtype=torch.float32, device="cuda")
        smmo.check(smmo.lib().smmo_nbody_backward(self._w, ctypes.c_void_p(g.data_ptr()),
                                                  smmo._stream(self.stream)), "nbody_backward")
        return g

    def sync(self):
        return self.heap.sync()

    def close(self):
        if self._w:
            smmo.lib().smmo_nbody_destroy(self._w)
            self._w = ctypes.c_void_p()
        self.heap.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class KineticEnergyAfterSteps(torch.autograd.Function):
    """L(v0) = 1/2 sum m |v_T|^2 after `steps` no-merge drift-kick-drift
    steps from (x0, v0); backward runs the checkpointed adjoint."""

    @staticmethod
    def forward(ctx, v0, x0, m, steps: int = 50, ckpt: int = 10, G=1.0, eps=1e-2, dt=1e-3):
        st = {"x": x0[:, 0], "y": x0[:, 1], "z": x0[:, 2], "vx": v0[:, 0].detach(),
              "vy": v0[:, 1].detach(), "vz": v0[:, 2].detach(), "m": m}
        sim = NBody(st, G=G, eps=eps, dt=dt, merge=False)
        loss = sim.forward_ckpt(steps, ckpt)
        ctx.sim = sim
        return torch.tensor(loss, dtype=torch.float64, device=v0.device)

    @staticmethod
    def backward(ctx, grad_out):
        g = ctx.sim.backward()
        ctx.sim.close()
        return (grad_out.to(torch.float32) * g).to(torch.float32), None, None, None, None, None, None, None
