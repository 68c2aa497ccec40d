"""The TTN energy as a differentiable PyTorch function.

``TTNEnergy.apply(sweeper, inst, v, *ws)`` returns the energy
<psi(ws, v)|H|psi(ws, v)> of one instance (Sec. II.C; FP64, computed by the
library's ascend and top contraction).  Its backward is the library's
environment (Sec. III.A): dE/dw_t for every isometry layer and dE/dv = 2 H_top v,
all in one call that keeps the ascended operators and recomputes the chi^3
intermediates.  Inputs are CUDA float64 tensors of the shapes ttn_sizes gives;
nothing here runs the contractions itself.
"""
from __future__ import annotations

import ctypes

import torch


def _cat(ws):
    return torch.cat([w.reshape(-1) for w in ws]).contiguous()


class TTNEnergy(torch.autograd.Function):
    @staticmethod
    def forward(ctx, sweeper, inst, v, *ws):
        flat = _cat(ws)
        vc = v.contiguous()
        dp = ctypes.POINTER(ctypes.c_double)
        rc = sweeper.lib.ttn_set_isometries(sweeper.h, inst, ctypes.cast(flat.data_ptr(), dp),
                                            ctypes.cast(vc.data_ptr(), dp))
        sweeper._check(rc, "set_isometries")
        E = sweeper.energy(inst)
        ctx.sweeper, ctx.inst = sweeper, inst
        ctx.shapes = [w.shape for w in ws]
        ctx.vshape = v.shape
        ctx.n_w = flat.numel()
        return torch.tensor(E, dtype=torch.float64, device=v.device)

    @staticmethod
    def backward(ctx, gE):
        s = ctx.sweeper
        out = torch.empty(ctx.n_w + ctx.vshape.numel(), dtype=torch.float64, device=gE.device)
        rc = s.lib.ttn_env(s.h, ctx.inst, -1, ctypes.c_void_p(out.data_ptr()))
        s._check(rc, "env")
        out = out * gE
        grads, off = [], 0
        for shp in ctx.shapes:
            n = shp.numel()
            grads.append(out[off:off + n].view(shp))
            off += n
        gv = out[off:].view(ctx.vshape)
        return (None, None, gv, *grads)


def energy(sweeper, inst, v, ws):
    """Differentiable energy of instance ``inst`` for tensors (v, ws)."""
    return TTNEnergy.apply(sweeper, inst, v, *ws)
