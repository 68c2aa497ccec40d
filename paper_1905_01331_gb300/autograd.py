"""The TTN energy as a differentiable PyTorch function.

``TTNEnergy.apply(sweeper, inst, prec, need_grad, v, *ws)`` returns the energy
<psi(ws, v)|H|psi(ws, v)> of one instance (Sec. II.C).  Its backward is the
library's environment kernel (Sec. III.A): dE/dw_t for every isometry layer
and dE/dv = 2 H_top v.  Forward and backward come from one call of
``ttn_value_and_grad``, which ascends the Hamiltonian, contracts the top and
then forms every layer's environment top-down while descending the density
matrices, with the contractions in precision ``prec`` (FP64 or a mixed
precision; the top contraction and the energy are FP64).  Whether the
ascended operators of every layer are stored or recomputed during the descent
is the Sweeper's ``recompute_ops`` option.  Inputs are CUDA float64 tensors of
the shapes ttn_sizes gives; nothing here runs the contractions itself.
"""
from __future__ import annotations

import ctypes

import torch

from . import PRECISIONS


def _cat(ws):
    return torch.cat([w.reshape(-1) for w in ws]).contiguous()


class TTNEnergy(torch.autograd.Function):
    @staticmethod
    def forward(ctx, sweeper, inst, prec, need_grad, v, *ws):
        flat = _cat(ws)
        vc = v.contiguous()
        dp = ctypes.POINTER(ctypes.c_double)
        rc = sweeper.lib.ttn_set_isometries(sweeper.h, inst, ctypes.cast(flat.data_ptr(), dp),
                                            ctypes.cast(vc.data_ptr(), dp))
        sweeper._check(rc, "set_isometries")
        grad = torch.empty(flat.numel() + vc.numel(), dtype=torch.float64, device=v.device) \
            if need_grad else None
        E = ctypes.c_double()
        rc = sweeper.lib.ttn_value_and_grad(sweeper.h, inst, int(prec), ctypes.byref(E),
                                            ctypes.c_void_p(grad.data_ptr()) if grad is not None else None)
        sweeper._check(rc, "value_and_grad")
        ctx.grad = grad
        ctx.shapes = [w.shape for w in ws]
        ctx.vshape = v.shape
        return torch.tensor(E.value, dtype=torch.float64, device=v.device)

    @staticmethod
    def backward(ctx, gE):
        out = ctx.grad * gE
        grads, off = [], 0
        for shp in ctx.shapes:
            n = shp.numel()
            grads.append(out[off:off + n].view(shp))
            off += n
        gv = out[off:].view(ctx.vshape)
        return (None, None, None, None, gv, *grads)


def energy(sweeper, inst, v, ws, prec="fp64"):
    """Differentiable energy of instance ``inst`` for tensors (v, ws), its
    contractions in precision ``prec`` ("fp64", "tf32", "tf32x3", "bf16",
    "bf16x3"; a mixed one needs a Sweeper created with a mixed precision)."""
    p = PRECISIONS[prec] if isinstance(prec, str) else int(prec)
    # the caller's grad mode decides whether the pass also forms the gradient
    # (inside Function.forward autograd is always off)
    need = torch.is_grad_enabled() and (v.requires_grad or any(w.requires_grad for w in ws))
    return TTNEnergy.apply(sweeper, inst, p, need, v, *ws)
