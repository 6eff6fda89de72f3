"""torch.autograd.Function for E_c^nl(n, grad n) on the CUDA library.

forward  : E_c^nl only (pointwise, plane and pencil transforms, contraction,
           FP64 energy); nothing of the Nq theta fields is kept.
backward : runs the pipeline again with the potential requested in its
           "gradient-output" form, which recomputes theta, and returns
             dE/dn_i         = dOmega v_loc,i
             dE/d(grad_c n)_i = dOmega w_c,i
           (Eq. Vi of the paper with the chain through grad n left to
           autograd), both scaled by the incoming gradient.

So when the caller builds grad n from n with its own differentiable
operator, autograd reproduces v_nl of Eq. (Vi) for that operator.
"""
from __future__ import annotations

import torch

from .vdwnl import VdwNL


class VdwEnergy(torch.autograd.Function):
    @staticmethod
    def forward(ctx, n, grad, handle: VdwNL):
        E = torch.empty(3, dtype=torch.float64, device=n.device)
        handle.energy_potential(n.contiguous(), grad.contiguous(), E, None, None)
        ctx.save_for_backward(n, grad)
        ctx.handle = handle
        return E[0].clone()

    @staticmethod
    def backward(ctx, gE):
        n, grad = ctx.saved_tensors
        h = ctx.handle
        v = torch.empty_like(n, dtype=torch.float32).contiguous()
        w = torch.empty_like(grad, dtype=torch.float32).contiguous()
        h.energy_potential(n.contiguous(), grad.contiguous(), None, v, w)
        scale = (gE * h.dOmega).to(torch.float32)
        dn = v * scale if ctx.needs_input_grad[0] else None
        dg = w * scale if ctx.needs_input_grad[1] else None
        return dn, dg, None


def vdw_energy(n, grad, handle: VdwNL):
    """E_c^nl (FP64 scalar tensor) with gradients w.r.t. n and grad n."""
    return VdwEnergy.apply(n, grad, handle)
