"""MO vgl as a differentiable PyTorch function of C and R_nuc.

``mo_vgl(context, C, R, coord)`` returns the MO vgl tensor [walk][elec][5][mo]
from the CUDA library; its backward calls the library's adjoint
(qk_mo_vgl_backward_device) for dL/dC (variational optimisation of the MO
coefficients) and dL/dR_nuc (structural optimisation, Sec. 3.6).  The AO
values are recomputed in the backward pass, not kept from the forward one.
"""
from __future__ import annotations

import numpy as np
import torch


class MOVgl(torch.autograd.Function):
    @staticmethod
    def forward(fctx, C, R, context, coord):
        context.set_nucleus(context.charges, R.detach().double().cpu().numpy())
        context.set_mo_coefficient(C.detach().double().cpu().numpy())
        context.set_points_device(coord)
        out = context.mo_vgl_device()
        fctx.context = context
        fctx.coord = coord
        fctx.dtypes = (C.dtype, C.device, R.dtype, R.device)
        return out

    @staticmethod
    def backward(fctx, grad_out):
        ctx = fctx.context
        ctx.set_points_device(fctx.coord)          # the forward's points, in case they moved
        need_c, need_r = fctx.needs_input_grad[0], fctx.needs_input_grad[1]
        dW = grad_out.to(ctx.dtype_torch).contiguous()
        dC, dR = ctx.backward_device(dW, need_dC=need_c, need_dR=need_r)
        cd, cdev, rd, rdev = fctx.dtypes
        gC = dC.to(dtype=cd, device=cdev) if need_c else None
        gR = dR.to(dtype=rd, device=rdev) if need_r else None
        return gC, gR, None, None


def mo_vgl(context, C: torch.Tensor, R: torch.Tensor, coord: torch.Tensor) -> torch.Tensor:
    """Differentiable MO vgl.  ``context`` must have its basis set
    (``Context.set_molecule``); C [mo][ao] and R [nucl][3] may require grad;
    coord is a CUDA float64 tensor [walk][elec][3]."""
    if getattr(context, "charges", None) is None:
        raise ValueError("context has no nuclear charges: call set_molecule first")
    return MOVgl.apply(C, R, context, coord)
