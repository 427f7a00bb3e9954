"""torch.autograd.Function for the (masked) synthesis D (M^t)^T z.

Forward is the library's synthesis kernel; backward is its adjoint kernels:
grad_z = m . D^T g (the code adjoint correlation) and grad_d = Z^T g (the
filter-gradient correlation), both from scsc_synth_backward.  No PyTorch
arithmetic runs on either pass.
"""
from __future__ import annotations

import torch

from . import scsc


class Synthesis(torch.autograd.Function):
    """xhat = sum_k d_k * (m_k . z_k) for a packed batch of images."""

    @staticmethod
    def forward(fctx, z, d, ctx: scsc.Context, batch: scsc.Batch, t: int = 0, masked: bool = False):
        z = z.contiguous()
        d = d.contiguous()
        xhat = scsc.scsc_synth(ctx, batch, z, d, t, masked)
        fctx.save_for_backward(z, d)
        fctx.scsc = (ctx, batch, t, masked)
        return xhat

    @staticmethod
    def backward(fctx, grad):
        z, d = fctx.saved_tensors
        ctx, batch, t, masked = fctx.scsc
        need_z, need_d = fctx.needs_input_grad[0], fctx.needs_input_grad[1]
        gz, gd = scsc.scsc_synth_backward(ctx, batch, grad.contiguous(), z, d, t, masked,
                                          need_z=need_z, need_d=need_d)
        if gd is not None:
            gd = gd.view_as(d)
        if gz is not None:
            gz = gz.view_as(z)
        return gz, gd, None, None, None, None


def synthesis(z, d, ctx: scsc.Context, batch: scsc.Batch, t: int = 0, masked: bool = False):
    return Synthesis.apply(z, d, ctx, batch, t, masked)
