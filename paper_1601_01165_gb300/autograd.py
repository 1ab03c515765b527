"""torch.autograd wrappers over the libdd kernels.

dedisperse(x, w, plan): forward = dd_forward (Algorithm 1 with per-channel
weights), backward = dd_adjoint (transpose of Algorithm 1 for x, per-channel
dot products for w).  boxcar_snr_loss(out): -max 8-sample boxcar S/N over
the dedispersed block (dd_boxcar_snr), with its gradient.  All arithmetic
runs in the CUDA kernels; these classes only route tensors.
"""
from __future__ import annotations

import torch

from . import binding


class DedisperseFn(torch.autograd.Function):
    @staticmethod
    def forward(ctx, x, w, plan):
        ctx.plan = plan
        ctx.save_for_backward(x, w)
        return plan.forward(x, w)

    @staticmethod
    def backward(ctx, g):
        x, w = ctx.saved_tensors
        plan = ctx.plan
        need_x, need_w = ctx.needs_input_grad[0], ctx.needs_input_grad[1]
        if not (need_x or need_w):
            return None, None, None
        gx = torch.zeros_like(x) if need_x else None
        _, gw = plan.adjoint(g.contiguous(), w=w, x=x if need_w else None, grad_in=need_x, grad_w=need_w,
                             grad_in_out=gx)
        return gx, gw, None


def dedisperse(x, w, plan):
    """Differentiable dedispersion: out[i][t] = sum_c w[c] x[c][t + d(c, i)]."""
    return DedisperseFn.apply(x, w, plan)


class BoxcarSNRLossFn(torch.autograd.Function):
    @staticmethod
    def forward(ctx, out):
        raw, g = binding.boxcar_snr(out, grad=True)
        ctx.save_for_backward(g)
        ctx.raw = raw
        return raw.view(torch.float64)[0].to(torch.float32)

    @staticmethod
    def backward(ctx, gl):
        (g,) = ctx.saved_tensors
        return g * gl.to(g.dtype)


def boxcar_snr_loss(out):
    """-max over (DM trial, time) of the 8-sample boxcar S/N of a dedispersed block."""
    return BoxcarSNRLossFn.apply(out)
