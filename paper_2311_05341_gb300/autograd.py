"""Differentiable float32 dedispersion: a torch.autograd.Function.

Forward is dd_run (Eq. 3 with time binning); backward is dd_run_adjoint, the
exact transpose of that linear map (re-dispersion as a gather), so gradients
of any loss of the DM-time planes flow back to the filterbank.  The paper has
no adjoint; this is the derivative of its Eq. 3.
"""
from __future__ import annotations

import torch

from . import Plan


def _aligned_rows(x: torch.Tensor) -> torch.Tensor:
    """x with a 16-byte aligned row stride and base (copying only if needed)."""
    if x.stride(1) == 1 and x.stride(0) % 4 == 0 and x.data_ptr() % 16 == 0:
        return x
    n_chan, n_samp = x.shape
    stride = (n_samp + 3) // 4 * 4
    buf = torch.zeros((n_chan, stride), dtype=torch.float32, device=x.device)
    buf[:, :n_samp] = x
    return buf


class DedispFn(torch.autograd.Function):
    """Y = A X for a float32 plan; returns the flat concatenated output planes."""

    @staticmethod
    def forward(ctx, x: torch.Tensor, plan: Plan) -> torch.Tensor:
        if plan.dtype != "f32":
            raise TypeError("DedispFn needs a float32 plan")
        n_samp = x.shape[1]
        xa = _aligned_rows(x.detach())
        out = plan.empty_output(n_samp, x.device)
        plan.run(xa, out=out, n_samp=n_samp)
        ctx.plan = plan
        ctx.n_samp = n_samp
        return out

    @staticmethod
    def backward(ctx, grad_out: torch.Tensor):
        g = grad_out.contiguous().to(torch.float32)
        xbar = ctx.plan.run_adjoint(g, ctx.n_samp)
        return xbar, None


def dedisperse(x: torch.Tensor, plan: Plan):
    """Differentiable forward transform: list of [n_dm_r][n_out_r] planes."""
    flat = DedispFn.apply(x, plan)
    return plan.split(flat, x.shape[1])
