"""torch.autograd.Function over the library's evaluation and adjoint.

``SRFunction.apply(consts, programs, lengths, X, y, N, ctx)`` returns the MSE
of every program (sr_eval); its backward calls sr_eval_grad, which recomputes
the forward pass on the device and sweeps it in reverse, and scales
dMSE/dconst by the incoming gradient.  Only the inputs are saved: no tape
survives the forward call.
"""
from __future__ import annotations

import torch

from . import binding


class SRFunction(torch.autograd.Function):
    @staticmethod
    def forward(fctx, consts, programs, lengths, X, y, N: int, sr_ctx: binding.Context):
        mse = binding.sr_eval(sr_ctx, programs, lengths, consts, X, y, N, binding.SR_MSE)
        fctx.save_for_backward(consts, programs, lengths, X, y)
        fctx.N = N
        fctx.sr_ctx = sr_ctx
        return mse

    @staticmethod
    def backward(fctx, grad_mse):
        consts, programs, lengths, X, y = fctx.saved_tensors
        _, dconst = binding.sr_eval_grad(fctx.sr_ctx, programs, lengths, consts, X, y, fctx.N)
        g = (grad_mse.to(torch.float64)[:, None] * dconst).to(consts.dtype)
        return g, None, None, None, None, None, None


def program_mse(consts, programs, lengths, X, y, N, sr_ctx):
    """Differentiable MSE of every program with respect to its constants."""
    return SRFunction.apply(consts, programs, lengths, X, y, N, sr_ctx)
