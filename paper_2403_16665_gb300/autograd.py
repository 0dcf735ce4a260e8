"""torch.autograd binding: forward = adfft_execute, backward = adfft_execute_adjoint.

    X = AlphaDFT.apply(x, M)            # x: CUDA [batch, N] real or complex
    loss = (X - Y).abs().pow(2).sum(); loss.backward()

The backward of X = S A x is the adjoint S A^H g (real part for a real x),
computed by the adjoint kernel of the same plan on the current stream.
"""
from __future__ import annotations

import torch

from . import adfft

_PLANS: dict = {}


def get_plan(N, M, batch, dtype, scale, device, algorithm=adfft.ALGO_AUTO):
    key = (int(N), int(M), int(batch), dtype, scale, device.index, algorithm)
    plan = _PLANS.get(key)
    if plan is None:
        with torch.cuda.device(device):
            plan = adfft.Plan(N, batch=batch, dtype=adfft._dtype_code(dtype), M=M)
            if scale is not None:
                plan.set_scale(scale)
            if algorithm != adfft.ALGO_AUTO:
                plan.set_algorithm(algorithm)
        _PLANS[key] = plan
    return plan


class AlphaDFT(torch.autograd.Function):
    """Differentiable alpha-DFT: X[b, m] = S sum_n x[b, n] exp(-2 pi i m n / M)."""

    @staticmethod
    def forward(ctx, x, M, scale=None):
        if not x.is_cuda:
            raise RuntimeError("AlphaDFT needs a CUDA tensor (no CPU path)")
        x2 = x.contiguous()
        one = x2.dim() == 1
        if one:
            x2 = x2.reshape(1, -1)
        B, N = x2.shape
        plan = get_plan(N, M, B, x2.dtype, scale, x2.device)
        X = torch.empty((B, int(M)), dtype=adfft.out_dtype(x2.dtype), device=x2.device)
        plan.execute(x2.data_ptr(), X.data_ptr(), torch.cuda.current_stream(x2.device))
        ctx.plan = plan
        ctx.one = one
        ctx.in_shape = x2.shape
        ctx.in_dtype = x2.dtype
        return X[0] if one else X

    @staticmethod
    def backward(ctx, gX):
        g = gX.reshape(ctx.in_shape[0], -1).contiguous()
        if g.dtype != adfft.out_dtype(ctx.in_dtype):
            g = g.to(adfft.out_dtype(ctx.in_dtype))
        gx = torch.empty(ctx.in_shape, dtype=ctx.in_dtype, device=g.device)
        ctx.plan.execute_adjoint(g.data_ptr(), gx.data_ptr(), torch.cuda.current_stream(g.device))
        if ctx.one:
            gx = gx[0]
        return gx, None, None


def alpha_dft_autograd(x, alpha=None, M=None, scale=None):
    N = x.shape[-1]
    if M is None:
        M = int(round(float(alpha) * N))
    return AlphaDFT.apply(x, M, scale)
