"""ln psi of the RBM as a torch.autograd.Function over the C ABI.

Forward: nk_rbm_logpsi (theta = b + W s rebuilt in the kernel).  Backward: the
hand-written adjoint, nk_vjp, which recomputes theta from the configurations
instead of storing it and returns J^T g for the incoming per-sample
gradient g (App. B.1 of the NetKet 3 paper: vector-Jacobian products).
Per-sample gradients (the rows O_k of the Jacobian, Eq. eq:log-derivative-O)
come from nk_jacobian.

Only the parameters are differentiable; configurations are integer data.
"""
from __future__ import annotations

import torch

from . import nk


class RBMLogPsi(torch.autograd.Function):
    """ln psi_theta(s) for a batch s [B, N] (int8 +-1) and parameters theta
    [N + M + M N] (float64 on the GPU)."""

    @staticmethod
    def forward(ctx, params, s, N, M, nkctx, precision="f64"):
        out = torch.empty(s.shape[0], dtype=torch.float64, device=params.device)
        nk.nk_rbm_logpsi(nkctx, params, N, M, s, out, precision=precision)
        ctx.save_for_backward(params, s)
        ctx.shape = (N, M)
        ctx.nkctx = nkctx
        ctx.precision = precision
        return out

    @staticmethod
    def backward(ctx, grad_out):
        params, s = ctx.saved_tensors
        N, M = ctx.shape
        g = grad_out.contiguous().to(torch.float64)
        grad = torch.empty_like(params)
        nk.nk_vjp(ctx.nkctx, params, N, M, s, g, grad, precision=ctx.precision)
        return grad, None, None, None, None, None


def logpsi(params, s, N, M, nkctx, precision="f64"):
    return RBMLogPsi.apply(params, s, N, M, nkctx, precision)


def per_sample_grad(params, s, N, M, nkctx, centered=False):
    """O [B, Np]: the per-sample log-derivatives d ln psi(s_k) / d theta."""
    B = s.shape[0]
    out = torch.empty((B, N + M + M * N), dtype=torch.float64, device=params.device)
    nk.nk_jacobian(nkctx, params, N, M, s, centered, 0, B, out)
    return out
