"""Differentiable best rank-one approximation: a torch.autograd.Function
whose forward is hoscf_solve and whose backward is hoscf_backward (the
envelope theorem for sigma plus the implicit-function adjoint of the KKT
system for the factors, solved on the GPU).  No counterpart in the paper."""
from __future__ import annotations

import torch

from .api import hoscf_backward, hoscf_solve


class HOSCFFunction(torch.autograd.Function):
    """(sigma, u) = HOSCF(T); u is the concatenation of the unit factors."""

    @staticmethod
    def forward(ctx, T, u0, tol, max_iter, variant):
        r = hoscf_solve(T.detach().contiguous(), u0.detach(), tol=tol, max_iter=max_iter,
                        variant=variant)
        ctx.save_for_backward(T, r.u)
        ctx.sigma = r.sigma
        sigma = torch.tensor(r.sigma, dtype=T.dtype, device=T.device)
        return sigma, r.u.clone()

    @staticmethod
    def backward(ctx, g_sigma, g_u):
        T, u = ctx.saved_tensors
        gs = float(g_sigma) if g_sigma is not None else 0.0
        gu = g_u.contiguous().float() if g_u is not None else None
        gT = hoscf_backward(T.detach().contiguous(), u, ctx.sigma, gs, gu)
        return gT, None, None, None, None


def hoscf(T: torch.Tensor, u0: torch.Tensor, tol: float = 1e-6, max_iter: int = 200,
          variant: str = "hoscf"):
    """Differentiable (sigma, u) of the best rank-one approximation of T."""
    return HOSCFFunction.apply(T, u0, tol, max_iter, variant)
