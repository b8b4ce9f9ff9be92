"""torch.autograd.Function for the squared objective f(U, V) = ||A - U V^T||_F^2.

The forward pass loads U and V into an espnmf context and evaluates f with
the library's FP64 identity (||A||^2 - 2 <U, A V> + <U^T U, V^T V>, never
forming U V^T); the backward pass is hand-written: it reloads the same U and
V and asks the library for

    grad_U = 2 (U V^T V - A V),    grad_V = 2 (V U^T U - A^T U),

which reuse the context's sparse products.  U and V must be non-negative
(the factors of the method are), dense, row-major, float32 or float64, on
the context's device or on the host.
"""
from __future__ import annotations

import torch

from . import binding as B


def _load_factors(ctx: B.Context, U: torch.Tensor, V: torch.Tensor):
    if U.is_cuda:
        torch.cuda.current_stream(U.device).synchronize()
    B.espnmf_set_factor(ctx, B.U, U.detach().contiguous())
    B.espnmf_set_factor(ctx, B.V, V.detach().contiguous())


class ReconstructionLoss(torch.autograd.Function):
    """f = ReconstructionLoss.apply(U, V, ctx): a float64 scalar tensor."""

    @staticmethod
    def forward(fctx, U, V, ctx):
        _load_factors(ctx, U, V)
        f = B.espnmf_loss(ctx)
        fctx.espnmf = ctx
        fctx.save_for_backward(U, V)
        return torch.tensor(f, dtype=torch.float64, device=U.device)

    @staticmethod
    def backward(fctx, g):
        U, V = fctx.saved_tensors
        ctx = fctx.espnmf
        _load_factors(ctx, U, V)
        gU = gV = None
        if fctx.needs_input_grad[0]:
            gU = torch.empty_like(U, memory_format=torch.contiguous_format)
            B.espnmf_grad(ctx, B.U, gU)
            gU = gU * g.to(gU.dtype)
        if fctx.needs_input_grad[1]:
            gV = torch.empty_like(V, memory_format=torch.contiguous_format)
            B.espnmf_grad(ctx, B.V, gV)
            gV = gV * g.to(gV.dtype)
        return gU, gV, None


def reconstruction_loss(U: torch.Tensor, V: torch.Tensor, ctx: B.Context) -> torch.Tensor:
    """f(U, V) = ||A - U V^T||_F^2 with A the context's matrix (differentiable)."""
    return ReconstructionLoss.apply(U, V, ctx)
