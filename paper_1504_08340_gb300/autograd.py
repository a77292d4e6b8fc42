"""torch.autograd access to the misfit J(lambda, mu) of Eq. (7) of arXiv:1504.08340
and to its gradient from the adjoint sweep (Sec. 3.1, Eqs. (C.1f), (C.1g)).

``misfit(ctx, lam, mu, observed)`` sets the context's material to (lam, mu) and
returns J as a 0-d float64 tensor. lam and mu are float32 CUDA tensors over the
interior nodes ([k][j][i], shape ``ctx.mat_shape()``); observed is the float32 CUDA
tensor of observed traces ([shot][step][receiver][component]). The backward pass
returns dJ/dlambda_i and dJ/dmu_i (the library's g_mis) times the incoming gradient,
in the dtypes of lam and mu.

The forward call already evaluates the gradient, because the adjoint sweep needs
the forward wavefield that the forward call computes; backward launches nothing.
How the adjoint obtains the forward displacement (stored history or sqrt(T)
checkpointing with recomputation) is the context's setting (``set_checkpointing``).
"""
from __future__ import annotations

import torch


class MisfitFunction(torch.autograd.Function):
    """J(lambda, mu) with its adjoint-state gradient (see the module docstring)."""

    @staticmethod
    def forward(fctx, lam, mu, ctx, observed, shot0=0, nshots=1):
        if not (lam.is_cuda and mu.is_cuda and observed.is_cuda):
            raise TypeError("lam, mu and observed must be CUDA tensors")
        ctx.set_material(lam.detach().to(torch.float32).contiguous(), mu.detach().to(torch.float32).contiguous())
        J, g_lambda, g_mu = ctx.adjoint_gradient(observed.detach().to(torch.float32).contiguous(), shot0, nshots)
        fctx.save_for_backward(g_lambda, g_mu)
        fctx.dtypes = (lam.dtype, mu.dtype)
        return torch.tensor(J, dtype=torch.float64, device=lam.device)

    @staticmethod
    def backward(fctx, grad_J):
        g_lambda, g_mu = fctx.saved_tensors
        return ((grad_J * g_lambda).to(fctx.dtypes[0]), (grad_J * g_mu).to(fctx.dtypes[1]), None, None, None, None)


def misfit(ctx, lam, mu, observed, shot0: int = 0, nshots: int = 1):
    """J summed over shots shot0 .. shot0 + nshots - 1, differentiable in lam and mu."""
    return MisfitFunction.apply(lam, mu, ctx, observed, shot0, nshots)
