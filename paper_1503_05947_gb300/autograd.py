"""torch.autograd binding of the differentiation form.

``rbd_loss(X, Xo, d)`` runs Algorithm 1 on X for d bases (tolerance 0), maps the out-of-sample
data Xo (Section 3.1), and returns L = w_rec ||X - Y T||_F^2 + w_proj ||Y' Xo||_F^2 as a 0-dim
tensor; its backward is the hand-written adjoint (rbd_grad) for the pivot set the forward
chose, which is held fixed.  Every step runs in librbd's kernels.
"""
from __future__ import annotations

import torch

from . import rbd


class RBDLoss(torch.autograd.Function):
    @staticmethod
    def forward(ctx, X: torch.Tensor, Xo: torch.Tensor, d: int, w_rec: float, w_proj: float):
        Xd = rbd.as_colmajor(X.detach())
        Xod = rbd.as_colmajor(Xo.detach()) if Xo is not None else None
        r = rbd.compress(Xd, 0.0, d)
        _, loss = rbd.grad(Xd, r.Y, r.T, r.pivots, Xod, w_rec, w_proj, need_grad=False)
        ctx.save_for_backward(Xd, Xod if Xod is not None else torch.empty(0, device=X.device), r.Y, r.T, r.pivots)
        ctx.weights = (w_rec, w_proj)
        ctx.has_xo = Xod is not None
        ctx.x_dtype = X.dtype
        return loss.to(X.dtype)

    @staticmethod
    def backward(ctx, gout):
        Xd, Xod, Y, T, piv = ctx.saved_tensors
        w_rec, w_proj = ctx.weights
        G, _ = rbd.grad(Xd, Y, T, piv, Xod if ctx.has_xo else None, w_rec, w_proj, need_grad=True)
        return (G * gout.to(torch.float64)).to(ctx.x_dtype), None, None, None, None


def rbd_loss(X: torch.Tensor, Xo: torch.Tensor | None, d: int, w_rec: float = 1.0, w_proj: float = 1.0):
    """L = w_rec ||X - Y T||_F^2 + w_proj ||Y' Xo||_F^2 with (Y, T) from d steps of Algorithm 1 on
    X; differentiable with respect to X for the fixed pivot set."""
    return RBDLoss.apply(X, Xo, d, w_rec, w_proj)
