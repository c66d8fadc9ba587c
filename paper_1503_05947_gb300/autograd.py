"""torch.autograd binding of the differentiation form.

``rbd_loss(X, Xo, d)`` runs Algorithm 1 on X for d bases (tolerance 0), maps the out-of-sample
data Xo (Section 3.1), and returns L = w_rec ||X - Y T||_F^2 + w_proj ||Y' Xo||_F^2 as a 0-dim
tensor; its backward is the hand-written adjoint (rbd_grad) for the pivot set the forward
chose, which is held fixed.  ``rbd_loss_batched`` does the same for a list of matrices with the
batched compression and the batched adjoint.  Every step runs in librbd's kernels.
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


class RBDLossBatched(torch.autograd.Function):
    """The differentiation form of a batch of matrices: the forward compresses every X in one
    batched launch (rbd_batch_*, tolerance 0, d bases each) and evaluates every loss in one
    rbd_grad_batched call; the backward evaluates every gradient in one more."""

    @staticmethod
    def forward(ctx, d: int, w_rec: float, w_proj: float, count: int, *tensors):
        Xs = [rbd.as_colmajor(x.detach()) for x in tensors[:count]]
        Xos = [rbd.as_colmajor(x.detach()) if x.numel() else None for x in tensors[count:]]
        plan = rbd.BatchPlan([{"X": X, "tol": 0.0, "d_max": d} for X in Xs])
        plan.run()
        res = plan.results()
        items = []
        for i, (X, Xo, r) in enumerate(zip(Xs, Xos, res)):
            c = plan.compressed(i, r)
            items.append({"X": X, "Y": c.Y, "T": c.T, "pivots": c.pivots, "Xo": Xo})
        losses = rbd.grad_batched(items, w_rec, w_proj, need_grad=False)
        ctx.items = items
        ctx.plan = plan  # owns Y, T and pivots
        ctx.weights = (w_rec, w_proj)
        ctx.dtypes = [x.dtype for x in tensors[:count]]
        return torch.stack([l for _, l in losses]).to(tensors[0].dtype)

    @staticmethod
    def backward(ctx, gout):
        w_rec, w_proj = ctx.weights
        outs = rbd.grad_batched(ctx.items, w_rec, w_proj, need_grad=True)
        g = gout.to(torch.float64)
        grads = [(G * g[i]).to(dt) for i, ((G, _), dt) in enumerate(zip(outs, ctx.dtypes))]
        count = len(grads)
        return (None, None, None, None, *grads, *([None] * count))


def rbd_loss_batched(Xs, Xos=None, d: int = 32, w_rec: float = 1.0, w_proj: float = 1.0) -> torch.Tensor:
    """The losses of ``rbd_loss`` for a list of matrices (one storage type, float32 or float64, on
    one device) and their out-of-sample data (a list of the same length, entries may be None), as
    a 1-D tensor; differentiable with respect to every X for the pivot sets the forward chose."""
    count = len(Xs)
    if Xos is None:
        Xos = [None] * count
    empty = torch.empty(0, dtype=Xs[0].dtype, device=Xs[0].device)
    return RBDLossBatched.apply(d, w_rec, w_proj, count, *Xs, *[x if x is not None else empty for x in Xos])
