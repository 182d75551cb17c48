"""Differentiable back-projection and batched least squares.

``BackProject`` wraps bp_backproject (Listing 1) as a torch.autograd.Function
whose backward is the matched voxel-driven forward projector fp_project (the
exact transpose, same taps, weights and scale); ``ForwardProject`` is the
mirror. ``least_squares`` runs gradient descent on 0.5 ||A x - p||^2 with
A = fp_project, the gradient A^T (A x - p) coming from autograd through the
two Functions, and the step 1/L with L the largest eigenvalue of A^T A
estimated by power iteration.
"""
from __future__ import annotations

import math

import torch

from . import api


class BackProject(torch.autograd.Function):
    """vol = scale * A^T proj; grad_proj = scale * A grad_vol."""

    @staticmethod
    def forward(fctx, proj: torch.Tensor, ctx: api.Context, scale: float):
        fctx.bp = ctx
        fctx.scale = float(scale)
        return api.bp_backproject(ctx, proj.contiguous(), scale=scale)

    @staticmethod
    def backward(fctx, grad_vol: torch.Tensor):
        g = api.fp_project(fctx.bp, grad_vol.contiguous(), scale=fctx.scale)
        return g, None, None


class ForwardProject(torch.autograd.Function):
    """proj = scale * A vol; grad_vol = scale * A^T grad_proj."""

    @staticmethod
    def forward(fctx, vol: torch.Tensor, ctx: api.Context, scale: float):
        fctx.bp = ctx
        fctx.scale = float(scale)
        return api.fp_project(ctx, vol.contiguous(), scale=scale)

    @staticmethod
    def backward(fctx, grad_proj: torch.Tensor):
        g = api.bp_backproject(fctx.bp, grad_proj.contiguous(), scale=fctx.scale)
        return g, None, None


def back_project(ctx: api.Context, proj: torch.Tensor, scale: float = 1.0) -> torch.Tensor:
    return BackProject.apply(proj, ctx, scale)


def forward_project(ctx: api.Context, vol: torch.Tensor, scale: float = 1.0) -> torch.Tensor:
    return ForwardProject.apply(vol, ctx, scale)


def _norm64(t: torch.Tensor) -> float:
    """Euclidean norm with an FP64 reduction of FP32 values."""
    return float(torch.linalg.vector_norm(t.double()).item())


def lipschitz(ctx: api.Context, batch: int = 1, iters: int = 20, seed: int = 0) -> float:
    """Largest eigenvalue of A^T A (A = fp_project, scale 1) by power iteration."""
    gen = torch.Generator(device="cuda").manual_seed(seed)
    shape = ctx.vol_shape() if batch == 1 else ctx.vol_shape(batch)
    x = torch.rand(shape, device="cuda", generator=gen, dtype=torch.float32)
    x /= _norm64(x)
    lam = 0.0
    for _ in range(iters):
        y = api.bp_backproject(ctx, api.fp_project(ctx, x))
        lam = _norm64(y)
        x = y / lam
    return lam


def loss_fn(ctx: api.Context, x: torch.Tensor, p: torch.Tensor) -> torch.Tensor:
    """0.5 * ||A x - p||^2 through the autograd Functions (FP64 reduction)."""
    r = forward_project(ctx, x) - p
    return 0.5 * (r.double() ** 2).sum()


def least_squares(ctx: api.Context, p: torch.Tensor, iters: int = 20, x0: torch.Tensor | None = None,
                  L: float | None = None, callback=None):
    """Gradient descent x <- x - (1/L) A^T (A x - p) on a batch of problems.

    p: measured projections ([B,]np,nv,nu). Returns (x, losses) where
    losses[i] is the loss before iteration i (and the final one last).
    """
    batch = 1 if p.dim() == 3 else p.shape[0]
    if L is None:
        L = lipschitz(ctx, batch=1)
    step = 1.0 / L
    shape = ctx.vol_shape() if p.dim() == 3 else ctx.vol_shape(batch)
    x = torch.zeros(shape, device=p.device, dtype=torch.float32) if x0 is None else x0.clone()
    losses = []
    for it in range(iters):
        x.requires_grad_(True)
        loss = loss_fn(ctx, x, p)
        (grad,) = torch.autograd.grad(loss, x)
        losses.append(float(loss.item()))
        with torch.no_grad():
            x = x - step * grad
        if callback is not None:
            callback(it, x)
    with torch.no_grad():
        losses.append(float(loss_fn(ctx, x, p).item()))
    return x.detach(), losses


__all__ = ["BackProject", "ForwardProject", "back_project", "forward_project", "lipschitz",
           "loss_fn", "least_squares"]
