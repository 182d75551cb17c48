"""Differentiable back-projection and batched least squares.

``BackProject`` wraps bp_backproject (Listing 1) as a torch.autograd.Function
whose backward is the matched voxel-driven forward projector fp_project (the
exact transpose, same taps, weights and scale); ``ForwardProject`` is the
mirror, and ``ResidualLoss`` is 0.5 ||y - p||^2 with its gradient y - p.
``least_squares`` runs gradient descent on 0.5 ||A x - p||^2 with
A = fp_project, the gradient A^T (A x - p) coming from autograd through the
Functions, and the step 1/L with L the largest eigenvalue of A^T A estimated
by power iteration. The residual, its FP64 sum and the update are the
library's element-wise kernels (include/iter.h); PyTorch only holds the
tensors and runs the autograd graph.
"""
from __future__ import annotations

import ctypes
import math

import torch

from . import _lib, api


def _p(t: torch.Tensor):
    return ctypes.c_void_p(t.data_ptr())


def _s():
    return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)


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


class ResidualLoss(torch.autograd.Function):
    """loss = 0.5 ||y - p||^2 (FP64 sum of FP32 residuals); grad_y = g (y - p)."""

    @staticmethod
    def forward(fctx, y: torch.Tensor, p: torch.Tensor):
        y, p = y.contiguous(), p.contiguous()
        if y.shape != p.shape or y.dtype != torch.float32 or p.dtype != torch.float32:
            raise ValueError("y and p must be float32 tensors of one shape")
        r = torch.empty_like(y)
        loss = torch.empty((), dtype=torch.float64, device=y.device)
        _lib.check(_lib.load().it_ls_residual(_p(y), _p(p), _p(r), y.numel(), _p(loss), _s()))
        fctx.save_for_backward(r)
        return loss

    @staticmethod
    def backward(fctx, g: torch.Tensor):
        (r,) = fctx.saved_tensors
        # the kernel reads the upstream gradient on the device
        g = g.to(device=r.device, dtype=torch.float64).contiguous()
        out = torch.empty_like(r)
        _lib.check(_lib.load().it_scale(_p(r), _p(g), _p(out), r.numel(), _s()))
        return out, None


def gd_step(x: torch.Tensor, grad: torch.Tensor, step: float) -> torch.Tensor:
    """In place x = x - (step * grad) (two FP32 roundings)."""
    if not (x.is_contiguous() and grad.is_contiguous() and x.shape == grad.shape):
        raise ValueError("x and grad must be contiguous tensors of one shape")
    _lib.check(_lib.load().it_gd_step(_p(x), _p(grad), x.numel(), float(step), _s()))
    return x


def back_project(ctx: api.Context, proj: torch.Tensor, scale: float = 1.0) -> torch.Tensor:
    return BackProject.apply(proj, ctx, scale)


def forward_project(ctx: api.Context, vol: torch.Tensor, scale: float = 1.0) -> torch.Tensor:
    return ForwardProject.apply(vol, ctx, scale)


def lipschitz(ctx: api.Context, batch: int = 1, iters: int = 20, seed: int = 0) -> float:
    """Largest eigenvalue of A^T A (A = fp_project, scale 1) by power iteration.

    Norms are FP64 sums of the FP32 values (it_ls_residual against zeros) and
    the normalisation is it_scale; the start vector is seeded uniform noise."""
    gen = torch.Generator(device="cuda").manual_seed(seed)
    shape = ctx.vol_shape() if batch == 1 else ctx.vol_shape(batch)
    x = torch.rand(shape, device="cuda", generator=gen, dtype=torch.float32)
    zeros = torch.zeros_like(x)
    scratch = torch.empty_like(x)
    sq = torch.empty((), dtype=torch.float64, device="cuda")
    lib = _lib.load()

    def norm(t: torch.Tensor) -> float:
        _lib.check(lib.it_ls_residual(_p(t), _p(zeros), _p(scratch), t.numel(), _p(sq), _s()))
        return math.sqrt(2.0 * float(sq))

    def scaled(t: torch.Tensor, c: float) -> torch.Tensor:
        s = torch.tensor(c, dtype=torch.float64, device="cuda")
        _lib.check(lib.it_scale(_p(t), _p(s), _p(t), t.numel(), _s()))
        return t

    x = scaled(x, 1.0 / norm(x))
    lam = 0.0
    for _ in range(iters):
        y = api.bp_backproject(ctx, api.fp_project(ctx, x))
        lam = norm(y)
        x = scaled(y, 1.0 / lam)
    api.bp_device_status(ctx)
    return lam


def loss_fn(ctx: api.Context, x: torch.Tensor, p: torch.Tensor) -> torch.Tensor:
    """0.5 * ||A x - p||^2 through the autograd Functions (FP64 reduction)."""
    return ResidualLoss.apply(forward_project(ctx, x), p)


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
    x = x.contiguous()
    losses = []
    for it in range(iters):
        x.requires_grad_(True)
        loss = loss_fn(ctx, x, p)
        (grad,) = torch.autograd.grad(loss, x)
        losses.append(loss.detach())
        x = gd_step(x.detach(), grad, step)
        if callback is not None:
            callback(it, x)
    with torch.no_grad():
        losses.append(loss_fn(ctx, x, p))
    # a device error of any projector launch surfaces here
    api.bp_device_status(ctx)
    return x, [float(v) for v in torch.stack(losses).cpu()]


__all__ = ["BackProject", "ForwardProject", "ResidualLoss", "back_project", "forward_project", "gd_step",
           "lipschitz", "loss_fn", "least_squares"]
