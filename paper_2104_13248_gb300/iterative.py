"""Iterative reconstruction on the projector pair: MLEM / ordered-subset EM
(Shepp and Vardi; Hudson and Larkin) and block SART (Andersen and Kak), the
methods the paper names as calling back-projection repeatedly (Section 1).

A is fp_project and A^T bp_backproject (scale 1). View subset t holds views
t, t + n, t + 2n, ... of n subsets and has its own context built from those
views' matrices, so A_t and A_t^T are the same kernels on fewer views. Every
arithmetic step runs in libbp (include/iter.h for the element-wise parts);
this module only allocates buffers and orders the calls. Per subset:

  MLEM  y = A_t x;  r = p_t / y;  x <- x (A_t^T r) / (A_t^T 1)
  SART  y = A_t x;  r = (p_t - y) / (A_t 1);  x <- x + lambda (A_t^T r) / (A_t^T 1)
"""
from __future__ import annotations

import ctypes

import numpy as np
import torch

from . import _lib, api
from ._lib import check


def _p(t: torch.Tensor):
    return ctypes.c_void_p(t.data_ptr())


def _s():
    return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)


def fill(x: torch.Tensor, value: float) -> torch.Tensor:
    check(_lib.load().it_fill(_p(x), x.numel(), float(value), _s()))
    return x


class Subsets:
    """Contexts and normalisations of n interleaved view subsets of a geometry."""

    def __init__(self, ctx: api.Context, n: int, need_rays: bool):
        if n < 1 or n > ctx.n_views:
            raise ValueError("subsets must be in [1, number of views]")
        P = api.bp_get_matrices(ctx)
        self.n = n
        self.views = [np.arange(t, ctx.n_views, n) for t in range(n)]
        self.ctx = [ctx] if n == 1 else [api.bp_create_from_matrices(P[v], ctx.nu, ctx.nv, ctx.nx, ctx.ny,
                                                                      ctx.nz) for v in self.views]
        self.owned = n > 1
        vol_shape = ctx.vol_shape()
        self.sens, self.rays = [], []
        for c in self.ctx:
            ones_p = fill(torch.empty(c.proj_shape(), device="cuda"), 1.0)
            self.sens.append(api.bp_backproject(c, ones_p, scale=1.0))          # A_t^T 1
            if need_rays:
                ones_v = fill(torch.empty(vol_shape, device="cuda"), 1.0)
                self.rays.append(api.fp_project(c, ones_v, scale=1.0))          # A_t 1
        self.y = [torch.empty(c.proj_shape(), device="cuda") for c in self.ctx]
        self.b = torch.empty(vol_shape, device="cuda")

    def data(self, p: torch.Tensor):
        """The measured projections of each subset (contiguous copies)."""
        if self.n == 1:
            return [p.contiguous()]
        return [p[torch.as_tensor(v, device=p.device)].contiguous() for v in self.views]

    def close(self):
        if self.owned:
            for c in self.ctx:
                c.close()
        self.ctx = []


def mlem(ctx: api.Context, p: torch.Tensor, iters: int, subsets: int = 1, x0: torch.Tensor | None = None,
         eps: float = 1e-9, sub: Subsets | None = None) -> torch.Tensor:
    """MLEM (subsets = 1) or OS-EM: ``iters`` passes over all subsets."""
    lib = _lib.load()
    own = sub is None
    sub = sub or Subsets(ctx, subsets, need_rays=False)
    try:
        x = fill(torch.empty(ctx.vol_shape(), device="cuda"), 1.0) if x0 is None else x0.clone()
        pt = sub.data(p)
        n_vox = x.numel()
        for _ in range(iters):
            for t, c in enumerate(sub.ctx):
                y = api.fp_project(c, x, proj=sub.y[t], scale=1.0)
                check(lib.it_ratio(_p(pt[t]), _p(y), _p(y), y.numel(), float(eps), _s()))
                b = api.bp_backproject(c, y, vol=sub.b, scale=1.0)
                check(lib.it_mlem_update(_p(x), _p(b), _p(sub.sens[t]), n_vox, float(eps), _s()))
        return x
    finally:
        if own:
            sub.close()


def sart(ctx: api.Context, p: torch.Tensor, iters: int, subsets: int = 1, lam: float = 1.0,
         nonneg: bool = False, x0: torch.Tensor | None = None, eps: float = 1e-9,
         sub: Subsets | None = None) -> torch.Tensor:
    """Block SART over view subsets (SIRT when subsets = 1)."""
    lib = _lib.load()
    own = sub is None
    sub = sub or Subsets(ctx, subsets, need_rays=True)
    try:
        x = torch.zeros(ctx.vol_shape(), device="cuda") if x0 is None else x0.clone()
        pt = sub.data(p)
        n_vox = x.numel()
        for _ in range(iters):
            for t, c in enumerate(sub.ctx):
                y = api.fp_project(c, x, proj=sub.y[t], scale=1.0)
                check(lib.it_residual(_p(pt[t]), _p(y), _p(sub.rays[t]), _p(y), y.numel(), float(eps), _s()))
                b = api.bp_backproject(c, y, vol=sub.b, scale=1.0)
                check(lib.it_sart_update(_p(x), _p(b), _p(sub.sens[t]), n_vox, float(lam), 1 if nonneg else 0,
                                         float(eps), _s()))
        return x
    finally:
        if own:
            sub.close()


__all__ = ["Subsets", "fill", "mlem", "sart"]
