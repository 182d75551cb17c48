"""Python face of libbp: the C-ABI calls under the same names, on torch tensors.

PyTorch provides device memory and the current CUDA stream; each function
checks shapes and dtypes, passes raw pointers to the library and raises
``BPError`` on a non-OK status. No arithmetic of the method happens here.
"""
from __future__ import annotations

import ctypes
import math

import numpy as np
import torch

from . import _lib
from ._lib import BP_F16, BP_F32, BPError, check


def _stream(t: torch.Tensor | None = None):
    dev = t.device if t is not None else torch.device("cuda", torch.cuda.current_device())
    return ctypes.c_void_p(torch.cuda.current_stream(dev).cuda_stream)


def _ptr(t: torch.Tensor):
    return ctypes.c_void_p(t.data_ptr())


def _dtype_code(t: torch.Tensor) -> int:
    if t.dtype == torch.float32:
        return BP_F32
    if t.dtype == torch.float16:
        return BP_F16
    raise TypeError(f"projections must be float32 or float16, got {t.dtype}")


def _need_cuda(t: torch.Tensor, name: str):
    if not (isinstance(t, torch.Tensor) and t.is_cuda):
        raise ValueError(f"{name} must be a CUDA tensor")
    if not t.is_contiguous():
        raise ValueError(f"{name} must be contiguous")


class Context:
    """Owns one ``bp_ctx`` (geometry, matrices, plan, device tables)."""

    def __init__(self, handle: ctypes.c_void_p, geom: dict | None):
        self._h = handle
        self.geom = geom
        lib = _lib.load()
        d = [ctypes.c_int() for _ in range(6)]
        check(lib.bp_get_dims(self._h, *[ctypes.byref(x) for x in d]), self._h)
        self.n_views, self.nu, self.nv, self.nx, self.ny, self.nz = (x.value for x in d)

    @property
    def handle(self):
        if self._h is None:
            raise ValueError("context destroyed")
        return self._h

    def close(self):
        if self._h is not None:
            _lib.load().bp_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()
        return False

    # shapes ---------------------------------------------------------------
    def proj_shape(self, batch: int | None = None):
        s = (self.n_views, self.nv, self.nu)
        return s if batch is None else (batch,) + s

    def vol_shape(self, batch: int | None = None):
        s = (self.nz, self.ny, self.nx)
        return s if batch is None else (batch,) + s

    def _batch_of(self, t: torch.Tensor, tail: tuple, name: str) -> int:
        if tuple(t.shape) == tail:
            return 1
        if t.dim() == len(tail) + 1 and tuple(t.shape[1:]) == tail:
            return t.shape[0]
        raise ValueError(f"{name} has shape {tuple(t.shape)}, expected {tail} or (B,)+{tail}")


def bp_create(geom: dict) -> Context:
    """Context from a circular geometry dict (keys of ``inputs.PRESETS[...]['geom']``)."""
    lib = _lib.load()
    g = _lib.bp_geometry()
    g.sid, g.sdd, g.n_views = geom["sid"], geom["sdd"], geom["np"]
    ang = geom.get("angles")
    keep = None
    if ang is not None:
        keep = np.ascontiguousarray(ang, dtype=np.float64)
        if keep.shape != (geom["np"],):
            raise ValueError("angles must have np entries")
        g.angles = keep.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
    g.nu, g.nv, g.du, g.dv = geom["nu"], geom["nv"], geom["du"], geom["dv"]
    g.u_off_px, g.v_off_px = geom.get("u_off", 0.0), geom.get("v_off", 0.0)
    g.nx, g.ny, g.nz = geom["nx"], geom["ny"], geom["nz"]
    g.sx, g.sy, g.sz = geom["sx"], geom["sy"], geom["sz"]
    g.ox, g.oy, g.oz = geom.get("ox", 0.0), geom.get("oy", 0.0), geom.get("oz", 0.0)
    h = ctypes.c_void_p()
    check(lib.bp_create(ctypes.byref(g), ctypes.byref(h)), None)
    return Context(h, dict(geom))


def bp_create_from_matrices(P, nu: int, nv: int, nx: int, ny: int, nz: int) -> Context:
    """Context from explicit [np][3][4] FP64 matrices acting on (i, j, k, 1)."""
    lib = _lib.load()
    P = np.ascontiguousarray(P, dtype=np.float64).reshape(-1, 12)
    h = ctypes.c_void_p()
    check(lib.bp_create_from_matrices(P.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), P.shape[0],
                                      nu, nv, nx, ny, nz, ctypes.byref(h)), None)
    return Context(h, None)


def bp_destroy(ctx: Context) -> None:
    ctx.close()


def bp_get_matrices(ctx: Context) -> np.ndarray:
    P = np.zeros((ctx.n_views, 3, 4), dtype=np.float64)
    check(_lib.load().bp_get_matrices(ctx.handle, P.ctypes.data_as(ctypes.POINTER(ctypes.c_double))),
          ctx.handle)
    return P


def bp_get_plan(ctx: Context) -> dict:
    v = [ctypes.c_int() for _ in range(6)]
    check(_lib.load().bp_get_plan(ctx.handle, *[ctypes.byref(x) for x in v]), ctx.handle)
    return dict(tk=v[0].value, bu32=v[1].value, bu16=v[2].value, bv=v[3].value, stages=v[4].value,
                symmetric=bool(v[5].value))


def bp_set_tuning(ctx: Context, tk: int = 32, ctas_per_sm: int = 2) -> None:
    """Back-projector variant: voxels per thread along z and target CTAs per SM."""
    check(_lib.load().bp_set_tuning(ctx.handle, int(tk), int(ctas_per_sm)), ctx.handle)


def bp_set_pipeline_depth(ctx: Context, stages: int) -> None:
    """Views the back-projector's staging producer keeps in flight (1..8)."""
    check(_lib.load().bp_set_pipeline_depth(ctx.handle, int(stages)), ctx.handle)


def bp_set_symmetry(ctx: Context, enable: bool = True) -> None:
    """Allow (default) or forbid the mid-plane symmetry of FP32 back-projection;
    enabling raises BPError when the geometry is not mirror-symmetric about
    the central slice."""
    check(_lib.load().bp_set_symmetry(ctx.handle, 1 if enable else 0), ctx.handle)


def bp_set_timeout(ctx: Context, seconds: float) -> None:
    check(_lib.load().bp_set_timeout(ctx.handle, float(seconds)), ctx.handle)


def bp_test_drop_view(ctx: Context, view: int) -> None:
    check(_lib.load().bp_test_drop_view(ctx.handle, int(view)), ctx.handle)


def bp_device_status(ctx: Context, stream=None) -> None:
    """Synchronise the stream and raise if a kernel recorded an error."""
    st = stream if stream is not None else _stream()
    check(_lib.load().bp_device_status(ctx.handle, st), ctx.handle)


def bp_filter(ctx: Context, proj: torch.Tensor, out: torch.Tensor | None = None,
              out_dtype: torch.dtype = torch.float32) -> torch.Tensor:
    """Cosine weight + Ram-Lak filter of FP32 projections ([B,]np,nv,nu)."""
    _need_cuda(proj, "proj")
    if proj.dtype != torch.float32:
        raise TypeError("bp_filter input must be float32")
    batch = ctx._batch_of(proj, ctx.proj_shape(), "proj")
    if out is None:
        out = torch.empty(proj.shape, dtype=out_dtype, device=proj.device)
    _need_cuda(out, "out")
    if out.shape != proj.shape:
        raise ValueError("out must have the shape of proj")
    check(_lib.load().bp_filter(ctx.handle, _ptr(proj), _ptr(out), _dtype_code(out), batch,
                                _stream(proj)), ctx.handle)
    return out


def bp_filter_views(ctx: Context, proj: torch.Tensor, out: torch.Tensor) -> torch.Tensor:
    """Filter a contiguous ([B,]n,nv,nu) block of views into ``out`` (FP32 or FP16)."""
    _need_cuda(proj, "proj")
    _need_cuda(out, "out")
    if proj.dtype != torch.float32 or tuple(proj.shape[-2:]) != (ctx.nv, ctx.nu) or out.shape != proj.shape:
        raise ValueError("proj must be float32 (..., n, nv, nu) and out of the same shape")
    n = proj.shape[-3]
    batch = proj.numel() // (n * ctx.nv * ctx.nu)
    check(_lib.load().bp_filter_views(ctx.handle, _ptr(proj), _ptr(out), _dtype_code(out), n, batch,
                                      _stream(proj)), ctx.handle)
    return out


def bp_backproject(ctx: Context, proj: torch.Tensor, vol: torch.Tensor | None = None,
                   scale: float = 1.0, accumulate: bool = False) -> torch.Tensor:
    """Back-projection of ([B,]np,nv,nu) FP32/FP16 projections into FP32 volumes."""
    _need_cuda(proj, "proj")
    batch = ctx._batch_of(proj, ctx.proj_shape(), "proj")
    if vol is None:
        shape = ctx.vol_shape() if proj.dim() == 3 else ctx.vol_shape(batch)
        vol = torch.empty(shape, dtype=torch.float32, device=proj.device)
        accumulate = False
    _need_cuda(vol, "vol")
    if vol.dtype != torch.float32 or vol.numel() != batch * ctx.nx * ctx.ny * ctx.nz:
        raise ValueError("vol must be float32 with the volume's shape")
    check(_lib.load().bp_backproject(ctx.handle, _ptr(proj), _dtype_code(proj), _ptr(vol), batch,
                                     float(scale), int(bool(accumulate)), _stream(proj)), ctx.handle)
    return vol


def bp_backproject_views(ctx: Context, proj: torch.Tensor, view0: int, vol: torch.Tensor,
                         scale: float = 1.0, accumulate: bool = True) -> torch.Tensor:
    """Back-project views view0 .. view0+n-1 given as a ([B,]n,nv,nu) tensor (or a view of one)."""
    if not proj.is_cuda:
        raise ValueError("proj must be a CUDA tensor")
    if proj.dim() == 3:
        batch, n, bstride = 1, proj.shape[0], 0
    else:
        batch, n = proj.shape[0], proj.shape[1]
        bstride = proj.stride(0)
    block = proj if proj.dim() == 3 else proj[0]
    if tuple(proj.shape[-2:]) != (ctx.nv, ctx.nu) or not block.is_contiguous():
        raise ValueError("each batch entry of proj must be a contiguous (n, nv, nu) block")
    _need_cuda(vol, "vol")
    check(_lib.load().bp_backproject_views(ctx.handle, _ptr(proj), _dtype_code(proj), int(view0), int(n),
                                           int(bstride), _ptr(vol), batch, float(scale),
                                           int(bool(accumulate)), _stream(proj)), ctx.handle)
    return vol


def bp_backproject_slab(ctx: Context, proj: torch.Tensor, view0: int, z0: int, nz_slab: int, vol: torch.Tensor,
                        mirror: bool = False, scale: float = 1.0, accumulate: bool = True) -> torch.Tensor:
    """Back-project views view0 .. view0+n-1 into slices z0 .. z0+nz_slab-1 of vol
    (and, with mirror, the mirrored slices nz-z0-nz_slab .. nz-1-z0); the rest
    of vol is left as it is."""
    if not proj.is_cuda:
        raise ValueError("proj must be a CUDA tensor")
    if proj.dim() == 3:
        batch, n, bstride = 1, proj.shape[0], 0
    else:
        batch, n = proj.shape[0], proj.shape[1]
        bstride = proj.stride(0)
    block = proj if proj.dim() == 3 else proj[0]
    if tuple(proj.shape[-2:]) != (ctx.nv, ctx.nu) or not block.is_contiguous():
        raise ValueError("each batch entry of proj must be a contiguous (n, nv, nu) block")
    _need_cuda(vol, "vol")
    check(_lib.load().bp_backproject_slab(ctx.handle, _ptr(proj), _dtype_code(proj), int(view0), int(n),
                                          int(bstride), int(z0), int(nz_slab), int(bool(mirror)), _ptr(vol), batch,
                                          float(scale), int(bool(accumulate)), _stream(proj)), ctx.handle)
    return vol


def fp_project(ctx: Context, vol: torch.Tensor, proj: torch.Tensor | None = None,
               scale: float = 1.0) -> torch.Tensor:
    """Matched forward projection (exact transpose of bp_backproject with the same scale)."""
    _need_cuda(vol, "vol")
    if vol.dtype != torch.float32:
        raise TypeError("vol must be float32")
    batch = ctx._batch_of(vol, ctx.vol_shape(), "vol")
    if proj is None:
        shape = ctx.proj_shape() if vol.dim() == 3 else ctx.proj_shape(batch)
        proj = torch.empty(shape, dtype=torch.float32, device=vol.device)
    _need_cuda(proj, "proj")
    if proj.dtype != torch.float32 or proj.numel() != batch * ctx.n_views * ctx.nu * ctx.nv:
        raise ValueError("proj must be float32 with the projections' shape")
    check(_lib.load().fp_project(ctx.handle, _ptr(vol), _ptr(proj), batch, float(scale), _stream(vol)),
          ctx.handle)
    return proj


def bp_phantom_project(ctx: Context, ellipsoids, out: torch.Tensor | None = None) -> torch.Tensor:
    """Analytic line integrals of an ellipsoid list ([n][16], see ``inputs``) on the GPU."""
    E = np.ascontiguousarray(np.asarray(ellipsoids, dtype=np.float64).reshape(-1, 16))
    if out is None:
        out = torch.empty(ctx.proj_shape(), dtype=torch.float32, device="cuda")
    _need_cuda(out, "out")
    check(_lib.load().bp_phantom_project(ctx.handle, E.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
                                         E.shape[0], _ptr(out), _stream(out)), ctx.handle)
    return out


class HostPipeline:
    """FDK from host memory with the host-to-device and device-to-host copies
    overlapped with the computation.

    The volume is computed in ``slabs`` parts, each a range of lower slices
    with its mirror (one pass of the mid-plane symmetric kernel where it
    applies). Views are split into ``chunks`` blocks: while block c+1 is
    copied on a copy stream, block c is filtered and back-projected into the
    first part on the compute stream. The first block is small (``first`` of
    the views), since nothing overlaps its copy; the copy of a view is about
    3x faster than its back-projection, so the later blocks land before they
    are needed. The other parts then back-project every view, each part's
    slices going back to the host while the next part is computed, so only the
    last part's copy is exposed. Device buffers are allocated once, here.
    """

    def __init__(self, ctx: Context, chunks: int = 8, dtype: torch.dtype = torch.float32,
                 first: float = 0.04, slabs: int = 4):
        self.ctx = ctx
        self.chunks = max(1, min(int(chunks), ctx.n_views))
        # an optional small first block (fraction ``first`` of the views) shortens
        # the copy nothing can overlap; the rest is split evenly
        n0 = int(round(first * ctx.n_views)) if self.chunks > 1 else 0
        n0 = min(max(n0, 0), ctx.n_views - 1)
        rest = np.linspace(n0, ctx.n_views, self.chunks + (0 if n0 else 1)).round().astype(int)
        edges = ([0] if n0 else []) + list(rest)
        self.blocks = [(int(a), int(b)) for a, b in zip(edges[:-1], edges[1:]) if b > a]
        # parts: lower-slice ranges [z0, z1) of the (nz+1)//2 lower slices, each with its mirror;
        # edges on multiples of 64 where possible, so the parts cut along the kernels' z-tiles
        nlow = (ctx.nz + 1) // 2
        nparts = max(1, min(int(slabs), nlow))
        zs = [0]
        for k in range(1, nparts):
            z = int(round(k * nlow / nparts / 64)) * 64
            zs.append(z if zs[-1] < z < nlow else int(round(k * nlow / nparts)))
        zs.append(nlow)
        self.parts = [(a, b) for a, b in zip(zs[:-1], zs[1:]) if b > a]
        self.raw = torch.empty(ctx.proj_shape(), dtype=torch.float32, device="cuda")
        self.filt = torch.empty(ctx.proj_shape(), dtype=dtype, device="cuda")
        self.vol = torch.empty(ctx.vol_shape(), dtype=torch.float32, device="cuda")
        self.copy_stream = torch.cuda.Stream()
        self.events = [torch.cuda.Event() for _ in self.blocks]
        self.part_done = [torch.cuda.Event() for _ in self.parts]

    def _ranges(self, z0: int, z1: int):
        """Slice ranges a part covers: [z0, z1) and its mirror (the middle slice once)."""
        nz = self.ctx.nz
        m0, m1 = max(nz - z1, z1), nz - z0
        return [(z0, z1)] + ([(m0, m1)] if m1 > m0 else [])

    def run(self, proj_host: torch.Tensor, vol_host: torch.Tensor) -> torch.Tensor:
        """proj_host: pinned FP32 (np,nv,nu); vol_host: pinned FP32 (nz,ny,nx)."""
        comp = torch.cuda.current_stream()
        self.copy_stream.wait_stream(comp)
        with torch.cuda.stream(self.copy_stream):
            for (a, b), ev in zip(self.blocks, self.events):
                self.raw[a:b].copy_(proj_host[a:b], non_blocking=True)
                ev.record(self.copy_stream)
        scale = math.pi / self.ctx.n_views
        (p0, p1) = self.parts[0]
        for i, ((a, b), ev) in enumerate(zip(self.blocks, self.events)):
            comp.wait_event(ev)
            bp_filter_views(self.ctx, self.raw[a:b], self.filt[a:b])
            bp_backproject_slab(self.ctx, self.filt[a:b], a, p0, p1 - p0, self.vol, mirror=True, scale=scale,
                                accumulate=i > 0)
        for k, (z0, z1) in enumerate(self.parts):
            if k > 0:
                bp_backproject_slab(self.ctx, self.filt, 0, z0, z1 - z0, self.vol, mirror=True, scale=scale,
                                    accumulate=False)
            self.part_done[k].record(comp)
            self.copy_stream.wait_event(self.part_done[k])
            with torch.cuda.stream(self.copy_stream):
                for r0, r1 in self._ranges(z0, z1):
                    vol_host[r0:r1].copy_(self.vol[r0:r1], non_blocking=True)
        comp.wait_stream(self.copy_stream)
        return vol_host


def fdk(ctx: Context, proj: torch.Tensor, out_dtype: torch.dtype = torch.float32,
        filtered: torch.Tensor | None = None, vol: torch.Tensor | None = None) -> torch.Tensor:
    """Feldkamp reconstruction: bp_filter then bp_backproject with scale pi/np."""
    q = bp_filter(ctx, proj, out=filtered, out_dtype=out_dtype)
    return bp_backproject(ctx, q, vol=vol, scale=math.pi / ctx.n_views)


__all__ = ["Context", "BPError", "HostPipeline", "bp_filter_views", "bp_create", "bp_create_from_matrices", "bp_destroy", "bp_filter",
           "bp_backproject", "bp_backproject_views", "bp_backproject_slab", "fp_project", "bp_phantom_project",
           "bp_get_matrices", "bp_get_plan", "bp_set_tuning", "bp_set_pipeline_depth", "bp_set_symmetry", "bp_set_timeout",
           "bp_test_drop_view", "bp_device_status", "fdk"]
