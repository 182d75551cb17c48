"""Back-projection of a range of slices (bp_backproject_slab): only those
slices are written, mirrored slabs go through the mid-plane symmetric kernel
(Section 3.1.2) where it applies, slab-by-slab volumes equal the one-call
volume, and each slab matches the FP64 oracle's slices (Listing 1) at the
FP32 / FP16 tolerances of the other parity tests."""
import math

import numpy as np
import pytest
import torch

import oracle
from paper_2104_13248_gb300 import _lib, api, inputs
from tests.test_gpu_parity import TOL16, TOL32, rel

pytestmark = pytest.mark.gpu
SENTINEL = 12345.0


@pytest.fixture(scope="module", autouse=True)
def _built():
    import __graft_entry__
    __graft_entry__.build()


def _geom(nz, v_off=0.0):
    return dict(sid=700.0, sdd=1100.0, np=36, angles=None, nu=96, nv=96, du=0.9, dv=0.9, u_off=1.3, v_off=v_off,
                nx=40, ny=36, nz=nz, sx=0.8, sy=0.8, sz=0.8, ox=0.5, oy=-0.3, oz=0.0)


@pytest.mark.parametrize("nz,v_off", [(256, 0.0), (45, 0.0), (64, 0.7)], ids=["sym256", "sym_odd45", "offcentre64"])
@pytest.mark.parametrize("dtype", [torch.float32, torch.float16], ids=["f32", "f16"])
def test_slabs_against_oracle_and_full_volume(nz, v_off, dtype):
    g = _geom(nz, v_off)
    q = inputs.uniform_array(77 + nz, (g["np"], g["nv"], g["nu"]), -1.0, 1.0).astype(np.float32)
    scale = math.pi / g["np"]
    P = oracle.matrices(g)
    qd = torch.from_numpy(q).cuda().to(dtype)
    tol = TOL32 if dtype == torch.float32 else TOL16
    nlow = (nz + 1) // 2
    with api.bp_create(g) as ctx:
        full = api.bp_backproject(ctx, qd, scale=scale).clone()
        # a plain slab: exactly its slices are written
        z0, n = 5, 23
        vol = torch.full(ctx.vol_shape(), SENTINEL, device="cuda")
        api.bp_backproject_slab(ctx, qd, 0, z0, n, vol, mirror=False, scale=scale, accumulate=False)
        v = vol.cpu().numpy()
        assert np.all(v[:z0] == SENTINEL) and np.all(v[z0 + n:] == SENTINEL)
        ref = oracle.backproject_slab(P, q, g["nx"], g["ny"], z0, n, scale)
        assert rel(v[z0:z0 + n], ref) <= tol
        # mirrored slabs covering the lower half rebuild the whole volume
        vol = torch.full(ctx.vol_shape(), SENTINEL, device="cuda")
        tiled = nz % 128 == 0          # slab edges on multiples of 64
        edges = [0, 64, nlow] if tiled else [0, nlow // 3, nlow]
        for a, b in zip(edges[:-1], edges[1:]):
            api.bp_backproject_slab(ctx, qd, 0, a, b - a, vol, mirror=True, scale=scale, accumulate=False)
        v = vol.cpu().numpy()
        assert not np.any(v == SENTINEL)
        if tiled:
            assert torch.equal(vol, full)          # the slabs cut along the kernels' z-tiles
        else:
            # other z-tiles, other box-relative FP32 coordinates: equal to rounding, both within TOL32 of the oracle
            assert rel(v, full.cpu().numpy()) <= TOL32
        # and the mirrored part of one slab against the oracle
        a, b = edges[0], edges[1]
        m0, m1 = max(nz - b, b), nz - a
        ref = oracle.backproject_slab(P, q, g["nx"], g["ny"], m0, m1 - m0, scale)
        assert rel(v[m0:m1], ref) <= tol
        # view blocks accumulate into a slab as into the whole volume
        vol = torch.zeros(ctx.vol_shape(), device="cuda")
        for s0 in range(0, g["np"], 10):
            e = min(g["np"], s0 + 10)
            api.bp_backproject_slab(ctx, qd[s0:e].contiguous(), s0, 0, nlow, vol, mirror=True, scale=scale,
                                    accumulate=s0 > 0)
        assert rel(vol.cpu().numpy(), full.cpu().numpy()) <= TOL32
        api.bp_device_status(ctx)


def test_slab_argument_errors():
    g = _geom(45)
    q = torch.zeros((g["np"], g["nv"], g["nu"]), device="cuda")
    lib = _lib.load()
    with api.bp_create(g) as ctx:
        vol = torch.zeros(ctx.vol_shape(), device="cuda")

        def call(z0, n, mirror):
            return lib.bp_backproject_slab(ctx.handle, q.data_ptr(), 0, 0, g["np"], 0, z0, n, mirror,
                                           vol.data_ptr(), 1, 1.0, 0, None)

        assert call(-1, 4, 0) == _lib.BP_ERR_INVALID_ARG
        assert call(40, 6, 0) == _lib.BP_ERR_INVALID_ARG          # past nz
        assert call(0, 0, 0) == _lib.BP_ERR_INVALID_ARG
        assert call(20, 4, 1) == _lib.BP_ERR_INVALID_ARG          # mirrored slab past the lower half (23 slices)
        assert call(19, 4, 1) == _lib.BP_OK
        assert call(0, 45, 0) == _lib.BP_OK
        api.bp_device_status(ctx)
