"""Back-projection with the mid-plane symmetry (Section 3.1.2, Algorithm 1)
against the FP64 oracle: v, its floor and fraction are computed once for
voxels k and nz-1-k, whose taps come from the staged box and its vertical
mirror. Same tolerances as the plain kernel: 1e-5 max-relative for FP32
projections, 2e-3 for FP16-stored ones."""
import math

import numpy as np
import pytest
import torch

import oracle
from paper_2104_13248_gb300 import _lib, api, inputs
from tests.test_gpu_parity import TOL16, TOL32, _band, rel

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    import __graft_entry__
    __graft_entry__.build()


def _check(g, q, views_chunk=None):
    scale = math.pi / g["np"]
    P = oracle.matrices(g)
    ref = oracle.backproject(P, q, g["nx"], g["ny"], g["nz"], scale)
    ref16 = oracle.backproject(P, q.astype(np.float16).astype(np.float64), g["nx"], g["ny"], g["nz"], scale)
    with api.bp_create(g) as ctx:
        d = torch.from_numpy(q).cuda()
        assert api.bp_get_plan(ctx)["symmetric"]          # the default for centred geometries
        sym = api.bp_backproject(ctx, d, scale=scale).cpu().numpy()
        sym16 = api.bp_backproject(ctx, d.half(), scale=scale).cpu().numpy()
        api.bp_set_symmetry(ctx, False)
        assert not api.bp_get_plan(ctx)["symmetric"]
        plain = api.bp_backproject(ctx, d, scale=scale).cpu().numpy()
        plain16 = api.bp_backproject(ctx, d.half(), scale=scale).cpu().numpy()
        api.bp_set_symmetry(ctx, True)
        if views_chunk:
            # accumulate over view ranges through the same symmetric kernel
            acc = torch.zeros(ctx.vol_shape(), device="cuda")
            for v0 in range(0, g["np"], views_chunk):
                n = min(views_chunk, g["np"] - v0)
                api.bp_backproject_views(ctx, d[v0:v0 + n].contiguous(), v0, acc, scale=scale, accumulate=True)
            assert rel(acc.cpu().numpy(), ref) <= TOL32
        api.bp_device_status(ctx)
    assert rel(sym, ref) <= TOL32
    assert rel(plain, ref) <= TOL32
    # FP16-stored projections (the plain kernel either way): against the
    # unquantised values, and the FP32 arithmetic on the quantised values
    assert rel(sym16, ref) <= TOL16
    assert rel(plain16, ref) <= TOL16
    assert rel(sym16, ref16) <= TOL32
    assert rel(plain16, ref16) <= TOL32
    return sym, plain


def test_symmetry_c1():
    p = inputs.preset("c1_small")
    g = p["geom"]
    E = inputs.random_ellipsoids(p["seed"], p["n_ell"], p["axes"], g)
    q = oracle.ramp_filter(g, oracle.phantom_project(g, E)).astype(np.float32)
    _check(g, q, views_chunk=37)


@pytest.mark.parametrize("n", [(45, 38, 37), (33, 70, 50), (40, 40, 1)])
def test_symmetry_ragged_and_odd(n):
    """Odd nz (the middle slice is its own mirror and is written once), a last
    half-block shorter than 16 slices, ragged x / y tiles, a single slice."""
    nx, ny, nz = n
    g = dict(sid=700.0, sdd=1100.0, np=40, angles=None, nu=96, nv=80, du=0.9, dv=0.9, u_off=1.4, v_off=0.0,
             nx=nx, ny=ny, nz=nz, sx=0.8, sy=0.8, sz=0.8, ox=0.7, oy=-0.4, oz=0.0)
    q = inputs.uniform_array(123 + nz, (g["np"], g["nv"], g["nu"]), -1.0, 1.0).astype(np.float32)
    _check(g, q)


def test_symmetry_needs_a_centred_geometry():
    g = inputs.preset("c1_small")["geom"]
    g = dict(g, v_off=0.5)
    with api.bp_create(g) as ctx:
        assert not api.bp_get_plan(ctx)["symmetric"]      # off-centre: the plain kernel
        with pytest.raises(_lib.BPError) as e:
            api.bp_set_symmetry(ctx, True)
        assert e.value.status == _lib.BP_ERR_UNSUPPORTED
    g = dict(inputs.preset("c1_small")["geom"], oz=0.3)
    with api.bp_create(g) as ctx:
        with pytest.raises(_lib.BPError):
            api.bp_set_symmetry(ctx, True)


def test_symmetry_full_size_slab():
    """c3 (the benchmark's workload) with the symmetric kernel: the slab
    k = 224..287 straddles the mid-plane (lower slices and mirrors)."""
    p = inputs.preset("c3_paper")
    g = p["geom"]
    P = oracle.matrices(g)
    E = inputs.random_ellipsoids(p["seed"], p["n_ell"], p["axes"], g)
    k0, nks = 224, 64
    r0, nr = _band(P, g, k0, nks)
    raw = oracle.phantom_project_rows(g, E, r0, nr)
    qb = oracle.ramp_filter_rows(g, raw, r0).astype(np.float32)
    q = np.zeros((g["np"], g["nv"], g["nu"]), dtype=np.float32)
    q[:, r0:r0 + nr, :] = qb
    scale = math.pi / g["np"]
    ref = oracle.backproject_slab(P, q, g["nx"], g["ny"], k0, nks, scale)
    with api.bp_create(g) as ctx:
        api.bp_set_symmetry(ctx, True)
        vol = api.bp_backproject(ctx, torch.from_numpy(q).cuda(), scale=scale)
        slab = vol[k0:k0 + nks].cpu().numpy()
        api.bp_device_status(ctx)
    assert rel(slab, ref) <= TOL32
