"""The staged back-projectors at every pipeline depth against the FP64 oracle.

The depth is the number of views the staging producer keeps in flight (the
GPU form of the view batching and prefetching of Section 3.1.3 and
Algorithm 2). It changes the slot and phase counters of both staged kernels,
so each depth is checked on its own: the mid-plane symmetric kernel and the
plain z-column kernel, FP32 and FP16-stored projections, on a centred c1-type
geometry whose volume is ragged in x, y and z (odd nz, so the symmetric
kernel also writes a middle slice that is its own mirror). The data are
filtered projections of the c1 ellipsoid phantom.

A second case is the plan's own choice: the paper's problem P7 (a 1024^2
detector over a 256^3 volume, few views) has boxes too large for four stages,
so the plan lowers the depth by itself; sampled voxels are compared.
"""
import math

import numpy as np
import pytest
import torch

import oracle
from paper_2104_13248_gb300 import api, inputs

pytestmark = pytest.mark.gpu

TOL32 = 1e-5
TOL16 = 2e-3


def rel(a, b):
    return float(np.abs(np.asarray(a, np.float64) - b).max() / max(np.abs(b).max(), 1e-300))


@pytest.fixture(scope="module", autouse=True)
def _built():
    import __graft_entry__
    __graft_entry__.build()


@pytest.fixture(scope="module")
def case():
    p = inputs.preset("c1_small")
    g = dict(p["geom"], nx=61, ny=53, nz=45)
    E = inputs.random_ellipsoids(p["seed"], p["n_ell"], p["axes"], p["geom"])
    q = oracle.ramp_filter(g, oracle.phantom_project(g, E)).astype(np.float32)
    q16 = q.astype(np.float16)
    P = oracle.matrices(g)
    scale = math.pi / g["np"]
    ref = oracle.backproject(P, q, g["nx"], g["ny"], g["nz"], scale)
    ref16 = oracle.backproject(P, q16.astype(np.float64), g["nx"], g["ny"], g["nz"], scale)
    return dict(g=g, q=q, q16=q16, ref=ref, ref16=ref16, scale=scale)


@pytest.mark.parametrize("stages", [1, 2, 3, 4, 6, 8])
@pytest.mark.parametrize("sym", [True, False], ids=["sym", "plain"])
def test_depth_fp32(case, stages, sym):
    g = case["g"]
    with api.bp_create(g) as ctx:
        api.bp_set_symmetry(ctx, sym)
        api.bp_set_pipeline_depth(ctx, stages)
        plan = api.bp_get_plan(ctx)
        assert plan["stages"] == stages and plan["bu32"] > 0
        if sym and not plan["symmetric"]:
            # the symmetric kernel stages two boxes per view: 2 x 8 may not fit
            assert stages == 8
            pytest.skip("two boxes per stage do not fit at depth 8")
        assert plan["symmetric"] == sym
        vol = api.bp_backproject(ctx, torch.from_numpy(case["q"]).cuda(), scale=case["scale"]).cpu().numpy()
        api.bp_device_status(ctx)
    e = rel(vol, case["ref"])
    print(f"depth {stages} {'sym' if sym else 'plain'} FP32 rel err {e:.2e}")
    assert e <= TOL32


@pytest.mark.parametrize("stages", [1, 2, 3, 4, 6, 8])
def test_depth_fp16(case, stages):
    """FP16-stored projections (the plain z-column kernel, scalar taps)."""
    g = case["g"]
    with api.bp_create(g) as ctx:
        api.bp_set_pipeline_depth(ctx, stages)
        plan = api.bp_get_plan(ctx)
        assert plan["stages"] == stages and plan["bu16"] > 0
        vol = api.bp_backproject(ctx, torch.from_numpy(case["q16"]).cuda(), scale=case["scale"]).cpu().numpy()
        api.bp_device_status(ctx)
    e, e16 = rel(vol, case["ref"]), rel(vol, case["ref16"])
    print(f"depth {stages} FP16-stored rel err {e:.2e} (vs quantised input {e16:.2e})")
    assert e <= TOL16
    assert e16 <= TOL32


def test_plan_lowers_depth_for_large_boxes():
    """P7 (1024^2 -> 256^3) with 12 views: four FP32 stages do not fit shared
    memory, the plan runs fewer (at least 2), and 3000 sampled voxels, the
    corners among them, match the oracle for FP32 and FP16-stored data."""
    g = inputs.paper_problem("P7", views=12)
    q = inputs.uniform_array(78, (g["np"], g["nv"], g["nu"]), 0.0, 1.0).astype(np.float32)
    rng = np.random.default_rng(9)
    n = g["nx"]
    ijk = rng.integers(0, n, size=(3000, 3))
    ijk[:8] = [[a, b, c] for a in (0, n - 1) for b in (0, n - 1) for c in (0, n - 1)]
    scale = math.pi / g["np"]
    with api.bp_create(g) as ctx:
        plan = api.bp_get_plan(ctx)
        print("P7 plan", plan)
        assert plan["bu32"] > 0 and 2 <= plan["stages"] < 4
        assert plan["bu16"] > 0
        d = torch.from_numpy(q).cuda()
        vol = api.bp_backproject(ctx, d, scale=scale)
        got = vol[ijk[:, 2], ijk[:, 1], ijk[:, 0]].cpu().numpy()
        vol16 = api.bp_backproject(ctx, d.half(), scale=scale)
        got16 = vol16[ijk[:, 2], ijk[:, 1], ijk[:, 0]].cpu().numpy()
        api.bp_device_status(ctx)
    P = oracle.matrices(g)
    ref = oracle.backproject_points(P, q, ijk, scale)
    ref16 = oracle.backproject_points(P, q.astype(np.float16).astype(np.float64), ijk, scale)
    e, e16 = rel(got, ref), rel(got16, ref16)
    print(f"P7 sampled: FP32 rel err {e:.2e}, FP16-stored vs quantised {e16:.2e}")
    assert e <= TOL32
    assert e16 <= TOL32
    assert rel(got16, ref) <= TOL16
