"""CUDA path vs the FP64 oracle, element by element, on the same seeded inputs.

Tolerances (max |gpu - oracle| / max |oracle|): 1e-5 for every FP32 path
(back-projection, forward projection, the FFT ramp filter and FDK end to end;
on uniform noise as well as on phantom data), 2e-3 for FP16-stored
projections (against the unquantised input), 1e-4 for the FP32 phantom
generator (input data only).
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
def c1():
    p = inputs.preset("c1_small")
    g = p["geom"]
    E = inputs.random_ellipsoids(p["seed"], p["n_ell"], p["axes"], g)
    raw = oracle.phantom_project(g, E).astype(np.float32)
    q = oracle.ramp_filter(g, raw).astype(np.float32)
    return dict(g=g, E=E, raw=raw, q=q, P=oracle.matrices(g))


def test_backproject_c1(c1):
    g = c1["g"]
    scale = math.pi / g["np"]
    ref = oracle.backproject(c1["P"], c1["q"], g["nx"], g["ny"], g["nz"], scale)
    with api.bp_create(g) as ctx:
        vol = api.bp_backproject(ctx, torch.from_numpy(c1["q"]).cuda(), scale=scale).cpu().numpy()
        api.bp_device_status(ctx)
    print(f"back-projection c1 rel err {rel(vol, ref):.2e}")
    assert rel(vol, ref) <= TOL32


def test_filter_c1(c1):
    g = c1["g"]
    ref = oracle.ramp_filter(g, c1["raw"])
    with api.bp_create(g) as ctx:
        out = api.bp_filter(ctx, torch.from_numpy(c1["raw"]).cuda()).cpu().numpy()
        out16 = api.bp_filter(ctx, torch.from_numpy(c1["raw"]).cuda(), out_dtype=torch.float16).cpu().numpy()
    print(f"filter c1 rel err {rel(out, ref):.2e}")
    assert rel(out, ref) <= TOL32
    # FP16 output = round-to-nearest of the FP32 result
    assert rel(out16.astype(np.float64), ref) <= 1e-3


@pytest.mark.parametrize("nu", [8, 20, 33, 100, 300, 512, 600, 700, 1248, 1900, 2100, 3000, 4600, 5200])
def test_filter_sizes(nu):
    """Every transform size: N = 32 .. 8192 and 1280 .. 10240 (the four-row
    kernel, radices 16 and 2/4/5/8/10) and N = 16384 (the two-row kernel);
    21 rows, so the last four-row group is ragged."""
    g = dict(sid=800.0, sdd=1300.0, np=3, angles=None, nu=nu, nv=7, du=0.45, dv=0.5, u_off=1.2,
             v_off=-0.8, nx=8, ny=8, nz=8, sx=1.0, sy=1.0, sz=1.0, ox=0, oy=0, oz=0)
    raw = inputs.uniform_array(40 + nu, (g["np"], g["nv"], g["nu"]), 0.0, 2.0).astype(np.float32)
    ref = oracle.ramp_filter(g, raw)
    with api.bp_create(g) as ctx:
        out = api.bp_filter(ctx, torch.from_numpy(raw).cuda()).cpu().numpy()
        out16 = api.bp_filter(ctx, torch.from_numpy(raw).cuda(), out_dtype=torch.float16).cpu().numpy()
    print(f"filter nu={nu} rel err {rel(out, ref):.2e}")
    assert rel(out, ref) <= TOL32
    assert rel(out16.astype(np.float64), ref) <= 1e-3


def test_host_pipeline_matches_device_fdk(c1):
    g = c1["g"]
    with api.bp_create(g) as ctx:
        dev = torch.from_numpy(c1["raw"]).cuda()
        ref = api.fdk(ctx, dev).cpu().numpy()
        host = torch.from_numpy(c1["raw"]).pin_memory()
        vol_host = torch.empty(ctx.vol_shape(), dtype=torch.float32).pin_memory()
        pipe = api.HostPipeline(ctx, chunks=7)
        for _ in range(2):
            pipe.run(host, vol_host)
            torch.cuda.synchronize()
            assert rel(vol_host.numpy(), ref) <= 1e-6


def test_fdk_end_to_end_c1(c1):
    g = c1["g"]
    ref = oracle.fdk(g, c1["raw"])
    with api.bp_create(g) as ctx:
        vol = api.fdk(ctx, torch.from_numpy(c1["raw"]).cuda()).cpu().numpy()
    print(f"FDK c1 rel err {rel(vol, ref):.2e}")
    assert rel(vol, ref) <= TOL32


def test_backproject_fp16_c1(c1):
    g = c1["g"]
    scale = math.pi / g["np"]
    ref = oracle.backproject(c1["P"], c1["q"], g["nx"], g["ny"], g["nz"], scale)
    q16 = c1["q"].astype(np.float16)
    ref16 = oracle.backproject(c1["P"], q16.astype(np.float64), g["nx"], g["ny"], g["nz"], scale)
    with api.bp_create(g) as ctx:
        vol = api.bp_backproject(ctx, torch.from_numpy(q16).cuda(), scale=scale).cpu().numpy()
        api.bp_device_status(ctx)
    assert rel(vol, ref) <= TOL16          # against the unquantised input
    assert rel(vol, ref16) <= TOL32        # the arithmetic itself stays FP32-accurate


RAGGED = [
    # TMA path (nu*4 and nu*2 multiples of 16), ragged tiles in x, y and z
    dict(nu=96, nv=70, nx=37, ny=29, nz=45),
    # nu*4 multiple of 16 but nu*2 not: FP32 via TMA, FP16 via global loads
    dict(nu=52, nv=40, nx=33, ny=9, nz=70),
    # nu*4 not a multiple of 16: global-load kernel for both types
    dict(nu=50, nv=44, nx=31, ny=17, nz=33),
    # a single voxel and a thin slab
    dict(nu=64, nv=64, nx=1, ny=1, nz=1),
    dict(nu=64, nv=64, nx=40, ny=40, nz=2),
]


@pytest.mark.parametrize("dims", RAGGED, ids=lambda d: "nu%d_nv%d_%dx%dx%d" % (d["nu"], d["nv"], d["nx"], d["ny"], d["nz"]))
@pytest.mark.parametrize("dtype", ["f32", "f16"])
def test_backproject_ragged(dims, dtype):
    rng = np.random.default_rng(3)
    g = dict(sid=600.0, sdd=900.0, np=17, angles=np.sort(rng.uniform(0, 2 * np.pi, 17)), du=1.0, dv=1.1,
             u_off=1.7, v_off=-2.3, sx=1.3, sy=1.2, sz=1.1, ox=0.7, oy=-1.4, oz=2.1, **dims)
    q = inputs.uniform_array(11, (g["np"], g["nv"], g["nu"]), -1, 1).astype(np.float32)
    if dtype == "f16":
        q = q.astype(np.float16)
    P = oracle.matrices(g)
    ref = oracle.backproject(P, q.astype(np.float64), g["nx"], g["ny"], g["nz"], 0.5)
    with api.bp_create(g) as ctx:
        vol = api.bp_backproject(ctx, torch.from_numpy(q).cuda(), scale=0.5).cpu().numpy()
        api.bp_device_status(ctx)
    print(f"ragged {dims} {dtype} uniform-noise rel err {rel(vol, ref):.2e}")
    # uniform noise is the hardest case for FP32 position rounding (steep data,
    # small max|vol| from cancellation); FP16 values are exact inputs here
    assert rel(vol, ref) <= TOL32


FP_GEOMS = {
    # the ragged tiles of the back-projection tests
    **{"ragged_%dx%dx%d" % (d["nx"], d["ny"], d["nz"]): dict(
        sid=600.0, sdd=900.0, du=1.0, dv=1.1, u_off=1.7, v_off=-2.3, sx=1.3, sy=1.2, sz=1.1, ox=0.7, oy=-1.4,
        oz=2.1, **d) for d in RAGGED},
    # a short source distance: the depth, and so the rows, of the columns of one
    # 8 x 4 patch differ enough that many taps fall beyond the lanes' windows
    "short_sid": dict(sid=120.0, sdd=260.0, du=1.0, dv=1.0, u_off=0.3, v_off=0.4, sx=0.8, sy=0.8, sz=0.8,
                      ox=0.0, oy=0.0, oz=0.0, nu=120, nv=110, nx=40, ny=36, nz=70),
    # less than one detector row per slice
    "dv_below_1": dict(sid=600.0, sdd=900.0, du=1.0, dv=1.2, u_off=0.0, v_off=0.0, sx=1.0, sy=1.0, sz=0.5,
                       ox=0.0, oy=0.0, oz=0.0, nu=80, nv=60, nx=33, ny=20, nz=70),
}


@pytest.mark.parametrize("name", sorted(FP_GEOMS))
def test_forward_project_ragged(name):
    rng = np.random.default_rng(4)
    g = dict(FP_GEOMS[name], np=7, angles=np.sort(rng.uniform(0, 2 * np.pi, 7)))
    P = oracle.matrices(g)
    x = inputs.uniform_array(23, (g["nz"], g["ny"], g["nx"]), 0, 1).astype(np.float32)
    q = inputs.uniform_array(24, (g["np"], g["nv"], g["nu"]), -1, 1).astype(np.float32)
    ref = oracle.forward_project(P, x, g["nu"], g["nv"], 0.5)
    with api.bp_create(g) as ctx:
        xd = torch.from_numpy(x).cuda()
        fx = api.fp_project(ctx, xd, scale=0.5)
        bq = api.bp_backproject(ctx, torch.from_numpy(q).cuda(), scale=0.5)
        api.bp_device_status(ctx)
        lhs = torch.dot(bq.double().flatten(), xd.double().flatten()).item()
        rhs = torch.dot(torch.from_numpy(q).cuda().double().flatten(), fx.double().flatten()).item()
        norm = bq.double().norm().item() * float(np.linalg.norm(x))
    print(f"fp {name} rel err {rel(fx.cpu().numpy(), ref):.2e}")
    assert rel(fx.cpu().numpy(), ref) <= TOL32
    assert abs(lhs - rhs) <= 1e-6 * norm


def test_flipped_detector_rows():
    """Matrices whose detector rows run against z (v -> nv - 1 - v): the row
    step per slice is negative; both operators follow the oracle."""
    g = dict(FP_GEOMS["ragged_37x29x45"], np=7, angles=np.sort(np.random.default_rng(5).uniform(0, 2 * np.pi, 7)))
    P = oracle.matrices(g)
    P[:, 1, :] = (g["nv"] - 1) * P[:, 2, :] - P[:, 1, :]
    x = inputs.uniform_array(25, (g["nz"], g["ny"], g["nx"]), 0, 1).astype(np.float32)
    q = inputs.uniform_array(26, (g["np"], g["nv"], g["nu"]), -1, 1).astype(np.float32)
    with api.bp_create_from_matrices(P, g["nu"], g["nv"], g["nx"], g["ny"], g["nz"]) as ctx:
        fx = api.fp_project(ctx, torch.from_numpy(x).cuda()).cpu().numpy()
        bq = api.bp_backproject(ctx, torch.from_numpy(q).cuda()).cpu().numpy()
        api.bp_device_status(ctx)
    print(f"flipped rows: fp rel err {rel(fx, oracle.forward_project(P, x, g['nu'], g['nv'])):.2e}, "
          f"bp {rel(bq, oracle.backproject(P, q, g['nx'], g['ny'], g['nz'])):.2e}")
    assert rel(fx, oracle.forward_project(P, x, g["nu"], g["nv"])) <= TOL32
    assert rel(bq, oracle.backproject(P, q, g["nx"], g["ny"], g["nz"])) <= TOL32


def test_backproject_batch_accumulate_and_view_chunks(c1):
    g = c1["g"]
    q = c1["q"]
    q2 = np.stack([q, np.flip(q, axis=2).copy()])
    scale = math.pi / g["np"]
    refs = [oracle.backproject(c1["P"], q2[b], g["nx"], g["ny"], g["nz"], scale) for b in range(2)]
    with api.bp_create(g) as ctx:
        d = torch.from_numpy(q2).cuda()
        vol = api.bp_backproject(ctx, d, scale=scale)
        for b in range(2):
            assert rel(vol[b].cpu().numpy(), refs[b]) <= TOL32
        # accumulate: vol + vol
        api.bp_backproject(ctx, d, vol=vol, scale=scale, accumulate=True)
        assert rel(vol[0].cpu().numpy(), 2 * refs[0]) <= TOL32
        # views in chunks of 25 accumulate to the full sum
        v2 = torch.zeros_like(vol)
        for s0 in range(0, g["np"], 25):
            n = min(25, g["np"] - s0)
            api.bp_backproject_views(ctx, d[:, s0:s0 + n], s0, v2, scale=scale, accumulate=True)
        assert rel(v2[1].cpu().numpy(), refs[1]) <= TOL32


def test_backproject_general_matrices():
    g = dict(sid=500.0, sdd=800.0, np=11, angles=np.linspace(0.1, 6.0, 11), nu=60, nv=50, du=1.0, dv=1.0,
             u_off=0.5, v_off=-0.5, nx=20, ny=18, nz=16, sx=1.5, sy=1.5, sz=1.5, ox=0, oy=0, oz=0)
    P = oracle.matrices(g)
    P[:, 0, 2] += 0.05      # detector tilt: u now depends on k
    P[:, 2, 2] += 1e-4      # and so does the depth
    q = inputs.uniform_array(5, (g["np"], g["nv"], g["nu"]), -1, 1).astype(np.float32)
    ref = oracle.backproject(P, q, g["nx"], g["ny"], g["nz"], 1.0)
    with api.bp_create_from_matrices(P, g["nu"], g["nv"], g["nx"], g["ny"], g["nz"]) as ctx:
        vol = api.bp_backproject(ctx, torch.from_numpy(q).cuda()).cpu().numpy()
        fp = api.fp_project(ctx, torch.from_numpy(ref.astype(np.float32)).cuda()).cpu().numpy()
    fref = oracle.forward_project(P, ref.astype(np.float32), g["nu"], g["nv"])
    print(f"general matrices uniform-noise: bp rel err {rel(vol, ref):.2e}, fp {rel(fp, fref):.2e}")
    assert rel(vol, ref) <= TOL32
    assert rel(fp, fref) <= TOL32


def test_forward_project_and_adjoint(c1):
    g = dict(c1["g"])
    g.update(np=30, angles=oracle.default_angles(30) + 0.2)
    P = oracle.matrices(g)
    x = inputs.uniform_array(21, (g["nz"], g["ny"], g["nx"]), 0, 1).astype(np.float32)
    q = inputs.uniform_array(22, (g["np"], g["nv"], g["nu"]), -1, 1).astype(np.float32)
    ref = oracle.forward_project(P, x, g["nu"], g["nv"], 0.7)
    with api.bp_create(g) as ctx:
        fx = api.fp_project(ctx, torch.from_numpy(x).cuda(), scale=0.7)
        bq = api.bp_backproject(ctx, torch.from_numpy(q).cuda(), scale=0.7)
        api.bp_device_status(ctx)
        lhs = torch.dot(bq.double().flatten(), torch.from_numpy(x).cuda().double().flatten()).item()
        rhs = torch.dot(torch.from_numpy(q).cuda().double().flatten(), fx.double().flatten()).item()
        norm = bq.double().norm().item() * float(np.linalg.norm(x))
    print(f"fp c1 rel err {rel(fx.cpu().numpy(), ref):.2e}")
    assert rel(fx.cpu().numpy(), ref) <= TOL32
    assert abs(lhs - rhs) <= 1e-6 * norm


def test_phantom_generator(c1):
    g = c1["g"]
    with api.bp_create(g) as ctx:
        out = api.bp_phantom_project(ctx, c1["E"]).cpu().numpy()
    assert rel(out, c1["raw"]) <= 1e-4


# ---------------------------------------------------------------------------
# Full-size workloads in the launch configuration the benchmark uses
# ---------------------------------------------------------------------------

def _band(P, g, k0, nks):
    """Detector rows every voxel of slices k0..k0+nks-1 can tap (plus margin)."""
    vs = []
    for i in (0, g["nx"] - 1):
        for j in (0, g["ny"] - 1):
            for k in (k0, k0 + nks - 1):
                h = P[:, :, :] @ np.array([i, j, k, 1.0])
                vs.append(h[:, 1] / h[:, 2])
    vs = np.concatenate(vs)
    r0 = max(0, int(np.floor(vs.min())) - 2)
    r1 = min(g["nv"], int(np.floor(vs.max())) + 4)
    return r0, r1 - r0


@pytest.mark.parametrize("name,k0,nks,sym", [("c2_fdk256", 112, 32, True), ("c3_paper", 224, 64, True),
                                             ("c3_paper", 224, 64, False)])
def test_full_size_slab(name, k0, nks, sym):
    """Oracle inputs on the detector band a z-slab sees; the GPU back-projects
    the whole volume in the benchmark's configuration (mid-plane symmetry on,
    the default for these centred geometries) and with the plain z-column
    kernel; the slab is compared voxel by voxel (FP32 and FP16-stored
    projections)."""
    p = inputs.preset(name)
    g = p["geom"]
    P = oracle.matrices(g)
    E = inputs.random_ellipsoids(p["seed"], p["n_ell"], p["axes"], g)
    r0, nr = _band(P, g, k0, nks)
    raw = oracle.phantom_project_rows(g, E, r0, nr)
    qb = oracle.ramp_filter_rows(g, raw, r0).astype(np.float32)
    q = np.zeros((g["np"], g["nv"], g["nu"]), dtype=np.float32)
    q[:, r0:r0 + nr, :] = qb
    scale = math.pi / g["np"]
    ref = oracle.backproject_slab(P, q, g["nx"], g["ny"], k0, nks, scale)
    with api.bp_create(g) as ctx:
        if not sym:
            api.bp_set_symmetry(ctx, False)
        assert api.bp_get_plan(ctx)["symmetric"] == sym
        d = torch.from_numpy(q).cuda()
        vol = api.bp_backproject(ctx, d, scale=scale)
        slab = vol[k0:k0 + nks].cpu().numpy()
        vol16 = api.bp_backproject(ctx, d.half(), scale=scale)
        slab16 = vol16[k0:k0 + nks].cpu().numpy()
        api.bp_device_status(ctx)
    e32, e16 = rel(slab, ref), rel(slab16, ref)
    print(f"{name} slab k={k0}..{k0 + nks - 1}: FP32 rel err {e32:.2e}, FP16-stored {e16:.2e}")
    assert e32 <= TOL32
    assert e16 <= TOL16


@pytest.mark.parametrize("label,views", [("P3", 512), ("P10", 64)])
def test_paper_problem_sampled(label, views):
    """The paper's problem grid at full volume size (P3: 1024^3 from a 256^2
    detector; P10: 1300^3, 8.8 GB, more than 2^31 voxels, ragged tiles in x, y
    and z): the whole back-projection runs on the GPU and 3000 voxels drawn
    over the volume (corners and the last slice included) match the oracle."""
    g = inputs.paper_problem(label, views=views)
    q = inputs.uniform_array(77, (g["np"], g["nv"], g["nu"]), -1.0, 1.0).astype(np.float32)
    rng = np.random.default_rng(3)
    n = g["nx"]
    ijk = rng.integers(0, n, size=(3000, 3))
    ijk[:8] = [[a, b, c] for a in (0, n - 1) for b in (0, n - 1) for c in (0, n - 1)]
    scale = math.pi / g["np"]
    with api.bp_create(g) as ctx:
        vol = api.bp_backproject(ctx, torch.from_numpy(q).cuda(), scale=scale)
        api.bp_device_status(ctx)
        got = vol[ijk[:, 2], ijk[:, 1], ijk[:, 0]].cpu().numpy()
        del vol
    ref = oracle.backproject_points(oracle.matrices(g), q, ijk, scale)
    assert rel(got, ref) <= TOL32


# ---------------------------------------------------------------------------
# The spec bar (1e-5 of max|vol|, FP32) on phantom data for every FP32
# kernel path: off-centre detector and volume (plain z-column kernel, staged
# and direct-load), general matrices (per-voxel kernel), the forward projector
# on ragged and off-centre geometries, and FDK end to end.
# ---------------------------------------------------------------------------

OFFC = {
    # staged (TMA) path for FP32 and FP16
    "tma_128": dict(nu=128, nv=128, nx=61, ny=53, nz=45),
    # nu*4 not a multiple of 16: direct global loads for both types
    "direct_126": dict(nu=126, nv=120, nx=59, ny=47, nz=50),
}


@pytest.fixture(scope="module")
def offc():
    out = {}
    p = inputs.preset("c1_small")
    E = inputs.random_ellipsoids(p["seed"], p["n_ell"], p["axes"], p["geom"])
    for name, dims in OFFC.items():
        g = dict(p["geom"], u_off=1.7, v_off=-2.3, ox=0.7, oy=-1.4, oz=2.1, **dims)
        q = oracle.ramp_filter(g, oracle.phantom_project(g, E)).astype(np.float32)
        P = oracle.matrices(g)
        scale = math.pi / g["np"]
        ref = oracle.backproject(P, q, g["nx"], g["ny"], g["nz"], scale)
        out[name] = dict(g=g, q=q, P=P, scale=scale, ref=ref)
    return out


@pytest.mark.parametrize("name", sorted(OFFC))
def test_offcentre_phantom_fp32_fp16(offc, name):
    c = offc[name]
    g = c["g"]
    q16 = c["q"].astype(np.float16)
    ref16 = oracle.backproject(c["P"], q16.astype(np.float64), g["nx"], g["ny"], g["nz"], c["scale"])
    with api.bp_create(g) as ctx:
        plan = api.bp_get_plan(ctx)
        assert not plan["symmetric"]
        vol = api.bp_backproject(ctx, torch.from_numpy(c["q"]).cuda(), scale=c["scale"]).cpu().numpy()
        vol16 = api.bp_backproject(ctx, torch.from_numpy(q16).cuda(), scale=c["scale"]).cpu().numpy()
        api.bp_device_status(ctx)
    e32, e16, e16q = rel(vol, c["ref"]), rel(vol16, c["ref"]), rel(vol16, ref16)
    print(f"off-centre {name}: FP32 {e32:.2e}, FP16-stored {e16:.2e} (vs quantised {e16q:.2e})")
    assert e32 <= TOL32
    assert e16 <= TOL16
    assert e16q <= TOL32


@pytest.mark.parametrize("name", sorted(OFFC))
def test_offcentre_forward_project_phantom(offc, name):
    """The forward projector of the FDK volume (smooth, non-negative data)."""
    c = offc[name]
    g = c["g"]
    x = np.ascontiguousarray(c["ref"].astype(np.float32))
    ref = oracle.forward_project(c["P"], x, g["nu"], g["nv"], 0.5)
    with api.bp_create(g) as ctx:
        fx = api.fp_project(ctx, torch.from_numpy(x).cuda(), scale=0.5).cpu().numpy()
        api.bp_device_status(ctx)
    e = rel(fx, ref)
    print(f"off-centre {name}: forward projection {e:.2e}")
    assert e <= TOL32


def test_general_matrices_phantom(c1):
    """Tilted detector (u and depth depend on k): the per-voxel kernel and the
    forward projector on filtered phantom data and its back-projection."""
    g = c1["g"]
    P = c1["P"].copy()
    P[:, 0, 2] += 0.05
    P[:, 2, 2] += 1e-4
    scale = math.pi / g["np"]
    ref = oracle.backproject(P, c1["q"], g["nx"], g["ny"], g["nz"], scale)
    x = np.ascontiguousarray(ref.astype(np.float32))
    fref = oracle.forward_project(P, x, g["nu"], g["nv"], scale)
    with api.bp_create_from_matrices(P, g["nu"], g["nv"], g["nx"], g["ny"], g["nz"]) as ctx:
        vol = api.bp_backproject(ctx, torch.from_numpy(c1["q"]).cuda(), scale=scale).cpu().numpy()
        fp = api.fp_project(ctx, torch.from_numpy(x).cuda(), scale=scale).cpu().numpy()
        api.bp_device_status(ctx)
    print(f"general matrices phantom: bp {rel(vol, ref):.2e}, fp {rel(fp, fref):.2e}")
    assert rel(vol, ref) <= TOL32
    assert rel(fp, fref) <= TOL32


@pytest.mark.parametrize("name", ["short_sid", "dv_below_1", "ragged_37x29x45"])
def test_forward_project_ragged_phantom(c1, name):
    """The ragged forward-projector geometries on a smooth volume: the c1 FDK
    volume resampled (nearest) to the geometry's grid."""
    rng = np.random.default_rng(4)
    g = dict(FP_GEOMS[name], np=7, angles=np.sort(rng.uniform(0, 2 * np.pi, 7)))
    P = oracle.matrices(g)
    src = oracle.fdk(c1["g"], c1["raw"])
    zi = np.arange(g["nz"]) * (src.shape[0] - 1) // max(g["nz"] - 1, 1)
    yi = np.arange(g["ny"]) * (src.shape[1] - 1) // max(g["ny"] - 1, 1)
    xi = np.arange(g["nx"]) * (src.shape[2] - 1) // max(g["nx"] - 1, 1)
    x = np.ascontiguousarray(src[np.ix_(zi, yi, xi)].astype(np.float32))
    ref = oracle.forward_project(P, x, g["nu"], g["nv"], 0.5)
    with api.bp_create(g) as ctx:
        fx = api.fp_project(ctx, torch.from_numpy(x).cuda(), scale=0.5).cpu().numpy()
        api.bp_device_status(ctx)
    e = rel(fx, ref)
    print(f"fp {name} phantom rel err {e:.2e}")
    assert e <= TOL32


# detector pixels per voxel (magnification x voxel / pitch): the u width of a
# warp's 8 x 4 column patch grows with it, so these geometries run the
# forward projector with each window width it is built for (17 .. 49 columns)
WINDOW_RATIOS = [1.2, 1.8, 2.2, 3.0, 4.0]


@pytest.mark.parametrize("ratio", WINDOW_RATIOS)
def test_forward_project_window_widths(ratio):
    rng = np.random.default_rng(int(ratio * 10))
    sid, sdd, sx = 600.0, 900.0, 1.0
    du = sdd / sid * sx / ratio
    n_det = int(np.ceil(36 * sx * sdd / sid / du)) + 8
    g = dict(sid=sid, sdd=sdd, np=9, angles=np.sort(rng.uniform(0, 2 * np.pi, 9)), nu=n_det, nv=n_det,
             du=du, dv=du, u_off=0.3, v_off=-0.2, nx=33, ny=30, nz=34, sx=sx, sy=sx, sz=sx, ox=0.0, oy=0.0, oz=0.0)
    P = oracle.matrices(g)
    # a smooth volume: the global reductions add in a varying order, and on
    # uniform noise the largest error (about 1e-5 px of position rounding at
    # 150-px boxes) would sit at the bar
    zz, yy, xx = np.meshgrid(np.linspace(-1, 1, g["nz"]), np.linspace(-1, 1, g["ny"]), np.linspace(-1, 1, g["nx"]),
                             indexing="ij")
    x = (0.2 + np.exp(-((xx - 0.1) ** 2 + (yy + 0.2) ** 2 + zz ** 2) / 0.3)).astype(np.float32)
    q = inputs.uniform_array(32, (g["np"], g["nv"], g["nu"]), -1, 1).astype(np.float32)
    ref = oracle.forward_project(P, x, g["nu"], g["nv"], 0.5)
    with api.bp_create(g) as ctx:
        xd = torch.from_numpy(x).cuda()
        fx = api.fp_project(ctx, xd, scale=0.5)
        bq = api.bp_backproject(ctx, torch.from_numpy(q).cuda(), scale=0.5)
        api.bp_device_status(ctx)
        lhs = torch.dot(bq.double().flatten(), xd.double().flatten()).item()
        rhs = torch.dot(torch.from_numpy(q).cuda().double().flatten(), fx.double().flatten()).item()
        norm = bq.double().norm().item() * float(np.linalg.norm(x))
    e = rel(fx.cpu().numpy(), ref)
    print(f"fp {ratio} px/voxel ({g['nu']}^2 detector) rel err {e:.2e}")
    assert e <= TOL32
    assert abs(lhs - rhs) <= 1e-6 * norm


@pytest.mark.parametrize("name,views", [("c2_fdk256", [0, 45, 117, 300]), ("c3_paper", [31, 400])])
def test_full_size_forward_project(name, views):
    """The forward projector at full volume and detector size, in the launch
    configuration the benchmark times (the same tiles and window width; only
    the number of views is cut), on a smooth phantom-like volume (a sum of
    Gaussian blobs) against the oracle's scatter of every voxel."""
    p = inputs.preset(name)
    g = dict(p["geom"])
    ang = oracle.default_angles(g["np"])[views]
    g.update(np=len(views), angles=ang)
    nz, ny, nx = g["nz"], g["ny"], g["nx"]
    z, y, x = np.meshgrid(np.linspace(-1, 1, nz), np.linspace(-1, 1, ny), np.linspace(-1, 1, nx), indexing="ij")
    vol = (np.exp(-((x - 0.2) ** 2 + y ** 2 + (z + 0.1) ** 2) / 0.2)
           + 0.5 * np.exp(-((x + 0.3) ** 2 + (y - 0.25) ** 2 + z ** 2) / 0.05)).astype(np.float32)
    P = oracle.matrices(g)
    ref = oracle.forward_project(P, vol, g["nu"], g["nv"], 1.0)
    with api.bp_create(g) as ctx:
        fx = api.fp_project(ctx, torch.from_numpy(vol).cuda()).cpu().numpy()
        api.bp_device_status(ctx)
    e = rel(fx, ref)
    print(f"full-size forward projection {name} views {views}: rel err {e:.2e}")
    assert e <= TOL32
