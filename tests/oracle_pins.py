"""Pins that tie the FP64 oracle to facts other than its own code.

Each pin is a plain function that raises AssertionError on failure. They are
run against the real oracle (tests/test_oracle.py) and against copies of
oracle.c with planted mistakes (tests/test_oracle_mutants.py), which must
each fail at least one pin.

What pins what:
  matrix_vs_ray           3x4 matrices (Section 2.1.1) vs a line-plane intersection
  z_invariance            P[0][2] = P[2][2] = 0 (u and w independent of k, Section 3.1.2)
  bp_constant             back-projection of constant data = scale*c*sum_s 1/w_s^2
  bp_linear               bilinear sampling reproduces linear data exactly
  bp_fp_hat_matrix        BP and FP vs a dense matrix built from hat functions
                          (bilinear weight = tent(u-c)*tent(v-r)), zero padding included
  bp_slab_points          slab and point back-projections vs that hat matrix and the whole loop
  adjoint_dot             <BP q, x> = <q, FP x>
  symmetry                v(nz-1-k) = nv-1-v(k) for a centred geometry (Section 3.1.2)
  filter_impulse          cosine weight from the 3-D ray angle, centre tap 1/(4 dp)
  filter_frequency        Ram-Lak frequency response |f|/dp on a cosine
  phantom_sphere          chord of a sphere = 2 sqrt(R^2 - rho^2)
  phantom_ray_integral    ellipsoid line integrals vs numerical ray marching
  phantom_siddon          analytic projections vs Siddon through the voxelised phantom
  fdk_sphere              FDK of a unit-density sphere in the central slices
  fdk_offcentre           FDK of an off-centre sphere lands at its true centre
  fdk_ellipsoids          FDK of the 10-ellipsoid phantom in the central slices
  conv_vs_scipy           3x3x3 convolution vs scipy.ndimage.correlate per channel pair
  conv_adjoints           <conv(x), dy> = <x, dgrad(dy)> and the weight gradient as the
                          derivative of that pairing in w (linearity check)
  mlem_counts             EM count preservation: sum (A^T 1) x+ = sum of p over rays with Ax > 0
  mlem_likelihood         EM never decreases the Poisson log-likelihood
  iter_fixed_points       the true volume is a fixed point of MLEM and SART on consistent data
  sart_constant_step      one SART or MLEM step maps a constant start to a constant volume's value
  iter_convergence        MLEM, OS-EM, SIRT and SART reach the true volume of a full-rank system
"""
import numpy as np

import oracle
from paper_2104_13248_gb300 import inputs
from tests import geometry_ref as gr


def _geom_offsets():
    rng = np.random.default_rng(7)
    ang = np.sort(rng.uniform(0, 2 * np.pi, 9))
    return dict(sid=500.0, sdd=800.0, np=9, angles=ang, nu=40, nv=36, du=1.1, dv=0.9,
                u_off=1.3, v_off=-0.7, nx=12, ny=10, nz=8, sx=1.2, sy=1.0, sz=1.5,
                ox=0.8, oy=-1.1, oz=0.6)


def _uvw(g, P, s, i, j, k):
    h = P[s] @ np.array([i, j, k, 1.0])
    return h[0] / h[2], h[1] / h[2], h[2]


def matrix_vs_ray():
    g = _geom_offsets()
    P = oracle.matrices(g)
    rng = np.random.default_rng(1)
    for s in range(g["np"]):
        for _ in range(20):
            i, j, k = rng.uniform(-2, 14), rng.uniform(-2, 12), rng.uniform(-2, 10)
            u, v, w = _uvw(g, P, s, i, j, k)
            X = gr.voxel_world(g, i, j, k)
            u2, v2, w2 = gr.project_point(g, g["angles"][s], X)
            assert abs(u - u2) < 1e-9 and abs(v - v2) < 1e-9 and abs(w - w2) < 1e-12, \
                (s, u, u2, v, v2, w, w2)


def z_invariance():
    g = _geom_offsets()
    P = oracle.matrices(g)
    assert np.all(P[:, 0, 2] == 0.0) and np.all(P[:, 2, 2] == 0.0)
    assert np.all(np.abs(P[:, 1, 2]) > 0.0)


def _interior_mask(g, P):
    """Voxels whose four taps lie inside the detector in every view."""
    nx, ny, nz = g["nx"], g["ny"], g["nz"]
    K, J, I = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    ok = np.ones(K.shape, dtype=bool)
    for s in range(P.shape[0]):
        w = P[s, 2, 0] * I + P[s, 2, 1] * J + P[s, 2, 2] * K + P[s, 2, 3]
        u = (P[s, 0, 0] * I + P[s, 0, 1] * J + P[s, 0, 2] * K + P[s, 0, 3]) / w
        v = (P[s, 1, 0] * I + P[s, 1, 1] * J + P[s, 1, 2] * K + P[s, 1, 3]) / w
        ok &= (u >= 0) & (u <= g["nu"] - 1.001) & (v >= 0) & (v <= g["nv"] - 1.001)
    return ok


def _big_detector_geom():
    g = _geom_offsets()
    g.update(nu=64, nv=60, du=1.0, dv=1.0)
    return g


def bp_constant():
    g = _big_detector_geom()
    P = oracle.matrices(g)
    c, scale = 1.7, 0.37
    q = np.full((g["np"], g["nv"], g["nu"]), c)
    vol = oracle.backproject(P, q, g["nx"], g["ny"], g["nz"], scale)
    mask = _interior_mask(g, P)
    assert mask.sum() > 0.8 * mask.size
    for k, j, i in zip(*np.nonzero(mask)):
        X = gr.voxel_world(g, i, j, k)
        ref = 0.0
        for s in range(g["np"]):
            er, _, _ = gr.frame(g["angles"][s])
            w = 1.0 - np.dot(X, er) / g["sid"]
            ref += 1.0 / (w * w)
        ref *= scale * c
        assert abs(vol[k, j, i] - ref) <= 1e-12 * abs(ref), (k, j, i, vol[k, j, i], ref)


def bp_linear():
    g = _big_detector_geom()
    P = oracle.matrices(g)
    rng = np.random.default_rng(3)
    al, be, ga = rng.normal(size=g["np"]), rng.normal(size=g["np"]), rng.normal(size=g["np"])
    r = np.arange(g["nv"])[:, None]
    c = np.arange(g["nu"])[None, :]
    q = np.stack([al[s] * c + be[s] * r + ga[s] for s in range(g["np"])])
    vol = oracle.backproject(P, q, g["nx"], g["ny"], g["nz"], 1.0)
    mask = _interior_mask(g, P)
    for k, j, i in list(zip(*np.nonzero(mask)))[::7]:
        X = gr.voxel_world(g, i, j, k)
        ref = 0.0
        for s in range(g["np"]):
            u, v, w = gr.project_point(g, g["angles"][s], X)
            ref += (al[s] * u + be[s] * v + ga[s]) / (w * w)
        assert abs(vol[k, j, i] - ref) <= 1e-10 * max(1.0, abs(ref)), (k, j, i, vol[k, j, i], ref)


def _tent(t):
    return np.maximum(0.0, 1.0 - np.abs(t))


def _hat_matrix(g, scale):
    """Dense A[(s,r,c),(k,j,i)] = scale * tent(u-c) * tent(v-r) / w^2 with
    (u, v, w) from the ray intersection; only detector pixels exist as rows,
    so taps outside the detector drop out (zero padding)."""
    nvox = g["nx"] * g["ny"] * g["nz"]
    A = np.zeros((g["np"] * g["nv"] * g["nu"], nvox))
    r = np.arange(g["nv"])[:, None]
    c = np.arange(g["nu"])[None, :]
    col = 0
    for k in range(g["nz"]):
        for j in range(g["ny"]):
            for i in range(g["nx"]):
                X = gr.voxel_world(g, i, j, k)
                for s in range(g["np"]):
                    u, v, w = gr.project_point(g, g["angles"][s], X)
                    wt = scale * _tent(u - c) * _tent(v - r) / (w * w)
                    A[s * g["nv"] * g["nu"]:(s + 1) * g["nv"] * g["nu"], col] = wt.reshape(-1)
                col += 1
    return A


def bp_fp_hat_matrix():
    # The volume overhangs the detector so that zero padding is exercised,
    # and some projections land at negative coordinates (floor vs truncation).
    rng = np.random.default_rng(11)
    g = _hat_geom()
    scale = 0.8
    A = _hat_matrix(g, scale)
    P = oracle.matrices(g)
    q = rng.normal(size=(g["np"], g["nv"], g["nu"]))
    x = rng.normal(size=(g["nz"], g["ny"], g["nx"]))
    bp = oracle.backproject(P, q, g["nx"], g["ny"], g["nz"], scale)
    fp = oracle.forward_project(P, x, g["nu"], g["nv"], scale)
    ref_bp = (A.T @ q.reshape(-1)).reshape(bp.shape)
    ref_fp = (A @ x.reshape(-1)).reshape(fp.shape)
    assert np.abs(ref_bp).max() > 0 and np.abs(ref_fp).max() > 0
    assert np.max(np.abs(bp - ref_bp)) <= 1e-12 * np.abs(ref_bp).max()
    assert np.max(np.abs(fp - ref_fp)) <= 1e-12 * np.abs(ref_fp).max()
    # some voxels fall (partly) off the detector: padding must have mattered
    assert (np.abs(A).sum(axis=0) == 0).any() or (A > 0).sum() < 4 * g["np"] * A.shape[1]


def _hat_geom():
    return dict(sid=300.0, sdd=450.0, np=4, angles=np.array([0.1, 1.3, 2.9, 4.4]), nu=16, nv=14,
                du=1.3, dv=1.1, u_off=2.2, v_off=-1.6, nx=8, ny=7, nz=6, sx=2.0, sy=2.1, sz=2.4,
                ox=1.0, oy=0.5, oz=-0.7)


def bp_slab_points():
    """The slab and point versions of Listing 1 (the references for sampled and
    slab parity) against the dense hat matrix, slice range by slice range and
    voxel by voxel, and against the whole-volume loop on a second geometry."""
    g = _hat_geom()
    scale = 0.8
    A = _hat_matrix(g, scale)
    P = oracle.matrices(g)
    rng = np.random.default_rng(12)
    q = rng.normal(size=(g["np"], g["nv"], g["nu"]))
    ref = (A.T @ q.reshape(-1)).reshape(g["nz"], g["ny"], g["nx"])
    tol = 1e-12 * np.abs(ref).max()
    nz = g["nz"]
    for k0, nks in [(0, nz), (0, 1), (nz - 1, 1), (2, 3), (1, nz - 2)]:
        slab = oracle.backproject_slab(P, q, g["nx"], g["ny"], k0, nks, scale)
        assert slab.shape == (nks, g["ny"], g["nx"])
        assert np.max(np.abs(slab - ref[k0:k0 + nks])) <= tol, (k0, nks)
    ijk = np.stack([rng.integers(0, g["nx"], 60), rng.integers(0, g["ny"], 60),
                    rng.integers(0, nz, 60)], axis=1)
    ijk[:4] = [[0, 0, 0], [g["nx"] - 1, g["ny"] - 1, nz - 1], [0, g["ny"] - 1, 0], [g["nx"] - 1, 0, nz - 1]]
    pts = oracle.backproject_points(P, q, ijk, scale)
    assert np.max(np.abs(pts - ref[ijk[:, 2], ijk[:, 1], ijk[:, 0]])) <= tol
    # second geometry, larger, against the whole-volume loop
    g = _geom_offsets()
    P = oracle.matrices(g)
    q = rng.normal(size=(g["np"], g["nv"], g["nu"]))
    full = oracle.backproject(P, q, g["nx"], g["ny"], g["nz"], 0.45)
    tol = 1e-14 * np.abs(full).max()
    for k0, nks in [(0, g["nz"]), (g["nz"] - 1, 1), (3, 2)]:
        slab = oracle.backproject_slab(P, q, g["nx"], g["ny"], k0, nks, 0.45)
        assert np.max(np.abs(slab - full[k0:k0 + nks])) <= tol, (k0, nks)
    ijk = np.stack(np.meshgrid(np.arange(g["nx"]), np.arange(g["ny"]), np.arange(g["nz"]),
                               indexing="ij"), axis=-1).reshape(-1, 3)
    pts = oracle.backproject_points(P, q, ijk, 0.45)
    assert np.max(np.abs(pts - full[ijk[:, 2], ijk[:, 1], ijk[:, 0]])) <= tol


def adjoint_dot():
    g = _geom_offsets()
    g.update(nx=16, ny=15, nz=14, np=7, angles=np.linspace(0, 6, 7))
    P = oracle.matrices(g)
    rng = np.random.default_rng(5)
    q = rng.normal(size=(g["np"], g["nv"], g["nu"]))
    x = rng.normal(size=(g["nz"], g["ny"], g["nx"]))
    bq = oracle.backproject(P, q, g["nx"], g["ny"], g["nz"], 0.6)
    fx = oracle.forward_project(P, x, g["nu"], g["nv"], 0.6)
    lhs, rhs = np.vdot(bq, x), np.vdot(q, fx)
    assert abs(lhs - rhs) <= 1e-12 * np.linalg.norm(bq) * np.linalg.norm(x), (lhs, rhs)


def symmetry():
    g = dict(sid=800.0, sdd=1200.0, np=10, angles=None, nu=50, nv=44, du=0.9, dv=0.7,
             u_off=0.0, v_off=0.0, nx=11, ny=9, nz=12, sx=1.3, sy=1.1, sz=1.7,
             ox=0.0, oy=0.0, oz=0.0)
    P = oracle.matrices(g)
    for s in range(g["np"]):
        for i in range(g["nx"]):
            for j in range(g["ny"]):
                for k in range(g["nz"]):
                    u1, v1, _ = _uvw(g, P, s, i, j, k)
                    u2, v2, _ = _uvw(g, P, s, i, j, g["nz"] - 1 - k)
                    assert abs(v1 + v2 - (g["nv"] - 1)) < 1e-10 and abs(u1 - u2) < 1e-10


def filter_impulse():
    g = dict(sid=700.0, sdd=1100.0, np=1, nu=33, nv=9, du=0.7, dv=0.6, u_off=1.5, v_off=-0.5)
    r0, c0 = 7, 29
    q = np.zeros((1, g["nv"], g["nu"]))
    q[0, r0, c0] = 1.0
    out = oracle.ramp_filter(g, q)
    er, _, _ = gr.frame(0.0)
    _, d = gr.pixel_ray(g, 0.0, r0, c0)
    cosw = np.dot(d, -er)                 # cosine between pixel ray and central ray
    dp = g["du"] * g["sid"] / g["sdd"]     # detector pitch scaled to the isocenter
    assert abs(out[0, r0, c0] - cosw / (4.0 * dp)) < 1e-12 * (1 / dp)
    # even offsets vanish, odd offsets are negative; other rows untouched
    for n in range(-c0, g["nu"] - c0):
        if n != 0:
            v = out[0, r0, c0 + n]
            assert (v == 0.0) if n % 2 == 0 else (v < 0.0)
    assert np.all(out[0, np.arange(g["nv"]) != r0] == 0.0)


def filter_frequency():
    nu = 2048
    g = dict(sid=1000.0, sdd=1600.0, np=1, nu=nu, nv=1, du=0.5, dv=0.5, u_off=0.0, v_off=0.0)
    dp = g["du"] * g["sid"] / g["sdd"]
    er, _, _ = gr.frame(0.0)
    cosw = np.array([np.dot(gr.pixel_ray(g, 0.0, 0, c)[1], -er) for c in range(nu)])
    m = np.arange(nu)
    for f in (0.05, 0.125, 0.3):
        sig = np.cos(2 * np.pi * f * m + 0.3)
        out = oracle.ramp_filter(g, (sig / cosw)[None, None, :])[0, 0]
        mid = slice(nu // 4, 3 * nu // 4)
        ref = (f / dp) * sig
        err = np.max(np.abs(out[mid] - ref[mid])) / (f / dp)
        assert err < 0.01, (f, err)


def phantom_sphere():
    g = dict(sid=600.0, sdd=900.0, np=3, angles=np.array([0.2, 2.0, 4.1]), nu=40, nv=30,
             du=1.2, dv=1.0, u_off=0.7, v_off=-1.2)
    for C, R in (((0.0, 0.0, 0.0), 15.0), ((4.0, -6.0, 3.0), 9.0)):
        E = inputs.sphere(R, 2.0, C)
        proj = oracle.phantom_project(g, E)
        hit = 0
        for s in range(g["np"]):
            for r in range(g["nv"]):
                for c in range(g["nu"]):
                    S, d = gr.pixel_ray(g, g["angles"][s], r, c)
                    rho = np.linalg.norm(np.cross(S - np.array(C), d))
                    ref = 2.0 * 2.0 * np.sqrt(max(0.0, R * R - rho * rho))
                    hit += ref > 0
                    assert abs(proj[s, r, c] - ref) < 1e-9 * max(1.0, ref), (s, r, c, proj[s, r, c], ref)
        assert hit > 50


def phantom_ray_integral():
    g = dict(sid=500.0, sdd=750.0, np=2, angles=np.array([0.4, 3.5]), nu=12, nv=10,
             du=2.0, dv=2.0, u_off=0.0, v_off=0.0)
    E = np.zeros((2, 16))
    rng = inputs.SplitMix64(9)
    for e, (C, a, rho) in enumerate((((1.0, -2.0, 1.5), (9.0, 5.0, 3.5), 1.0),
                                     ((-3.0, 2.0, -1.0), (4.0, 7.0, 6.0), 0.5))):
        q = np.array([rng.gauss() for _ in range(4)])
        q /= np.linalg.norm(q)
        E[e, 0:3], E[e, 3:6], E[e, 15] = C, a, rho
        E[e, 6:15] = inputs._quat_to_rot(q).reshape(-1)
    proj = oracle.phantom_project(g, E)
    t = np.linspace(g["sid"] - 30, g["sid"] + 30, 60001)
    dt = t[1] - t[0]
    n_hit = 0
    for s in range(g["np"]):
        for r in range(g["nv"]):
            for c in range(g["nu"]):
                S, d = gr.pixel_ray(g, g["angles"][s], r, c)
                pts = S[None, :] + t[:, None] * d[None, :]
                dens = inputs.density_at(E, pts[:, 0], pts[:, 1], pts[:, 2])
                ref = dens.sum() * dt
                n_hit += ref > 1.0
                assert abs(proj[s, r, c] - ref) < 0.02 + 2e-3 * ref, (s, r, c, proj[s, r, c], ref)
    assert n_hit > 20


def phantom_siddon():
    g = dict(sid=400.0, sdd=640.0, np=3, angles=np.array([0.3, 1.9, 4.0]), nu=48, nv=40,
             du=1.0, dv=1.0, u_off=0.0, v_off=0.0, nx=48, ny=44, nz=40, sx=0.6, sy=0.6,
             sz=0.6, ox=0.5, oy=-0.4, oz=0.3)
    E = np.zeros((1, 16))
    E[0, 0:3] = (2.0, -1.0, 1.0)
    E[0, 3:6] = (9.0, 6.0, 7.0)
    c, s_ = np.cos(0.5), np.sin(0.5)
    E[0, 6:15] = np.array([[c, -s_, 0], [s_, c, 0], [0, 0, 1]]).reshape(-1)
    E[0, 15] = 1.0
    # voxel value = mean of 4^3 sub-samples of the density (partial-volume voxelisation)
    x, y, z = oracle.voxel_centres(g)
    sub = (np.arange(4) - 1.5) / 4.0
    vol = np.zeros((g["nz"], g["ny"], g["nx"]))
    for a in sub:
        for b in sub:
            for cc in sub:
                Z, Y, X = np.meshgrid(z + cc * g["sz"], y + b * g["sy"], x + a * g["sx"], indexing="ij")
                vol += inputs.density_at(E, X, Y, Z)
    vol /= 64.0
    ana = oracle.phantom_project(g, E)
    sid_ = oracle.siddon(g, vol)
    # chords through the bulk agree up to the staircase error of 0.6 mm voxels
    m = ana > 8.0
    assert m.sum() > 300
    rel = np.abs(sid_[m] - ana[m]) / ana[m]
    assert rel.mean() < 0.03 and rel.max() < 0.15, (rel.mean(), rel.max())
    # projection centroids agree to a tenth of a pixel (a half-pixel offset or
    # a flipped axis between the ray geometry and the voxel grid would not)
    cu = np.arange(g["nu"])[None, :]
    rv = np.arange(g["nv"])[:, None]
    for s in range(g["np"]):
        a, b = ana[s], sid_[s]
        du_c = (a * cu).sum() / a.sum() - (b * cu).sum() / b.sum()
        dv_c = (a * rv).sum() / a.sum() - (b * rv).sum() / b.sum()
        assert abs(du_c) < 0.1 and abs(dv_c) < 0.1, (s, du_c, dv_c)


def _c1():
    return inputs.preset("c1_small")


def _grid(g):
    x, y, z = oracle.voxel_centres(g)
    return np.meshgrid(z, y, x, indexing="ij")


def fdk_sphere():
    g = _c1()["geom"]
    E = inputs.sphere(20.0)
    vol = oracle.fdk(g, oracle.phantom_project(g, E))
    Z, Y, X = _grid(g)
    truth = inputs.density_at(E, X, Y, Z)
    far = inputs.surface_distance_mask(E, X, Y, Z, 3.0)
    R = np.sqrt(X ** 2 + Y ** 2)
    for k in (g["nz"] // 2 - 1, g["nz"] // 2):
        inside = far[k] & (truth[k] > 0)
        assert inside.sum() > 500
        assert np.max(np.abs(vol[k][inside] - 1.0)) < 0.01
        ring = far[k] & (R[k] <= 28.0)
        assert np.max(np.abs(vol[k][ring] - truth[k][ring])) < 0.06


def fdk_offcentre():
    g = _c1()["geom"]
    C = (8.0, -6.0, 5.0)
    E = inputs.sphere(9.0, 1.0, C)
    vol = oracle.fdk(g, oracle.phantom_project(g, E))
    Z, Y, X = _grid(g)
    m = vol > 0.5
    wsum = vol[m].sum()
    cen = [(X[m] * vol[m]).sum() / wsum, (Y[m] * vol[m]).sum() / wsum, (Z[m] * vol[m]).sum() / wsum]
    assert np.max(np.abs(np.array(cen) - np.array(C))) < 0.25, cen
    inner = inputs.surface_distance_mask(E, X, Y, Z, 3.0) & (inputs.density_at(E, X, Y, Z) > 0)
    assert np.max(np.abs(vol[inner] - 1.0)) < 0.05


def fdk_ellipsoids():
    p = _c1()
    g = p["geom"]
    E = inputs.random_ellipsoids(p["seed"], p["n_ell"], p["axes"], g)
    vol = oracle.fdk(g, oracle.phantom_project(g, E))
    Z, Y, X = _grid(g)
    truth = inputs.density_at(E, X, Y, Z)
    far = inputs.surface_distance_mask(E, X, Y, Z, 3.0)
    R = np.sqrt(X ** 2 + Y ** 2)
    for k in (g["nz"] // 2 - 1, g["nz"] // 2):
        m = far[k] & (R[k] <= 28.0)
        assert m.sum() > 300
        err = np.abs(vol[k][m] - truth[k][m])
        assert err.mean() < 0.06 and err.max() < 0.30, (err.mean(), err.max())


def conv_vs_scipy():
    ndimage = __import__("scipy.ndimage", fromlist=["correlate"])
    rng = np.random.default_rng(12)
    N, D, H, W, cin, cout = 2, 5, 6, 7, 3, 4
    x = rng.normal(size=(N, D, H, W, cin))
    w = rng.normal(size=(cout, 27, cin))
    b = rng.normal(size=cout)
    y = oracle.conv3d(x, w, b)
    for n in range(N):
        for co in range(cout):
            ref = np.full((D, H, W), b[co])
            for ci in range(cin):
                ref += ndimage.correlate(x[n, ..., ci], w[co, :, ci].reshape(3, 3, 3), mode="constant", cval=0.0)
            assert np.max(np.abs(y[n, ..., co] - ref)) < 1e-10


def conv_adjoints():
    rng = np.random.default_rng(13)
    N, D, H, W, cin, cout = 1, 6, 5, 7, 5, 3
    x = rng.normal(size=(N, D, H, W, cin))
    w = rng.normal(size=(cout, 27, cin))
    dy = rng.normal(size=(N, D, H, W, cout))
    y = oracle.conv3d(x, w)
    dx = oracle.conv3d_dgrad(dy, w)
    assert abs(np.vdot(y, dy) - np.vdot(x, dx)) < 1e-9 * np.linalg.norm(y) * np.linalg.norm(dy)
    dw, db = oracle.conv3d_wgrad(x, dy)
    # <conv_w(x), dy> is linear in w with gradient dw: check on random directions
    for seed in range(3):
        w2 = np.random.default_rng(100 + seed).normal(size=w.shape)
        assert abs(np.vdot(oracle.conv3d(x, w2), dy) - np.vdot(w2, dw)) < 1e-9 * np.abs(dw).sum() * 10
    b2 = rng.normal(size=cout)
    lhs = np.vdot(oracle.conv3d(x, 0 * w, b2), dy)
    assert abs(lhs - np.vdot(b2, db)) < 1e-9 * max(1.0, abs(lhs))


def _iter_system():
    """A small system with full column rank (60 voxels, 8 views of 12 x 10
    pixels, the whole volume in view): consistent data from a positive volume."""
    g = dict(sid=300.0, sdd=450.0, np=8, angles=np.linspace(0.1, 2 * np.pi, 8, endpoint=False), nu=12,
             nv=10, du=1.5, dv=1.5, u_off=0.3, v_off=-0.2, nx=5, ny=4, nz=3, sx=2.0, sy=2.0, sz=2.0,
             ox=0.2, oy=-0.1, oz=0.1)
    P = oracle.matrices(g)
    rng = np.random.default_rng(3)
    xt = rng.uniform(0.5, 1.5, size=(g["nz"], g["ny"], g["nx"]))
    p = oracle.forward_project(P, xt, g["nu"], g["nv"], 1.0)
    return g, P, xt, p, rng


def mlem_counts():
    # EM preserves counts: after x+ = x A^T(p / Ax) / A^T 1, sum_j (A^T 1)_j x+_j
    # = sum of p over the rays with Ax > 0 (a property of the update, any x > 0)
    g, P, xt, p, rng = _iter_system()
    pn = p * (1 + 0.2 * rng.uniform(-1, 1, size=p.shape))
    x0 = rng.uniform(0.2, 2.0, size=xt.shape)
    x1 = oracle.mlem(P, pn, g["nx"], g["ny"], g["nz"], iters=1, x0=x0)
    sens = oracle.backproject(P, np.ones_like(p), g["nx"], g["ny"], g["nz"], 1.0)
    y0 = oracle.forward_project(P, x0, g["nu"], g["nv"], 1.0)
    lhs, rhs = (sens * x1).sum(), pn[y0 > 1e-9].sum()
    assert abs(lhs - rhs) <= 1e-12 * rhs, (lhs, rhs)
    assert (x1 >= 0).all()


def mlem_likelihood():
    # EM never decreases the Poisson log-likelihood sum_i p_i log y_i - y_i
    g, P, xt, p, rng = _iter_system()
    pn = p * (1 + 0.3 * rng.uniform(-1, 1, size=p.shape))
    x = np.ones_like(xt)
    prev = -np.inf
    for _ in range(8):
        x = oracle.mlem(P, pn, g["nx"], g["ny"], g["nz"], iters=1, x0=x)
        y = oracle.forward_project(P, x, g["nu"], g["nv"], 1.0)
        m = y > 0
        ll = (pn[m] * np.log(y[m]) - y[m]).sum() - y[~m].sum()
        assert ll >= prev - 1e-9 * abs(ll), (ll, prev)
        prev = ll


def iter_fixed_points():
    # consistent data: the true volume is a fixed point of MLEM and SART
    g, P, xt, p, _ = _iter_system()
    for nsub in (1, 3):
        xm = oracle.mlem(P, p, g["nx"], g["ny"], g["nz"], iters=1, subsets=nsub, x0=xt)
        xs = oracle.sart(P, p, g["nx"], g["ny"], g["nz"], iters=1, subsets=nsub, x0=xt)
        assert np.abs(xm - xt).max() <= 1e-13 and np.abs(xs - xt).max() <= 1e-13


def sart_constant_step():
    # both normalisations together map constants to constants: for p = A (c' 1)
    # every normalised residual (p_i - (A c 1)_i) / (A 1)_i equals c' - c, so one
    # step with lambda = 1 from c 1 lands on c' 1 exactly (every subset step too)
    g, P, xt, _, _ = _iter_system()
    one = np.ones_like(xt)
    p = oracle.forward_project(P, 2.5 * one, g["nu"], g["nv"], 1.0)
    for nsub in (1, 3):
        x = oracle.sart(P, p, g["nx"], g["ny"], g["nz"], iters=1, subsets=nsub, x0=0.7 * one)
        assert np.abs(x - 2.5).max() <= 1e-12, nsub
        x = oracle.mlem(P, p, g["nx"], g["ny"], g["nz"], iters=1, subsets=nsub, x0=0.7 * one)
        assert np.abs(x - 2.5).max() <= 1e-12, nsub


def iter_convergence():
    # consistent data and full column rank: both methods reach the true volume
    g, P, xt, p, _ = _iter_system()
    n = (g["nx"], g["ny"], g["nz"])
    assert np.abs(oracle.mlem(P, p, *n, iters=1000) - xt).max() <= 1e-10
    assert np.abs(oracle.mlem(P, p, *n, iters=300, subsets=4) - xt).max() <= 1e-10
    assert np.abs(oracle.sart(P, p, *n, iters=1000) - xt).max() <= 1e-10
    assert np.abs(oracle.sart(P, p, *n, iters=300, subsets=4, nonneg=True) - xt).max() <= 1e-10
    # and not in one step (the pins above would not see a no-op update)
    assert np.abs(oracle.sart(P, p, *n, iters=1) - xt).max() > 1e-2


ALL = [matrix_vs_ray, z_invariance, bp_constant, bp_linear, bp_fp_hat_matrix, bp_slab_points, adjoint_dot,
       symmetry, filter_impulse, filter_frequency, phantom_sphere, phantom_ray_integral,
       phantom_siddon, fdk_sphere, fdk_offcentre, fdk_ellipsoids, conv_vs_scipy, conv_adjoints,
       mlem_counts, mlem_likelihood, iter_fixed_points, sart_constant_step, iter_convergence]
