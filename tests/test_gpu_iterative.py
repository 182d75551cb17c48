"""MLEM / OS-EM and SART / SIRT on the GPU vs the FP64 oracle, iterate by iterate.

Data: a voxelised ellipsoid phantom of the small FDK workload (64^3, 90
views, 128^2 detector), its projections by the oracle's forward projector
(FP64, rounded to FP32 for both sides), plus 10% multiplicative noise for
the inconsistent case. Tolerance: max |gpu - oracle| / max |oracle| <= 1e-4
after up to three passes. Each pass composes one forward and one
back-projection (each within 1e-5 of the oracle in FP32) with element-wise
steps that add a few ulp; the iterations do not amplify errors (MLEM and
SART with lambda <= 1 are non-expansive here), so three passes stay below
6e-5.
"""
import math

import numpy as np
import pytest
import torch

import oracle
from paper_2104_13248_gb300 import api, inputs, iterative

pytestmark = pytest.mark.gpu

TOL = 1e-4


def rel(a, b):
    return float(np.abs(np.asarray(a, np.float64) - b).max() / max(np.abs(b).max(), 1e-300))


@pytest.fixture(scope="module", autouse=True)
def _built():
    import __graft_entry__
    __graft_entry__.build()


@pytest.fixture(scope="module")
def problem():
    p = inputs.preset("c1_small")
    g = p["geom"]
    E = inputs.random_ellipsoids(p["seed"], p["n_ell"], p["axes"], g)
    xs, ys, zs = oracle.voxel_centres(g)
    X, Y, Z = np.meshgrid(xs, ys, zs, indexing="ij")
    dens = inputs.density_at(E, X, Y, Z).transpose(2, 1, 0)      # [z][y][x]
    P = oracle.matrices(g)
    q = oracle.forward_project(P, dens, g["nu"], g["nv"], 1.0)
    rng = np.random.default_rng(8)
    noisy = q * (1.0 + 0.1 * rng.uniform(-1.0, 1.0, size=q.shape))
    return dict(g=g, P=P, x=dens, q=q.astype(np.float32), noisy=noisy.astype(np.float32))


@pytest.mark.parametrize("subsets,iters,data", [(1, 3, "q"), (5, 2, "noisy"), (9, 1, "q")])
def test_mlem_matches_oracle(problem, subsets, iters, data):
    g, P = problem["g"], problem["P"]
    q = problem[data]
    ref = oracle.mlem(P, q, g["nx"], g["ny"], g["nz"], iters=iters, subsets=subsets)
    with api.bp_create(g) as ctx:
        x = iterative.mlem(ctx, torch.from_numpy(q).cuda(), iters=iters, subsets=subsets)
        api.bp_device_status(ctx)
    assert rel(x.cpu().numpy(), ref) <= TOL


@pytest.mark.parametrize("subsets,iters,lam,nonneg,data",
                         [(1, 3, 1.0, False, "q"), (6, 2, 0.8, True, "noisy"), (10, 1, 1.0, False, "noisy")])
def test_sart_matches_oracle(problem, subsets, iters, lam, nonneg, data):
    g, P = problem["g"], problem["P"]
    q = problem[data]
    ref = oracle.sart(P, q, g["nx"], g["ny"], g["nz"], iters=iters, subsets=subsets, lam=lam, nonneg=nonneg)
    with api.bp_create(g) as ctx:
        x = iterative.sart(ctx, torch.from_numpy(q).cuda(), iters=iters, subsets=subsets, lam=lam,
                           nonneg=nonneg)
        api.bp_device_status(ctx)
    assert rel(x.cpu().numpy(), ref) <= TOL
    if nonneg:
        assert float(x.min()) >= 0.0


def test_iterations_approach_the_phantom(problem):
    """More OS-EM / SART passes bring the reconstruction closer to the phantom
    (consistent data, inside the field of view)."""
    g = problem["g"]
    q = torch.from_numpy(problem["q"]).cuda()
    truth = torch.from_numpy(problem["x"]).float().cuda()
    with api.bp_create(g) as ctx:
        errs = []
        for it in (1, 4, 12):
            x = iterative.mlem(ctx, q, iters=it, subsets=10)
            errs.append(float((x - truth).norm() / truth.norm()))
        errs_s = []
        for it in (1, 4, 12):
            x = iterative.sart(ctx, q, iters=it, subsets=10, nonneg=True)
            errs_s.append(float((x - truth).norm() / truth.norm()))
    assert errs[0] > errs[1] > errs[2] and errs[2] < 0.5 * errs[0], errs
    assert errs_s[0] > errs_s[1] > errs_s[2] and errs_s[2] < 0.5 * errs_s[0], errs_s


def test_elementwise_steps_exact():
    """The element-wise calls against their FP32 definitions, with ragged
    lengths (vector body plus scalar tail) and an unaligned start."""
    from paper_2104_13248_gb300 import _lib
    lib = _lib.load()
    g = torch.Generator(device="cuda").manual_seed(1)
    for n in (1, 7, 4096 + 3):
        base = torch.rand(n + 1, device="cuda", generator=g)
        p, y, w = (torch.rand(n, device="cuda", generator=g) for _ in range(3))
        y[::5] = 0.0
        w[::7] = 0.0
        for off in (0, 1):
            base[off:off + n].copy_(p)
            pp, yy = base[off:off + n], y      # off = 1: 4-byte aligned only (scalar path)
            r = torch.empty(n, device="cuda")
            iterative.check(lib.it_ratio(iterative._p(pp), iterative._p(yy), iterative._p(r), n, 1e-9,
                                         iterative._s()))
            torch.cuda.synchronize()
            ref = torch.where(yy > 1e-9, pp / torch.where(yy > 1e-9, yy, torch.ones_like(yy)), torch.zeros_like(yy))
            assert torch.equal(r, ref)
        r = torch.empty(n, device="cuda")
        iterative.check(lib.it_residual(iterative._p(p), iterative._p(y), iterative._p(w), iterative._p(r), n,
                                        1e-9, iterative._s()))
        torch.cuda.synchronize()
        ref = torch.where(w > 1e-9, (p - y) / torch.where(w > 1e-9, w, torch.ones_like(w)), torch.zeros_like(w))
        assert torch.equal(r, ref)
        x = torch.rand(n, device="cuda", generator=g) - 0.5
        x2 = x.clone()
        iterative.check(lib.it_sart_update(iterative._p(x2), iterative._p(p), iterative._p(w), n, 0.7, 1, 1e-9,
                                           iterative._s()))
        torch.cuda.synchronize()
        upd = torch.where(w > 1e-9, x + (0.7 * p) / torch.where(w > 1e-9, w, torch.ones_like(w)), x)
        assert torch.equal(x2, torch.clamp(upd, min=0.0))
        x3 = x.clone()
        iterative.check(lib.it_mlem_update(iterative._p(x3), iterative._p(p), iterative._p(w), n, 1e-9,
                                           iterative._s()))
        torch.cuda.synchronize()
        assert torch.equal(x3, torch.where(w > 1e-9, (x * p) / torch.where(w > 1e-9, w, torch.ones_like(w)), x))
        f = torch.empty(n, device="cuda")
        iterative.fill(f, 2.5)
        torch.cuda.synchronize()
        assert bool((f == 2.5).all())
