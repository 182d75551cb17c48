"""Differentiation: back-projection as an autograd Function whose backward is
the matched forward projector, checked by the dot-product test, central
finite differences, the FP64 oracle's gradient and the oracle's own
least-squares iterates (32^3 subcase of the differentiable workload)."""
import numpy as np
import pytest
import torch

import oracle
from paper_2104_13248_gb300 import api, autograd, inputs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    import __graft_entry__
    __graft_entry__.build()


def small_geom():
    g = inputs.scaled_geom(inputs.preset("c4_diff")["geom"], np=36, nu=96, nv=80, du=0.8, dv=0.8,
                           nx=32, ny=32, nz=32, sx=1.0, sy=1.0, sz=1.0)
    return g


@pytest.fixture(scope="module")
def setup():
    g = small_geom()
    E = inputs.random_ellipsoids(100, 8, (2.0, 8.0), g)
    p = oracle.phantom_project(g, E).astype(np.float32)
    return g, p, oracle.matrices(g)


def test_autograd_matches_adjoint_pair(setup):
    g, p, P = setup
    with api.bp_create(g) as ctx:
        q = torch.from_numpy(inputs.uniform_array(3, ctx.proj_shape(), -1, 1).astype(np.float32)).cuda()
        q.requires_grad_(True)
        vol = autograd.back_project(ctx, q, 0.3)
        w = torch.from_numpy(inputs.uniform_array(4, ctx.vol_shape(), -1, 1).astype(np.float32)).cuda()
        (vol * w).sum().backward()
        # d/dq <BP q, w> = FP w
        ref = api.fp_project(ctx, w, scale=0.3)
        # the forward projector accumulates with atomics: equal up to summation order
        assert (q.grad - ref).abs().max().item() <= 1e-6 * ref.abs().max().item()
        x = w.clone().requires_grad_(True)
        pr = autograd.forward_project(ctx, x, 0.3)
        (pr * q.detach()).sum().backward()
        assert torch.equal(x.grad, api.bp_backproject(ctx, q.detach(), scale=0.3))


def test_dot_product(setup):
    g, p, P = setup
    with api.bp_create(g) as ctx:
        for seed in range(3):
            x = torch.from_numpy(inputs.uniform_array(10 + seed, ctx.vol_shape(), -1, 1).astype(np.float32)).cuda()
            q = torch.from_numpy(inputs.uniform_array(20 + seed, ctx.proj_shape(), -1, 1).astype(np.float32)).cuda()
            ax = api.fp_project(ctx, x)
            atq = api.bp_backproject(ctx, q)
            lhs = torch.dot(ax.double().flatten(), q.double().flatten()).item()
            rhs = torch.dot(x.double().flatten(), atq.double().flatten()).item()
            scale = atq.double().norm().item() * x.double().norm().item()
            assert abs(lhs - rhs) <= 1e-6 * scale


def test_finite_differences(setup):
    g, p, P = setup
    with api.bp_create(g) as ctx:
        pt = torch.from_numpy(p).cuda()
        x = torch.from_numpy(inputs.uniform_array(31, ctx.vol_shape(), 0, 0.5).astype(np.float32)).cuda()
        x.requires_grad_(True)
        loss = autograd.loss_fn(ctx, x, pt)
        (grad,) = torch.autograd.grad(loss, x)
        for d in range(8):
            delta = torch.from_numpy(inputs.uniform_array(40 + d, ctx.vol_shape(), -1, 1).astype(np.float32)).cuda()
            eps = 1e-2
            with torch.no_grad():
                lp = autograd.loss_fn(ctx, x + eps * delta, pt).item()
                lm = autograd.loss_fn(ctx, x - eps * delta, pt).item()
            fd = (lp - lm) / (2 * eps)
            an = torch.dot(grad.double().flatten(), delta.double().flatten()).item()
            assert abs(fd - an) <= 1e-3 * abs(an), (d, fd, an)


def test_gradient_matches_oracle(setup):
    g, p, P = setup
    with api.bp_create(g) as ctx:
        x32 = inputs.uniform_array(31, ctx.vol_shape(), 0, 0.5).astype(np.float32)
        x = torch.from_numpy(x32).cuda().requires_grad_(True)
        loss = autograd.loss_fn(ctx, x, torch.from_numpy(p).cuda())
        (grad,) = torch.autograd.grad(loss, x)
    r = oracle.forward_project(P, x32, g["nu"], g["nv"]) - p
    ref = oracle.backproject(P, r, g["nx"], g["ny"], g["nz"], 1.0)
    err = np.abs(grad.cpu().numpy() - ref).max() / np.abs(ref).max()
    assert err <= 1e-5, err


def test_least_squares_matches_oracle_iterates(setup):
    g, p, P = setup
    iters = 20
    with api.bp_create(g) as ctx:
        L = autograd.lipschitz(ctx, iters=30)
        x, losses = autograd.least_squares(ctx, torch.from_numpy(p).cuda(), iters=iters, L=L)
        x = x.cpu().numpy()
    # oracle gradient descent with the same step
    xo = np.zeros((g["nz"], g["ny"], g["nx"]))
    for _ in range(iters):
        r = oracle.forward_project(P, xo, g["nu"], g["nv"]) - p
        xo = xo - oracle.backproject(P, r, g["nx"], g["ny"], g["nz"], 1.0) / L
    assert all(b < a for a, b in zip(losses, losses[1:])), losses
    assert losses[-1] < 0.5 * losses[0]
    err = np.abs(x - xo).max() / np.abs(xo).max()
    assert err <= 1e-4, err


def test_batched_least_squares_equals_single(setup):
    g, p, P = setup
    with api.bp_create(g) as ctx:
        p2 = torch.from_numpy(np.stack([p, 0.5 * p])).cuda()
        L = autograd.lipschitz(ctx, iters=20)
        xb, _ = autograd.least_squares(ctx, p2, iters=5, L=L)
        x1, _ = autograd.least_squares(ctx, p2[1], iters=5, L=L)
        assert torch.allclose(xb[1], x1, rtol=1e-5, atol=1e-6 * x1.abs().max().item())


def test_least_squares_elementwise_exact():
    """The least-squares residual, loss, gradient scale and update against
    their FP32 definitions (bit for bit; the loss's FP64 sum to 1e-12), with
    ragged lengths (vector body and scalar tail) and an unaligned start."""
    import ctypes

    from paper_2104_13248_gb300 import _lib
    lib = _lib.load()
    P = lambda t: ctypes.c_void_p(t.data_ptr())
    S = lambda: ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    g = torch.Generator(device="cuda").manual_seed(2)
    for n in (1, 7, 4096 + 3):
        for off in (0, 1):
            base = torch.rand(n + 1, device="cuda", generator=g)
            y = base[off:off + n]
            p = torch.rand(n, device="cuda", generator=g)
            r = torch.empty(n, device="cuda")
            loss = torch.empty((), dtype=torch.float64, device="cuda")
            _lib.check(lib.it_ls_residual(P(y), P(p), P(r), n, P(loss), S()))
            torch.cuda.synchronize()
            assert torch.equal(r, y - p)
            ref = 0.5 * float(((y - p).double() ** 2).sum())
            assert abs(float(loss) - ref) <= 1e-12 * max(ref, 1e-300)
            s = torch.tensor(-1.7, dtype=torch.float64, device="cuda")
            out = torch.empty(n, device="cuda")
            _lib.check(lib.it_scale(P(r), P(s), P(out), n, S()))
            torch.cuda.synchronize()
            assert torch.equal(out, r * torch.tensor(-1.7, dtype=torch.float32, device="cuda"))
            x = torch.rand(n, device="cuda", generator=g)
            x2 = x.clone()
            autograd.gd_step(x2, r, 0.37)
            torch.cuda.synchronize()
            assert torch.equal(x2, torch.sub(x, torch.mul(torch.tensor(0.37, device="cuda"), r)))
    # the loss Function's gradient through autograd: g (y - p)
    y = torch.rand(1000, device="cuda", generator=g, requires_grad=True)
    p = torch.rand(1000, device="cuda", generator=g)
    loss = autograd.ResidualLoss.apply(y, p)
    loss.backward(torch.tensor(2.0, dtype=torch.float64, device="cuda"))
    assert torch.equal(y.grad, (y.detach() - p) * torch.tensor(2.0, device="cuda"))
