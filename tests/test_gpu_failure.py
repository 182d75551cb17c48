"""Failure detection on the GPU without a fault: a bounded wait that runs out.

The staging producer of the back-projector is told to skip one view's load
(bp_test_drop_view), so no copy ever completes that view's barrier. Every
wait in the kernel has a time limit: the consumers give up on the missing
view, the producer gives up on the slot they never release, both record
DEV_ERR_TIMEOUT in the context's device word and the CTA returns after the
copies it did issue have landed. The host then reads BP_ERR_TIMEOUT from
bp_device_status, and the same context (and CUDA context) keeps working: the
next call without the hook reproduces the result of a clean call bit for bit.

The problem is one wave of CTAs (64^3 voxels, 90 views) and the limit is
50 ms, so the failing launch ends in about a tenth of a second.
"""
import math

import pytest
import torch

from paper_2104_13248_gb300 import _lib, api, inputs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    import __graft_entry__
    __graft_entry__.build()


@pytest.mark.parametrize("sym,half", [(True, False), (False, False), (False, True)],
                         ids=["sym_fp32", "plain_fp32", "plain_fp16"])
def test_dropped_view_times_out_and_context_survives(sym, half):
    """The staged kernels: the mid-plane symmetric one (default for this
    centred geometry) and the plain z-column kernel, with FP32 and with
    FP16-stored projections."""
    g = inputs.preset("c1_small")["geom"]
    q = torch.from_numpy(inputs.uniform_array(11, (g["np"], g["nv"], g["nu"]), -1.0, 1.0)).float().cuda()
    if half:
        q = q.half()
    scale = math.pi / g["np"]
    with api.bp_create(g) as ctx:
        api.bp_set_symmetry(ctx, sym)
        plan = api.bp_get_plan(ctx)
        assert plan["symmetric"] == sym
        if (plan["bu16"] if half else plan["bu32"]) < 0:
            pytest.skip("the staged (TMA) kernel is not used for this geometry")
        ref = api.bp_backproject(ctx, q, scale=scale)
        api.bp_device_status(ctx)

        api.bp_set_timeout(ctx, 0.05)
        api.bp_test_drop_view(ctx, 7)
        vol = torch.zeros(ctx.vol_shape(), device="cuda")
        api.bp_backproject(ctx, q, vol=vol, scale=scale)
        with pytest.raises(_lib.BPError) as e:
            api.bp_device_status(ctx)
        assert e.value.status == _lib.BP_ERR_TIMEOUT

        # the word was cleared by the read, the hook is off: a clean call again
        api.bp_test_drop_view(ctx, -1)
        api.bp_device_status(ctx)
        again = api.bp_backproject(ctx, q, scale=scale)
        api.bp_device_status(ctx)
        assert torch.equal(again, ref)
        # other kernels on the same CUDA context are unaffected
        assert torch.isfinite(api.bp_filter(ctx, q.float())).all()


def test_failed_allocation_reports_oom_and_leaks_nothing(monkeypatch):
    """Host-side injection: the n-th device allocation of bp_create fails as an
    out-of-memory cudaMalloc would. Every n up to the number bp_create makes
    returns BP_ERR_OOM with a message, and the allocations made before the
    failing one are released (the library's live-allocation count is back
    where it was); past that number the context is created normally."""
    lib = _lib.load()
    g = inputs.preset("c1_small")["geom"]
    base = lib.bp_test_live_allocations()
    n_failed = 0
    for nth in range(1, 20):
        monkeypatch.setenv("BP_TEST_FAIL_ALLOC", str(nth))
        try:
            ctx = api.bp_create(g)
        except _lib.BPError as e:
            assert e.status == _lib.BP_ERR_OOM, e
            assert "out of memory" in str(e), e
            assert lib.bp_test_live_allocations() == base, nth
            n_failed += 1
            continue
        with ctx:
            assert lib.bp_test_live_allocations() > base
        break
    else:
        raise AssertionError("bp_create never succeeded")
    assert n_failed >= 4          # matrices, error word, filter tables, phantom buffer
    assert lib.bp_test_live_allocations() == base
    monkeypatch.delenv("BP_TEST_FAIL_ALLOC")
    with api.bp_create(g) as ctx:
        q = torch.ones(ctx.proj_shape(), device="cuda")
        api.bp_backproject(ctx, q)
        api.bp_device_status(ctx)
