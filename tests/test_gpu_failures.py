"""Failure paths, exercised without faulting the GPU: a device-side wait that runs out, a
non-finite input and a core that cannot be factorised are each reported as a status, and
the context keeps working afterwards.

The timeout is provoked by setting the context's wait limit to one nanosecond: every
bounded wait of the tensor-core sketch then gives up after sixteen short polls, the CTAs
that gave up drain their own copies and products (those waits keep their one-second limit),
free their tensor memory and leave, and the call reports CKINV_ETIMEOUT.  Restoring the
default limit, the same call must give the bits of an undisturbed run.
"""
import numpy as np
import pytest
import torch

import synth

from gpu_util import col

pytestmark = pytest.mark.gpu

ck = None


@pytest.fixture(scope="module")
def ctx():
    global ck
    import __graft_entry__
    __graft_entry__.build()
    from paper_1312_1869_gb300 import ckinv as _ck
    ck = _ck
    c = _ck.Context(0)
    yield c
    c.close()


def test_sketch_wait_timeout_is_reported_and_the_context_recovers(ctx):
    n, d = 16384, 512          # 128 CTAs: one wave, so a timed-out call ends in seconds
    pts = torch.from_numpy(synth.points(n, 2, 3)).cuda()
    plan = ck.Plan(n=n, d=d, dim=2, prec=ck.BF16, seed=9)
    kern = ck.Kernel(ck.SE, 0.1, 1.0, 1e-6)
    Y_ref = ck.sketch(ctx, plan, kern, pts).clone()
    ck.check(ctx)
    timed_out = False
    try:
        ck.set_wait_limit(ctx, 1)
        for _ in range(4):
            ck.sketch(ctx, plan, kern, pts)
            try:
                ck.check(ctx)
            except ck.CKInvError as e:
                assert e.status == ck.ETIMEOUT, e
                timed_out = True
                break
    finally:
        ck.set_wait_limit(ctx, 0)
    assert timed_out, "no wait ran out with a 1 ns limit"
    Y = ck.sketch(ctx, plan, kern, pts)
    ck.check(ctx)
    assert torch.equal(Y, Y_ref)


def test_wait_limit_rejects_out_of_range_values(ctx):
    with pytest.raises(ck.CKInvError) as e:
        ck.set_wait_limit(ctx, 61 * 10**9)
    assert e.value.status == ck.EINVAL


def test_non_finite_points_are_reported(ctx):
    n, d = 2048, 64
    x = synth.points(n, 2, 4)
    x[777, 1] = np.nan
    plan = ck.Plan(n=n, d=d, dim=2, prec=ck.BF16, seed=1)
    kern = ck.Kernel(ck.SE, 0.2, 1.0, 1e-4)
    ck.sketch(ctx, plan, kern, torch.from_numpy(x).cuda())
    with pytest.raises(ck.CKInvError) as e:
        ck.check(ctx)
    assert e.value.status == ck.EINVAL and "non-finite" in str(e.value)
    x[777, 1] = 0.5
    ck.sketch(ctx, plan, kern, torch.from_numpy(x).cuda())
    ck.check(ctx)


def test_non_finite_targets_fail_the_likelihood_call(ctx):
    n, d = 2048, 64
    x = synth.points(n, 2, 5)
    y = synth.gp_targets(x, 0.2, 1.0, 1e-3, seed=5)
    y[10] = np.inf
    plan = ck.Plan(n=n, d=d, dim=2, block_rows=512, prec=ck.FP32, seed=1)
    with pytest.raises(ck.CKInvError) as e:
        ck.nll_grad(ctx, plan, ck.Kernel(ck.SE, 0.2, 1.0, 1e-3), torch.from_numpy(x).cuda(),
                    torch.from_numpy(y).cuda())
    assert e.value.status == ck.EINVAL


def test_an_unfactorisable_core_is_reported_as_singular(ctx):
    """A sketch with an infinite entry leaves B and C' without a finite pivot: the LU
    reports it (CKINV_ESINGULAR) instead of returning NaNs silently."""
    n, d = 2048, 64
    rng = np.random.default_rng(3)
    Y = rng.standard_normal((n, d)).astype(np.float32)
    Y[5, 3] = np.inf
    plan = ck.Plan(n=n, d=d, block_rows=512, seed=2)
    f = ck.tsqr(ctx, plan, ck.Kernel(ck.SE, 1.0, 1.0, 1e-3), col(Y))
    with pytest.raises(ck.CKInvError) as e:
        ck.check(ctx)
    assert e.value.status == ck.ESINGULAR
    f.free()
    Y[5, 3] = 0.25
    f = ck.tsqr(ctx, plan, ck.Kernel(ck.SE, 1.0, 1.0, 1e-3), col(Y))
    ck.check(ctx)
    f.free()
