"""The two-pass core, the column-space error and the predictive mean on the GPU against the
FP64 oracle (oracle/projection.py), through the C ABI.

Both sides factor the same FP32 sketch (the oracle's, rounded once), the GPU with FP64
leaves so that its Q_hat differs from the oracle's only by FP32 storage.  Bars:
  S = Q^T K0 Q        2e-5 relative: kernel entries and Q_hat carried in three BF16 terms,
                      FP32 tensor-core accumulation over 4096-point ranges (at most 256 steps
                      of K = 16: 256 * 2^-23 = 3e-5 worst case), ranges folded in FP64
  column-space error  5e-3 absolute: ||K0||_F^2 - ||K0 Q||_F^2 with both norms to ~1e-6
  two-pass solve      1e-5 relative at nugget 1e-2 (S + tau I well conditioned)
  predictive mean     1e-12 relative for a given alpha (FP64 entries and sums); 1e-5 through
                      the whole path at nugget 1e-2
"""
import numpy as np
import pytest
import torch

import synth
from oracle import kernels as okk
from oracle import lowrank as olr
from oracle import omega as oom
from oracle import projection as opr
from oracle import sketch as osk

from gpu_util import col, host, rel

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


CASES = [
    # n, d, kind, ell, dim, block_rows
    (4096, 128, okk.SE, 0.1, 2, 1024),
    (9000, 256, okk.MATERN52, 0.15, 3, 2048),
]


@pytest.mark.parametrize("case", CASES)
def test_two_pass_core_solve_and_colspace_error(ctx, case):
    n, d, kind, ell, dim, b = case
    tau = 1e-2
    pts = synth.points(n, dim, 2)
    O = oom.omega_matrix(n, d, 8)
    Y = osk.sketch(pts.astype(np.float64), kind, ell, 1.2, O).astype(np.float32)   # common input
    plan = ck.Plan(n=n, d=d, dim=dim, block_rows=b, seed=8, refine_steps=1, leaf_fp64=1)
    kern = ck.Kernel(kind, ell, 1.2, tau)
    f = ck.tsqr(ctx, plan, kern, col(Y))
    tp = torch.from_numpy(pts).cuda()
    S, err = ck.project(ctx, f, plan, kern, tp)
    A = synth.rhs(n, 4, 3)
    X = host(ck.solve(ctx, f, col(A)))
    ck.check(ctx)
    t = olr.factorise(Y.astype(np.float64), O, tau, b)
    So = opr.two_pass_core(pts.astype(np.float64), kind, ell, 1.2, t.Q)
    eo = opr.colspace_error(pts.astype(np.float64), kind, ell, 1.2, t.Q)
    Xo = opr.two_pass_solve(t.Q, So, tau, A.astype(np.float64))
    es, ex = rel(host(S), So), rel(X, Xo)
    print("two-pass n=%d d=%d: S err %.2e, colspace %.4e vs %.4e, solve err %.2e" % (n, d, es, err, eo, ex))
    assert es <= 2e-5
    assert abs(err - eo) <= 5e-3
    assert ex <= 1e-5


def test_predictive_mean_for_a_given_alpha(ctx):
    n, n_new, dim = 5000, 700, 2
    pts = synth.points(n, dim, 4)
    xnew = synth.points(n_new, dim, 5)
    alpha = synth.rhs(n, 1, 6)[:, 0] * 1e4          # large, cancelling terms
    plan = ck.Plan(n=n, d=64, dim=dim)
    kern = ck.Kernel(ck.MATERN52, 0.2, 1.4, 1e-4)
    mu = ck.predict_mean(ctx, plan, kern, torch.from_numpy(pts).cuda(), torch.from_numpy(alpha.copy()).cuda(),
                         torch.from_numpy(xnew).cuda())
    ck.check(ctx)
    ref = okk.kernel_matrix(xnew.astype(np.float64), pts.astype(np.float64), okk.MATERN52, 0.2, 1.4) @ \
        alpha.astype(np.float64)
    e = rel(mu.cpu().numpy(), ref)
    print("predictive mean, given alpha: rel err %.2e" % e)
    assert e <= 1e-12


def test_predictive_mean_through_the_whole_path(ctx):
    n, d, n_new, dim, tau, ell = 4096, 128, 512, 2, 1e-2, 0.1
    pts = synth.points(n, dim, 7)
    y = synth.gp_targets(pts, 0.15, 1.0, tau, seed=7)
    xnew = synth.points(n_new, dim, 8)
    plan = ck.Plan(n=n, d=d, dim=dim, block_rows=1024, seed=9, refine_steps=1, leaf_fp64=1)
    kern = ck.Kernel(ck.SE, ell, 1.0, tau)
    tp = torch.from_numpy(pts).cuda()
    alpha = ck.kinv_a(ctx, plan, kern, tp, torch.from_numpy(y).cuda())
    mu = ck.predict_mean(ctx, plan, kern, tp, alpha, torch.from_numpy(xnew).cuda())
    ck.check(ctx)
    mo = opr.predictive_mean(pts.astype(np.float64), y.astype(np.float64), xnew.astype(np.float64), okk.SE, ell, 1.0,
                             tau, d, 9, 1024, 1)
    e = rel(mu.cpu().numpy(), mo)
    print("predictive mean through the path: rel err %.2e" % e)
    assert e <= 1e-5
