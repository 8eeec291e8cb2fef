"""The row-shard entry points on one GPU, with every shard of a problem held by one process
(the orchestration of several processes is tested over gloo in test_sharded.py).

  * a shard's rows of the sketch are bit-identical to the same rows of the whole sketch (the
    contraction over all points runs in the same order), in the tensor-core and SIMT forms;
  * the sharded R and X equal the FP64 oracle's single-process R and X (FP64 leaves, no
    refinement on either side), for 2, 3 and 4 shards, and the library's single-GPU solve.
"""
import numpy as np
import pytest
import torch

import synth
from oracle import lowrank as olr

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


@pytest.mark.parametrize("prec", ["bf16", "bf16x3", "fp32", "fp32_wht"])
def test_sketch_rows_are_the_rows_of_the_sketch(ctx, prec):
    n, d = 5000, 128
    pts = torch.from_numpy(synth.points(n, 2, 1)).cuda()
    plan = ck.Plan(n=n, d=d, dim=2, prec=ck.PRECISIONS[prec], seed=4)
    kern = ck.Kernel(ck.SE, 0.1, 1.0, 1e-4)
    Y = ck.sketch(ctx, plan, kern, pts)
    for r0, m in [(0, 1000), (1000, 2500), (4000, 1000), (777, 130)]:
        Yr = ck.sketch_rows(ctx, plan, kern, r0, m, points=pts)
        torch.cuda.synchronize()
        assert torch.equal(Yr, Y[r0:r0 + m]), (prec, r0, m)
    ck.check(ctx)


@pytest.mark.parametrize("G", [2, 3, 4])
def test_sharded_solve_equals_the_oracle_and_the_single_gpu_solve(ctx, G):
    from paper_1312_1869_gb300 import sharded
    n, d, ell, tau, m = 4096, 128, 0.1, 1e-3, 4
    pts_np = synth.points(n, 2, 2)
    A_np = synth.rhs(n, m, 2)
    plan = ck.Plan(n=n, d=d, dim=2, block_rows=512, prec=ck.FP32, seed=7, refine_steps=0, leaf_fp64=1)
    kern = ck.Kernel(ck.SE, ell, 1.0, tau)
    pts = torch.from_numpy(pts_np).cuda()
    bounds = sharded.shard_bounds(n, G, d)
    A_rows = {g: col(A_np[bounds[g]:bounds[g + 1]]) for g in range(G)}
    X, R, _ = sharded.kinv_a_sharded(sharded.LibraryBackend(ctx), sharded.LocalComm(), plan, kern, pts, A_rows,
                                     list(range(G)), G)
    ck.check(ctx)
    Xs = np.vstack([host(X[g]) for g in range(G)])
    Xo, fo, _ = olr.kinv_a(pts_np.astype(np.float64), A_np.astype(np.float64), 0, ell, 1.0, tau, d, 7, 512,
                           refine_steps=0)
    f1 = ck.tsqr(ctx, plan, kern, ck.sketch(ctx, plan, kern, pts))
    R1 = host(f1.r())
    X1 = host(ck.solve(ctx, f1, col(A_np)))
    ck.check(ctx)
    er, er1, ex, e1 = rel(host(R), fo.R), rel(host(R), R1), rel(Xs, Xo), rel(Xs, X1)
    print("G=%d shards: R err vs oracle %.2e, vs one GPU %.2e; X err vs oracle %.2e, vs one GPU %.2e"
          % (G, er, er1, ex, e1))
    assert er1 <= 1e-10          # FP64 leaves and tree: the tree's shape changes only rounding
    assert e1 <= 1e-5            # Q_hat stored in FP32 on both
    assert er <= 1e-4 and ex <= 1e-4
