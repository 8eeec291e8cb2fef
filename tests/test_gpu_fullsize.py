"""Parity at the benchmark's full size, on outputs the oracle can compute one by one.

The 262144-point precision-form workload (d = 512, BF16 sketch) in the launch configuration
`bench.py` times: 48 rows of Y = K0 Omega, spread over the whole range, against the FP64
oracle's rows (a kernel-matrix row block times the explicit Omega).  The bar is the BF16
form's (2^-9 rounding of every kernel entry; 1.5e-3 measured at small and full size).
"""
import numpy as np
import pytest
import torch

import synth
from oracle import omega as oom
from oracle import sketch as osk

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


def test_sketch_full_size_sampled_rows(ctx):
    cfg = synth.CONFIGS["c3_bf16_n262144"]
    n, d, dim = cfg["n"], cfg["d"], cfg["dim"]
    pts = synth.points(n, dim, 0)
    plan = ck.Plan(n=n, d=d, dim=dim, block_rows=cfg["block_rows"], prec=ck.BF16, seed=4242)
    kern = ck.Kernel(cfg["kind"], cfg["ell"], cfg["var"], cfg["tau"])
    Y = ck.sketch(ctx, plan, kern, torch.from_numpy(pts).cuda())
    torch.cuda.synchronize()
    ck.check(ctx)
    rows = np.linspace(0, n - 1, 48).astype(np.int64)
    Yg = Y[torch.from_numpy(rows).cuda()].double().cpu().numpy()
    Yo = osk.sketch_rows(pts.astype(np.float64), rows, cfg["kind"], cfg["ell"], cfg["var"],
                         oom.omega_matrix(n, d, 4242))
    err = float(np.linalg.norm(Yg - Yo) / np.linalg.norm(Yo))
    print("full-size sketch, 48 sampled rows: rel err %.3e" % err)
    assert err <= 4e-3
