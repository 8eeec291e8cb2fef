"""Parity at the benchmark's full size, on outputs the oracle can compute one by one.

The 262144-point precision-form workload (d = 512) in the launch configuration `bench.py`
times: 48 rows of Y = K0 Omega, spread over the whole range, against the FP64 oracle's rows
(a kernel-matrix row block times the explicit Omega).  Bars: the BF16 form's 4e-3 (2^-9
rounding of every kernel entry; 1.5e-3 measured at small and full size); for the multi-term
forms, whose kernel entries carry 16 or 24 bits, the accumulation of the tensor cores sets
the bar at this length: each K = 16 step of an MMA adds into the FP32 accumulator with a
relative error up to 2^-23 (measured: 1.75e-4 at n = 65536 against 4e-6 at n = 2085), so the
bar is max(1e-5, (n / 16) 2^-23) - the sum of those steps' worst cases.
"""
import os

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


def accumulation_bar(n):
    return max(1e-5, (n / 16.0) * 2.0 ** -23)


@pytest.mark.parametrize("prec", ["bf16", "bf16x3", "fp32_wht"])
def test_sketch_full_size_sampled_rows(ctx, prec):
    cfg = synth.CONFIGS["c3_bf16_n262144"]
    n, d, dim = cfg["n"], cfg["d"], cfg["dim"]
    pts = synth.points(n, dim, 0)
    plan = ck.Plan(n=n, d=d, dim=dim, block_rows=cfg["block_rows"], prec=ck.PRECISIONS[prec], seed=4242)
    kern = ck.Kernel(cfg["kind"], cfg["ell"], cfg["var"], cfg["tau"])
    Y = ck.sketch(ctx, plan, kern, torch.from_numpy(pts).cuda())
    torch.cuda.synchronize()
    ck.check(ctx)
    rows = np.linspace(0, n - 1, 48).astype(np.int64)
    Yg = Y[torch.from_numpy(rows).cuda()].double().cpu().numpy()
    Yo = osk.sketch_rows(pts.astype(np.float64), rows, cfg["kind"], cfg["ell"], cfg["var"],
                         oom.omega_matrix(n, d, 4242))
    err = float(np.linalg.norm(Yg - Yo) / np.linalg.norm(Yo))
    tol = {"bf16": 4e-3, "bf16x3": accumulation_bar(n), "fp32_wht": 1e-5}[prec]
    print("full-size sketch (%s), 48 sampled rows: rel err %.3e (bar %.1e)" % (prec, err, tol))
    assert err <= tol


@pytest.mark.parametrize("prec", ["fp32", "bf16x3", "fp32_wht"])
def test_materialised_kernel_sketch_full_size_sampled_rows(ctx, prec):
    """The plain method with K held in HBM: n = 65536 points in [0, 1]^3, Matern-5/2 l = 0.15,
    d = 256.  K0 (17.2 GB FP32) is materialised by the library, then sketched as a given
    matrix (FP32 SIMT contraction, three BF16 terms on the tensor cores, or the fast
    Walsh-Hadamard transform over K0's columns in FP32); 48 rows of Y
    against the oracle's rows, which it builds from the points in FP64."""
    cfg = synth.CONFIGS["c2_dense_n65536"]
    n, d, dim = cfg["n"], cfg["d"], cfg["dim"]
    pts = synth.points(n, dim, 0)
    plan = ck.Plan(n=n, d=d, dim=dim, block_rows=cfg["block_rows"], prec=ck.PRECISIONS[prec], seed=11)
    kern = ck.Kernel(cfg["kind"], cfg["ell"], cfg["var"], cfg["tau"])
    K = ck.kernel_matrix(ctx, plan, kern, torch.from_numpy(pts).cuda())
    Y = ck.sketch(ctx, plan, ck.Kernel(ck.DENSE, 0, 0, cfg["tau"]), K=K)
    torch.cuda.synchronize()
    ck.check(ctx)
    del K
    rows = np.linspace(0, n - 1, 48).astype(np.int64)
    Yg = Y[torch.from_numpy(rows).cuda()].double().cpu().numpy()
    Yo = osk.sketch_rows(pts.astype(np.float64), rows, cfg["kind"], cfg["ell"], cfg["var"],
                         oom.omega_matrix(n, d, 11))
    err = float(np.linalg.norm(Yg - Yo) / np.linalg.norm(Yo))
    tol = accumulation_bar(n) if prec == "bf16x3" else 1e-5
    print("materialised-K sketch (%s), 48 sampled rows: rel err %.3e (bar %.1e)" % (prec, err, tol))
    assert err <= tol


GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "likelihood_n131072_d384.json")


@pytest.mark.parametrize("prec", ["fp32_wht", "fp32"])
@pytest.mark.parametrize("leaf64", [0, 1])
def test_likelihood_full_size_against_the_stored_oracle_value(ctx, leaf64, prec):
    """The 131072-point likelihood workload (SE l = 0.12, nugget 1e-4, d = 384) in the forms
    that carry kernel entries and the sketch to FP32 precision (the fast-transform sketch and
    the SIMT one) against the FP64 oracle's value stored in tests/golden (written by
    make_likelihood_golden.py, which calls only the oracle).  Bar for the NLL: 2 x the floor of
    FP32 working precision - the oracle's own change with every kernel entry rounded to FP32,
    the two sketches and alpha stored in FP32 and FP32 leaf factorisations (2.2e-4 here; the
    FP64-leaf runs are held to the same bar).  The gradient is printed, and asserted only for
    components that this floor leaves determined to better than 5 % (none here: kappa(Y) is
    about 1e11, FP32 entries alone move the gradient by 240-650 % and the full working
    precision by 19-220 %).  The three-term tensor-core form is not held to
    this bar: its FP32 accumulation over n = 131072 points leaves Y about 3e-4 off (the full-size
    sketch test), which moves its NLL by about 1e-3."""
    import json
    if not os.path.exists(GOLDEN):
        pytest.skip("stored oracle likelihood not written")
    gold = json.load(open(GOLDEN))
    if "fp32_working_precision" not in gold:
        pytest.skip("stored oracle likelihood has no FP32 working-precision floor")
    cfg = synth.CONFIGS["c4_nll_n131072"]
    n, d, dim = cfg["n"], cfg["d"], cfg["dim"]
    pts = synth.points(n, dim, seed=0)
    y = synth.gp_targets(pts, cfg["ell"], cfg["var"], cfg["tau"], seed=0)
    plan = ck.Plan(n=n, d=d, dim=dim, block_rows=cfg["block_rows"], prec=ck.PRECISIONS[prec], seed=cfg["seed"],
                   refine_steps=1, leaf_fp64=leaf64)
    kern = ck.Kernel(cfg["kind"], cfg["ell"], cfg["var"], cfg["tau"])
    val, g = ck.nll_grad(ctx, plan, kern, torch.from_numpy(pts).cuda(), torch.from_numpy(y).cuda())
    ex, fl = gold["exact"], gold["fp32_working_precision"]
    floor_v = abs(fl["nll"] - ex["nll"]) / abs(ex["nll"])
    floor_g = np.abs(np.array(fl["grad"]) - ex["grad"]) / np.abs(ex["grad"])
    ev = abs(val - ex["nll"]) / abs(ex["nll"])
    eg = np.abs(np.array(g) - ex["grad"]) / np.abs(ex["grad"])
    print("likelihood n=%d %s leaf64=%d: NLL err %.2e (floor %.2e); grad err %s (floor %s)"
          % (n, prec, leaf64, ev, floor_v, eg, floor_g))
    assert ev <= 2 * floor_v
    det = floor_g <= 0.05
    assert np.all(eg[det] <= np.maximum(1e-3, 2 * floor_g[det]))
