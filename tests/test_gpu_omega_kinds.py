"""The four choices of Omega (Definition 1's T = Walsh-Hadamard, discrete Hartley, discrete
cosine, and Sec. 5.1's scaled Gaussian projection) on the GPU against the FP64 oracle, and
the blocking simulation's covariance K = E D E^T (Sec. 5.1) through the materialised path.

Bars: Omega entrywise to FP32 rounding (each entry is evaluated in FP64 and rounded once on
the GPU: |diff| <= 2^-24 |Omega_kj| plus one FP64-level ulp of slack); the sketch of K in FP32
1e-5 (the Y bar); K^-1 A 1e-5 with FP64 leaves on this well-conditioned simulation (the
eigenvalues exp(-0.01 i) decay slowly, so the d columns of Y are far from dependent); the
matrix-free sketch with a dense Omega on the tensor cores max(1e-5, (n / 16) 2^-23), the bound
of their FP32 accumulation (as for the multi-term forms at full size).
"""
import numpy as np
import pytest
import torch

import synth
from oracle import lowrank as olr
from oracle import omega as oom
from oracle import sketch as osk
from oracle import transforms as otr

from gpu_util import col, host, rel

pytestmark = pytest.mark.gpu

ck = None
KINDS = ["wht", "gaussian", "hartley", "cosine"]


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


def oracle_omega(kind, n, d, seed):
    if kind == "wht":
        return oom.omega_matrix(n, d, seed)
    if kind == "gaussian":
        return oom.gaussian_omega(n, d, seed)
    return otr.omega_matrix_t(n, d, seed, kind)


def kind_id(kind):
    return {"wht": ck.WHT, "gaussian": ck.GAUSSIAN, "hartley": ck.HARTLEY, "cosine": ck.COSINE}[kind]


@pytest.mark.parametrize("kind", KINDS)
@pytest.mark.parametrize("n,d", [(2000, 64), (4096, 128), (777, 48)])
def test_omega_matrix_matches_the_oracle(ctx, kind, n, d):
    Om = host(ck.omega_matrix(ctx, n, d, 11, kind_id(kind)))
    ck.check(ctx)
    Oo = oracle_omega(kind, n, d, 11)
    assert np.all(np.abs(Om - Oo) <= 2.0 ** -24 * np.abs(Oo) + 1e-15)


@pytest.mark.parametrize("kind", KINDS)
def test_blocking_simulation_solve_against_the_oracle(ctx, kind):
    n, d, b, tau, m = 2000, 64, 512, 1e-3, 4
    K = synth.ede_matrix(n, seed=2)
    A = synth.rhs(n, m, 2)
    plan = ck.Plan(n=n, d=d, block_rows=b, prec=ck.FP32, seed=5, refine_steps=1, leaf_fp64=1,
                   omega_kind=kind_id(kind))
    dense = ck.Kernel(ck.DENSE, 0, 0, tau)
    Kg = col(K)
    Y = ck.sketch(ctx, plan, dense, K=Kg)
    Yh = host(Y)
    f = ck.tsqr(ctx, plan, dense, Y)
    X = host(ck.solve(ctx, f, col(A)))
    ck.check(ctx)
    K32 = K.astype(np.float32).astype(np.float64)
    O = oracle_omega(kind, n, d, 5)
    Yo = osk.sketch_dense(K32, O)
    fo = olr.factorise(Yo, O, tau, b)
    Xo = olr.solve_refined(fo, A.astype(np.float64), 1)
    ey, ex = rel(Yh, Yo), rel(X, Xo)
    print("EDE^T n=%d %s: Y err %.2e, K^-1 A err %.2e" % (n, kind, ey, ex))
    assert ey <= 1e-5
    assert ex <= 1e-5


@pytest.mark.parametrize("kind", ["hartley", "gaussian"])
def test_matrix_free_sketch_with_a_dense_omega(ctx, kind):
    n, d = 3000, 64
    pts = synth.points(n, 2, 9)
    plan = ck.Plan(n=n, d=d, dim=2, prec=ck.BF16X3, seed=3, omega_kind=kind_id(kind))
    kern = ck.Kernel(ck.SE, 0.15, 1.1, 1e-4)
    Y = host(ck.sketch(ctx, plan, kern, torch.from_numpy(pts).cuda()))
    ck.check(ctx)
    Yo = osk.sketch(pts.astype(np.float64), 0, 0.15, 1.1, oracle_omega(kind, n, d, 3))
    e = rel(Y, Yo)
    tol = max(1e-5, (n / 16.0) * 2.0 ** -23)   # the tensor cores' FP32 accumulation (tests/test_gpu_fullsize.py)
    print("matrix-free sketch, %s Omega: rel err %.2e (bar %.1e)" % (kind, e, tol))
    assert e <= tol
