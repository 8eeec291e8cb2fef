"""Parity of the CUDA path (through the C ABI) with the FP64 oracle on seeded inputs.

Tolerances (relative Frobenius error unless stated):
  Omega signs and columns   bit-exact (integer work)
  sketch FP32 / BF16X3      1e-5  (the bar on Y in FP32)
  sketch BF16X2             3e-5  (kernel tile carried to ~2^-17 before FP32 accumulation)
  sketch BF16               4e-3  (kernel tile rounded to 2^-9 relative)
  TSQR R, Q_hat             2e-5 on well-conditioned inputs (FP32 Householder, u_32 * d)
  K^-1 A                    1e-4  (the bar on the solve, FP32 path + refinement)
"""
import math

import numpy as np
import pytest
import torch

import synth
from oracle import kernels as okk
from oracle import lowrank as olr
from oracle import omega as oom
from oracle import sketch as osk
from oracle import tsqr as ots

from gpu_util import bits_to_signs, col, host, rel

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


# ------------------------------------------------------------------------- Omega
@pytest.mark.parametrize("n,d,seed", [(2048, 64, 0), (1000, 48, 3), (16, 16, 7), (4097, 128, 11),
                                      (262144, 512, 0), (131072, 384, 0), (65536, 256, 5)])
def test_omega_bit_exact(ctx, n, d, seed):
    bits, cols = ck.omega(ctx, n, d, seed)
    torch.cuda.synchronize()
    ck.check(ctx)
    assert np.array_equal(bits_to_signs(bits, n), oom.rademacher_signs(n, seed))
    assert np.array_equal(cols.cpu().numpy().astype(np.int64), oom.subsample_columns(n, d, seed))


# ------------------------------------------------------------------------- sketch
SKETCH_CASES = [
    # n, d, kind, ell, dim
    (2048, 64, okk.SE, 0.2, 2),
    (1000, 48, okk.MATERN52, 0.15, 3),
    (777, 272, okk.SE, 0.1, 2),
    (2085, 512, okk.SE, 0.1, 2),
    (300, 16, okk.MATERN52, 0.3, 1),
]
PREC_TOL = [("fp32", 1e-5), ("bf16", 4e-3), ("bf16x2", 3e-5), ("bf16x3", 1e-5), ("fp32_wht", 1e-5)]


@pytest.mark.parametrize("prec,tol", PREC_TOL)
@pytest.mark.parametrize("n,d,kind,ell,dim", SKETCH_CASES)
def test_sketch_matches_oracle(ctx, prec, tol, n, d, kind, ell, dim):
    pts = synth.points(n, dim, 1)
    plan = ck.Plan(n=n, d=d, dim=dim, prec=ck.PRECISIONS[prec], seed=2)
    kern = ck.Kernel(kind, ell, 1.3, 1e-4)
    Y = ck.sketch(ctx, plan, kern, torch.from_numpy(pts).cuda())
    torch.cuda.synchronize()
    ck.check(ctx)
    O = oom.omega_matrix(n, d, 2)
    Yo = osk.sketch(pts.astype(np.float64), kind, ell, 1.3, O)
    err = rel(host(Y), Yo)
    print("sketch %s n=%d d=%d err=%.3e" % (prec, n, d, err))
    assert err <= tol


@pytest.mark.parametrize("n,d,dim,kind,deriv", [
    (1025, 64, 1, okk.SE, False),         # one live entry in the second chunk
    (1024, 16, 2, okk.MATERN52, False),   # exactly one chunk; one output slot a lane
    (4100, 512, 3, okk.SE, False),        # sixteen slots a lane, a 4-entry last chunk
    (3000, 96, 3, okk.MATERN52, True),    # Matern derivative: the masked last chunk
    (2049, 48, 2, okk.SE, True),          # SE derivative: clamped distances to the padding
])
def test_fast_transform_sketch_edges(ctx, n, d, dim, kind, deriv):
    """The FP32 fast-transform sketch at the shapes its chunking and output slots make
    special, against the oracle's sketch (bar 1e-5, the FP32 Y bar), and a row range ending
    in a partial 8-row block bit-identical to the same rows of the whole sketch."""
    pts = synth.points(n, dim, 7)
    plan = ck.Plan(n=n, d=d, dim=dim, prec=ck.FP32_WHT, seed=13)
    kern = ck.Kernel(kind, 0.2, 0.9, 1e-4)
    P = torch.from_numpy(pts).cuda()
    Y = ck.sketch_dlogl(ctx, plan, kern, P) if deriv else ck.sketch(ctx, plan, kern, P)
    torch.cuda.synchronize()
    ck.check(ctx)
    Yo = osk.sketch(pts.astype(np.float64), kind, 0.2, 0.9, oom.omega_matrix(n, d, 13), derivative=deriv)
    err = rel(host(Y), Yo)
    print("fast-transform sketch n=%d d=%d dim=%d kind=%d deriv=%d: err %.3e" % (n, d, dim, kind, deriv, err))
    assert err <= 1e-5
    if not deriv:
        r0, m = 5, n - 11                 # m % 8 != 0
        Yr = ck.sketch_rows(ctx, plan, kern, r0, m, points=P)
        torch.cuda.synchronize()
        assert torch.equal(Yr, Y[r0:r0 + m])


@pytest.mark.parametrize("prec,tol", [("fp32", 1e-5), ("bf16x3", 1e-5), ("bf16", 4e-3), ("fp32_wht", 1e-5)])
@pytest.mark.parametrize("kind", [okk.SE, okk.MATERN52])
def test_derivative_sketch_matches_oracle(ctx, prec, tol, kind):
    n, d, dim = 1500, 64, 2
    pts = synth.points(n, dim, 4)
    plan = ck.Plan(n=n, d=d, dim=dim, prec=ck.PRECISIONS[prec], seed=9)
    kern = ck.Kernel(kind, 0.17, 0.8, 1e-4)
    Yd = ck.sketch_dlogl(ctx, plan, kern, torch.from_numpy(pts).cuda())
    torch.cuda.synchronize()
    O = oom.omega_matrix(n, d, 9)
    Yo = osk.sketch(pts.astype(np.float64), kind, 0.17, 0.8, O, derivative=True)
    assert rel(host(Yd), Yo) <= tol


@pytest.mark.parametrize("prec,tol", [("fp32", 1e-5), ("bf16x3", 1e-5), ("bf16x2", 3e-5), ("bf16", 4e-3),
                                      ("fp32_wht", 1e-5)])
@pytest.mark.parametrize("n,d", [(1536, 64), (1000, 272)])
def test_dense_sketch_matches_oracle(ctx, prec, tol, n, d):
    """Materialised K (the plain-method workload with K in HBM): SIMT FP32, tensor cores, or
    the fast transform over K's columns."""
    pts = synth.points(n, 3, 2).astype(np.float64)
    K = okk.kernel_matrix(pts, pts, okk.MATERN52, 0.15, 1.0)
    plan = ck.Plan(n=n, d=d, dim=3, seed=0, prec=ck.PRECISIONS[prec])
    Y = ck.sketch(ctx, plan, ck.Kernel(ck.DENSE, 0, 0, 1e-5), K=col(K))
    torch.cuda.synchronize()
    ck.check(ctx)
    Yo = osk.sketch_dense(K.astype(np.float32).astype(np.float64), oom.omega_matrix(n, d, 0))
    err = rel(host(Y), Yo)
    print("dense sketch %s n=%d d=%d err=%.3e" % (prec, n, d, err))
    assert err <= tol


# ------------------------------------------------------------------------- TSQR
TSQR_CASES = [
    # n, d, b, fp64 tree levels, fp64 leaves
    (4096, 64, 512, 1, 0),
    (4100, 64, 512, 0, 0),
    (4100, 64, 512, -1, 0),
    (3000, 48, 700, 2, 0),
    (2048, 128, 2048, 1, 0),
    (20000, 128, 1024, 2, 0),
    (9000, 512, 2048, 1, 0),
    (4100, 64, 512, 0, 1),
    (9000, 512, 2048, 1, 1),
    (3000, 48, 3000, 0, 1),
    # 64 leaves: FP64 tree levels with 32 and 16 combines, where every update CTA takes
    # several tiles (the shape of the 262144-point workload's lowest levels)
    (65536, 128, 1024, -1, 0),
]


@pytest.mark.parametrize("n,d,b,f64,leaf64", TSQR_CASES)
def test_tsqr_matches_oracle(ctx, n, d, b, f64, leaf64):
    rng = np.random.default_rng(n + d)
    Y = rng.standard_normal((n, d)).astype(np.float32)
    plan = ck.Plan(n=n, d=d, block_rows=b, seed=1, tree_fp64_levels=f64, leaf_fp64=leaf64)
    f = ck.tsqr(ctx, plan, ck.Kernel(ck.SE, 1, 1, 1e-3), col(Y))
    R = host(f.r())
    Q = host(f.q())
    torch.cuda.synchronize()
    ck.check(ctx)
    t = ots.tsqr(Y.astype(np.float64), b)
    print("tsqr n=%d d=%d b=%d: R %.3e Q %.3e" % (n, d, b, rel(R, t["R"]), rel(Q, t["Q"])))
    assert np.allclose(R, np.triu(R)) and np.all(np.diag(R) >= 0)
    tol = 1e-7 if leaf64 else 2e-5      # FP64 Householder: only Q_hat's FP32 storage rounds
    assert rel(R, t["R"]) <= (1e-12 if leaf64 else 2e-5)
    assert rel(Q, t["Q"]) <= tol
    assert np.abs(Q.T @ Q - np.eye(d)).max() <= (1e-6 if leaf64 else 1e-5)


@pytest.mark.parametrize("f64,bar", [(-1, 1e-11), (2, None), (0, None)])
def test_tree_combine_precision(ctx, f64, bar):
    """The precision of the R-tree combine alone.  Every leaf block of Y is already upper
    triangular (zero below its first d rows), so the leaves' Householder QR reflects nothing
    and hands the tree its blocks exactly; the final R's error is then the tree's own.  With
    every level combined in the FP64-class arithmetic (double-FP32, ~2^-47 per operation)
    R must match the oracle's FP64 TSQR to 1e-11; with FP32 levels it cannot (printed: the
    test shows that the bar separates the two)."""
    L, d, b = 16, 128, 512
    rng = np.random.default_rng(77)
    Y = np.zeros((L * b, d), np.float32)
    for i in range(L):
        Ri = np.triu(rng.standard_normal((d, d))) + np.diag(3.0 + np.abs(rng.standard_normal(d)))
        Y[i * b:i * b + d] = Ri.astype(np.float32)
    plan = ck.Plan(n=L * b, d=d, block_rows=b, seed=1, tree_fp64_levels=f64, leaf_fp64=0)
    f = ck.tsqr(ctx, plan, ck.Kernel(ck.SE, 1, 1, 1e-3), col(Y))
    R = host(f.r())
    torch.cuda.synchronize()
    ck.check(ctx)
    Ro = ots.tsqr(Y.astype(np.float64), b)["R"]
    err = rel(R, Ro)
    print("tree combine, %s FP64-class levels: R err %.3e" % ("all" if f64 < 0 else f64, err))
    if bar is not None:
        assert err <= bar
    else:
        assert err > 1e-9        # FP32 levels: the bar above would catch an FP32 combine


@pytest.mark.parametrize("n,d,b,f64", [(20000, 128, 1024, 1), (9000, 512, 2048, 1), (65536, 128, 1024, -1),
                                       (32768, 512, 2048, -1)])
def test_tsqr_bf16_forms_tensor_core_gemms(ctx, n, d, b, f64):
    """A BF16-form plan runs the TSQR's large GEMMs on the tensor cores (each FP32 operand as
    three BF16 terms, FP32 accumulation in TMEM).  The accumulation is coarser than FP32
    FMAs: measured R 6.3e-6, Q_hat 1.9e-5 and |Q^T Q - I| 1.0e-5 at n = 9000, d = 512, against
    9e-8, 5e-7 and 5e-7 on the CUDA cores (nine term products instead of six change nothing,
    so the dropped products are not the cause).  The bars below leave ~3x margin; they sit
    far under those forms' sketch error (BF16: ~1.5e-3)."""
    rng = np.random.default_rng(n + d)
    Y = rng.standard_normal((n, d)).astype(np.float32)
    plan = ck.Plan(n=n, d=d, block_rows=b, seed=1, prec=ck.BF16, tree_fp64_levels=f64)
    f = ck.tsqr(ctx, plan, ck.Kernel(ck.SE, 1, 1, 1e-3), col(Y))
    R = host(f.r())
    Q = host(f.q())
    torch.cuda.synchronize()
    ck.check(ctx)
    t = ots.tsqr(Y.astype(np.float64), b)
    orth = np.abs(Q.T.astype(np.float64) @ Q - np.eye(d)).max()
    print("tsqr (tensor-core GEMMs) n=%d d=%d: R %.3e Q %.3e orth %.3e" % (n, d, rel(R, t["R"]), rel(Q, t["Q"]), orth))
    assert np.allclose(R, np.triu(R)) and np.all(np.diag(R) >= 0)
    assert rel(R, t["R"]) <= 2e-5
    assert rel(Q, t["Q"]) <= 6e-5
    assert orth <= 3e-5


@pytest.mark.parametrize("n,d,b,prec", [(4096, 64, 1024, "fp32"), (4096, 512, 1024, "fp32"),
                                        (4096, 512, 1024, "bf16"), (4096, 512, 1024, "fp32_wht"),
                                        (3000, 128, 1024, "fp32_wht")])
def test_core_matches_oracle(ctx, n, d, b, prec):
    """B = Omega^T Q_hat, C' = R^T + tau B and log det K_tilde from the FP64 LUs (32-column
    panels: 16 of them at d = 512).  The BF16 and fast-transform forms apply the
    Walsh-Hadamard Omega to Q_hat's columns by the fast transform in FP32 (n = 3000: a
    zero-padded last chunk); the BF16 form runs its TSQR's GEMMs on the tensor cores (~1e-5)."""
    tau = 1e-3
    rng = np.random.default_rng(5)
    Y = rng.standard_normal((n, d)).astype(np.float32)
    plan = ck.Plan(n=n, d=d, block_rows=b, seed=4, prec=ck.PRECISIONS[prec])
    f = ck.tsqr(ctx, plan, ck.Kernel(ck.SE, 1, 1, tau), col(Y))
    B, C, logdet = f.core()
    O = oom.omega_matrix(n, d, 4)
    fo = olr.factorise(Y.astype(np.float64), O, tau, b)
    tol = 6e-5 if prec == "bf16" else 2e-5
    print("core n=%d d=%d %s: B %.2e C' %.2e logdet %.2e" % (n, d, prec, rel(host(B), fo.B), rel(host(C), fo.Cp),
                                                            abs(logdet - fo.logdet()) / abs(fo.logdet())))
    assert rel(host(B), fo.B) <= tol
    assert rel(host(C), fo.Cp) <= tol
    assert abs(logdet - fo.logdet()) <= 1e-6 * abs(fo.logdet())


# ------------------------------------------------------------------------- solve
@pytest.mark.parametrize("refine,leaf64,tol", [(0, 1, 1e-6), (1, 1, 1e-6), (1, 0, 5e-4)])
def test_solve_matches_oracle_given_same_sketch(ctx, refine, leaf64, tol):
    """Same FP32 sketch on both sides.  With FP64 Householder only FP32 storage of Q_hat and
    the FP32 solve round; FP32 Householder on this sketch (kappa(Y) ~ 1.5e5) is limited to
    ~kappa(Y) u_32 ~ 3e-4, which is what a textbook FP32 Householder QR gives as well."""
    cfg = synth.CONFIGS["c1_plain_n2048"]
    n, d, b, tau = cfg["n"], cfg["d"], cfg["block_rows"], cfg["tau"]
    pts = synth.points(n, 2, 0).astype(np.float64)
    O = oom.omega_matrix(n, d, 0)
    Y = osk.sketch(pts, okk.SE, cfg["ell"], 1.0, O).astype(np.float32)   # common input
    A = synth.rhs(n, 4, 0)
    plan = ck.Plan(n=n, d=d, block_rows=b, seed=0, refine_steps=refine, leaf_fp64=leaf64)
    f = ck.tsqr(ctx, plan, ck.Kernel(ck.SE, cfg["ell"], 1.0, tau), col(Y))
    X = host(ck.solve(ctx, f, col(A)))
    fo = olr.factorise(Y.astype(np.float64), O, tau, b)
    Xo = olr.solve_refined(fo, A.astype(np.float64), 1)
    err = rel(X, Xo)
    print("solve refine=%d leaf64=%d err=%.3e" % (refine, leaf64, err))
    assert err <= tol


@pytest.mark.parametrize("leaf64,tol", [(1, 1e-6), (0, 1e-5)])
def test_solve_at_d512_given_same_sketch(ctx, leaf64, tol):
    """d = 512 (16 LU panels, the widest triangular solves and refinement shapes) on a sketch
    whose kappa(Y) is about 1e2 (SE l = 0.03 on 4096 points), the same FP32 Y on both sides."""
    n, d, b, tau, ell = 4096, 512, 1024, 1e-6, 0.03
    pts = synth.points(n, 2, 1).astype(np.float64)
    O = oom.omega_matrix(n, d, 6)
    Y = osk.sketch(pts, okk.SE, ell, 1.0, O).astype(np.float32)
    A = synth.rhs(n, 8, 2)
    plan = ck.Plan(n=n, d=d, block_rows=b, seed=6, refine_steps=1, leaf_fp64=leaf64)
    f = ck.tsqr(ctx, plan, ck.Kernel(ck.SE, ell, 1.0, tau), col(Y))
    X = host(ck.solve(ctx, f, col(A)))
    ck.check(ctx)
    fo = olr.factorise(Y.astype(np.float64), O, tau, b)
    Xo = olr.solve_refined(fo, A.astype(np.float64), 1)
    err = rel(X, Xo)
    print("solve d=512 leaf64=%d err=%.3e" % (leaf64, err))
    assert err <= tol


def test_kinv_a_end_to_end_c1(ctx):
    """The plain-method workload: n = 2048, SE l = 0.2, nugget 1e-6, d = 64, FP32."""
    cfg = synth.CONFIGS["c1_plain_n2048"]
    n, d = cfg["n"], cfg["d"]
    pts = synth.points(n, 2, 0)
    A = synth.rhs(n, cfg["m"], 0)
    plan = ck.Plan(n=n, d=d, dim=2, block_rows=cfg["block_rows"], prec=ck.FP32, seed=0, refine_steps=1,
                   leaf_fp64=cfg["leaf_fp64"])
    kern = ck.Kernel(ck.SE, cfg["ell"], 1.0, cfg["tau"])
    X = ck.kinv_a(ctx, plan, kern, torch.from_numpy(pts).cuda(), col(A))
    torch.cuda.synchronize()
    Xo, _, _ = olr.kinv_a(pts.astype(np.float64), A.astype(np.float64), okk.SE, cfg["ell"], 1.0, cfg["tau"], d, 0,
                          cfg["block_rows"], 1)
    err = rel(host(X), Xo)
    print("c1 end-to-end K^-1 A error %.3e" % err)
    assert err <= 1e-4


def test_kinv_a_host_buffers(ctx):
    n, d = 1024, 32
    pts = synth.points(n, 2, 3)
    A = synth.rhs(n, 2, 3)
    plan = ck.Plan(n=n, d=d, dim=2, block_rows=256, seed=1)
    kern = ck.Kernel(ck.SE, 0.25, 1.0, 1e-4)
    Xh = torch.empty((2, n), dtype=torch.float32).t()
    ck.kinv_a(ctx, plan, kern, torch.from_numpy(pts), torch.from_numpy(np.asfortranarray(A)), Xh)
    Xd = ck.kinv_a(ctx, plan, kern, torch.from_numpy(pts).cuda(), col(A))
    torch.cuda.synchronize()
    assert rel(Xh.numpy(), host(Xd)) <= 1e-6


# ------------------------------------------------------------------------- NLL
def _oracle_nll_grad(pts, y, kind, ell, var, tau, d, seed, b, round_mode=None):
    """Oracle NLL and gradient.  round_mode 'Y' rounds the two sketches to FP32, 'K' rounds
    the kernel matrices to FP32 before the (exact) sketch: the floors of a method that stores
    the sketch, or the kernel entries, in FP32."""
    pts = pts.astype(np.float64)
    O = oom.omega_matrix(len(pts), d, seed)
    if round_mode == "K":
        r32 = lambda M: M.astype(np.float32).astype(np.float64)
        Y = r32(r32(okk.kernel_matrix(pts, pts, kind, ell, var)) @ O)
        Yd = r32(r32(okk.dkernel_matrix(pts, pts, kind, ell, var)) @ O)
    else:
        Y = osk.sketch(pts, kind, ell, var, O)
        Yd = osk.sketch(pts, kind, ell, var, O, derivative=True)
    if round_mode == "Y":
        Y = Y.astype(np.float32).astype(np.float64)
        Yd = Yd.astype(np.float32).astype(np.float64)
    f = olr.factorise(Y, O, tau, b)
    v, a = olr.nll(f, y.astype(np.float64), 1)
    g, _ = olr.grad(f, y, Y, Yd, a)
    return v, g


@pytest.mark.parametrize("kind", [okk.SE, okk.MATERN52])
def test_nll_grad_matches_oracle(ctx, kind):
    """Tolerance: 3x the floor set by FP32 kernel entries and FP32 sketches (measured by the
    oracle on rounded inputs), and never tighter than 1e-6 (NLL) / 1e-4 (gradient) relative:
    the gradient is assembled from d x d inner products of FP32-stored Q_hat data whose terms
    cancel, so it carries a few 1e-5 of relative rounding."""
    n, d, tau, ell, var = 1024, 48, 1e-3, 0.25, 1.2
    pts = synth.points(n, 2, 5)
    y = synth.gp_targets(pts, 0.2, 1.0, tau, seed=5)
    plan = ck.Plan(n=n, d=d, dim=2, block_rows=256, prec=ck.FP32, seed=3, refine_steps=1, leaf_fp64=1)
    kern = ck.Kernel(kind, ell, var, tau)
    val, g = ck.nll_grad(ctx, plan, kern, torch.from_numpy(pts).cuda(), torch.from_numpy(y).cuda())
    vo, go = _oracle_nll_grad(pts, y, kind, ell, var, tau, d, 3, 256)
    floors_v, floors_g = [], []
    for mode in ("Y", "K"):
        vf, gf = _oracle_nll_grad(pts, y, kind, ell, var, tau, d, 3, 256, mode)
        floors_v.append(abs(vf - vo) / abs(vo))
        floors_g.append(np.abs(gf - go) / np.abs(go))
    tol_v = max(1e-6, 3 * max(floors_v))
    tol_g = np.maximum(1e-4, 3 * np.maximum(*floors_g))
    print("nll %.10g vs %.10g (floor %.2e); grad %s vs %s (floor %s)" % (val, vo, tol_v / 3, g, go, tol_g / 3))
    assert abs(val - vo) <= tol_v * abs(vo)
    assert np.all(np.abs(np.array(g) - go) <= tol_g * np.abs(go))


def test_invalid_arguments_are_rejected(ctx):
    pts = torch.zeros((64, 2), device="cuda")
    with pytest.raises(ck.CKInvError) as e:
        ck.sketch(ctx, ck.Plan(n=64, d=24, dim=2), ck.Kernel(), pts)          # d % 16 != 0
    assert e.value.status == ck.EINVAL
    with pytest.raises(ck.CKInvError) as e:
        ck.sketch(ctx, ck.Plan(n=8, d=16, dim=2), ck.Kernel(), pts)           # n < d
    assert e.value.status == ck.EINVAL
    with pytest.raises(ck.CKInvError) as e:
        ck.sketch(ctx, ck.Plan(n=64, d=16, dim=4), ck.Kernel(), pts)          # dim
    assert e.value.status == ck.EINVAL
    with pytest.raises(ck.CKInvError) as e:
        ck.sketch(ctx, ck.Plan(n=64, d=16, dim=2), ck.Kernel(ck.SE, 0.1, 1.0, 0.0), pts)  # nugget
    assert e.value.status == ck.EINVAL
