"""Batched likelihood (all problems captured into one CUDA graph, launched once) and the
TSQR leaf-height autotuner.

The batched entry must give each problem the value the single-problem entry gives; the
single-problem entry is pinned to the oracle in test_gpu_parity.py.  Every reduction in
the library sums in a fixed order (split-K partials and row-split partials are folded in
split order, dot products run in one block), so a problem gives the same bits whether it
runs alone or inside the batched graph, where it shares the GPU with other problems.  The
bar is therefore 1e-12 relative: reproducibility, not rounding, is what is tested.  (Some
members of the 64-problem workload are numerically rank deficient at FP32/BF16 precision
(large lengthscale, d = 256, n ~ 5000), and their gradient depends on rounding-level
detail; without fixed-order reductions two identical calls disagreed there by up to 100 %.)
"""
import time

import numpy as np
import pytest
import torch

import synth
from oracle import kernels as okk
from oracle import lowrank as olr
from oracle import omega as oom

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


def _problems(specs, auto_every=0, prec=None):
    plans, kerns, pts, ys = [], [], [], []
    for i, s in enumerate(specs):
        block_rows = 0 if (auto_every and i % auto_every == 0) else s["block_rows"]
        plans.append(ck.Plan(n=s["n"], d=s["d"], dim=s["dim"], block_rows=block_rows, seed=1000 + s["seed"],
                             prec=ck.BF16X3 if prec is None else prec))
        kerns.append(ck.Kernel(s["kind"], s["ell"], s["var"], s["tau"]))
        p = synth.points(s["n"], s["dim"], s["seed"])
        pts.append(torch.from_numpy(p).cuda())
        ys.append(torch.from_numpy(synth.gp_targets(p, 0.2, 1.0, s["tau"], seed=s["seed"])).cuda())
    return plans, kerns, pts, ys


def _compare(vb, gb, vs, gs):
    assert abs(vb - vs) <= 1e-12 * abs(vs), (vb, vs)
    gb, gs = np.array(gb), np.array(gs)
    assert np.all(np.abs(gb - gs) <= 1e-12 * np.abs(gs)), (gb, gs)


def test_single_calls_are_reproducible(ctx):
    specs = synth.batch_specs(3, seed=3, n_lo=4096, n_hi=8192)
    plans, kerns, pts, ys = _problems(specs)
    for p in range(len(plans)):
        v1, g1 = ck.nll_grad(ctx, plans[p], kerns[p], pts[p], ys[p])
        v2, g2 = ck.nll_grad(ctx, plans[p], kerns[p], pts[p], ys[p])
        assert v1 == v2 and list(g1) == list(g2)


def test_batched_graph_matches_single_calls(ctx):
    specs = synth.batch_specs(10, seed=1, n_lo=4096, n_hi=20000)
    plans, kerns, pts, ys = _problems(specs, auto_every=2)   # half the leaf heights autotuned
    vb, gb = ck.nll_grad_batched(ctx, plans, kerns, pts, ys)
    for p in range(len(plans)):
        vs, gs = ck.nll_grad(ctx, plans[p], kerns[p], pts[p], ys[p])
        _compare(vb[p], gb[p], vs, gs)


def test_batched_full_workload_64_problems(ctx):
    """The 64-problem workload (n log-uniform in [4096, 65536], D in {2, 3}, SE and
    Matern-5/2, d in {64, 128, 256}) in one graph against 64 single calls."""
    specs = synth.batch_specs(64, seed=0)
    plans, kerns, pts, ys = _problems(specs, prec=ck.BF16)
    ck.nll_grad_batched(ctx, plans[:2], kerns[:2], pts[:2], ys[:2])   # warm-up
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    vb, gb = ck.nll_grad_batched(ctx, plans, kerns, pts, ys)
    t_batch = time.perf_counter() - t0
    t0 = time.perf_counter()
    single = [ck.nll_grad(ctx, plans[p], kerns[p], pts[p], ys[p]) for p in range(len(plans))]
    t_single = time.perf_counter() - t0
    print("64 problems: one graph %.1f ms, 64 single calls %.1f ms" % (1e3 * t_batch, 1e3 * t_single))
    for p in range(len(plans)):
        _compare(vb[p], gb[p], *single[p])


def test_batched_rejects_a_bad_problem(ctx):
    specs = synth.batch_specs(3, seed=2, n_lo=4096, n_hi=8192)
    plans, kerns, pts, ys = _problems(specs)
    plans[1].d = 24                                    # d % 16 != 0
    with pytest.raises(ck.CKInvError) as e:
        ck.nll_grad_batched(ctx, plans, kerns, pts, ys)
    assert e.value.status == ck.EINVAL


def test_autotune_picks_a_candidate_and_is_used(ctx):
    n, d = 32768, 128
    plan = ck.Plan(n=n, d=d, dim=2, block_rows=0, seed=7, prec=ck.BF16)
    b = ck.autotune(ctx, plan)
    assert b in (256, 512, 1024, 2048, 4096) and b >= d and 2 * b <= n
    pts = torch.from_numpy(synth.points(n, 2, 7)).cuda()
    A = torch.from_numpy(np.ascontiguousarray(synth.rhs(n, 4, 7).T)).cuda().t()
    kern = ck.Kernel(ck.SE, 0.15, 1.0, 1e-4)
    X_auto = ck.kinv_a(ctx, plan, kern, pts, A)
    plan_b = ck.Plan(n=n, d=d, dim=2, block_rows=b, seed=7, prec=ck.BF16)
    X_b = ck.kinv_a(ctx, plan_b, kern, pts, A)
    torch.cuda.synchronize()
    err = float((X_auto - X_b).norm() / X_b.norm())
    assert err <= 1e-5, err


def _oracle_nll_grad(pts, y, kind, ell, var, tau, d, seed, b, round32=False):
    """Oracle NLL and gradient; round32 rounds the kernel and derivative entries to FP32
    before the (exact) sketch, and the sketches, Q_hat and alpha = K_tilde^-1 y after it: the
    floor of a method that carries entries to FP32 precision and stores those arrays in FP32."""
    pts = pts.astype(np.float64)
    O = oom.omega_matrix(len(pts), d, seed)
    K = okk.kernel_matrix(pts, pts, kind, ell, var)
    Kd = okk.dkernel_matrix(pts, pts, kind, ell, var)
    r32 = (lambda M: np.asarray(M, dtype=np.float32).astype(np.float64)) if round32 else (lambda M: M)
    Y, Yd = r32(r32(K) @ O), r32(r32(Kd) @ O)
    f = olr.factorise(Y, O, tau, b)
    if round32:
        f = olr.Factor(r32(f.Q), f.R, O, tau)
    v, a = olr.nll(f, y.astype(np.float64), 1)
    g, _ = olr.grad(f, y, Y, Yd, r32(a))
    return v, g


def test_batched_problems_against_the_oracle(ctx):
    """Eight problems of uneven size, kernel, dimension and width in one graph, each against
    the FP64 oracle (not only against single calls).  Members alternate between the FP32
    form and the three-term tensor-core form (both carry kernel entries to FP32 precision),
    FP64 leaves, nugget 1e-2 (at 1e-3 storing alpha in FP32 alone moves one member's
    length-scale derivative by 1e-3).  Bar: three times the floor of FP32 kernel entries with
    the sketches, Q_hat and alpha stored in FP32, and never tighter than 1e-5 (NLL) and 1e-3
    (gradient): the library forms the gradient's d x d reductions from FP32 products summed
    in FP64 per 256 rows, measured at up to 1.2e-6 (NLL) and 1.6e-4 (gradient) on these
    problems, whose kappa(Y) reaches 1e4."""
    rng = np.random.default_rng(11)
    plans, kerns, pts, ys, host_in = [], [], [], [], []
    for p in range(8):
        n = int(rng.integers(1024, 3001))
        dim = 2 + p % 2
        kind = ck.MATERN52 if p % 3 == 2 else ck.SE
        ell = float(rng.uniform(0.18, 0.3))
        d = [32, 48, 64][p % 3]
        b = 512 if n >= 1024 else n
        x = synth.points(n, dim, 100 + p)
        y = synth.gp_targets(x, 0.2, 1.0, 1e-2, seed=100 + p)
        plans.append(ck.Plan(n=n, d=d, dim=dim, block_rows=b, seed=200 + p, refine_steps=1, leaf_fp64=1,
                             prec=ck.FP32 if p % 2 == 0 else ck.BF16X3))
        kerns.append(ck.Kernel(kind, ell, 1.1, 1e-2))
        pts.append(torch.from_numpy(x).cuda())
        ys.append(torch.from_numpy(y).cuda())
        host_in.append((x, y, kind, ell, d, b))
    vb, gb = ck.nll_grad_batched(ctx, plans, kerns, pts, ys)
    for p, (x, y, kind, ell, d, b) in enumerate(host_in):
        vo, go = _oracle_nll_grad(x, y, kind, ell, 1.1, 1e-2, d, 200 + p, b)
        vf, gf = _oracle_nll_grad(x, y, kind, ell, 1.1, 1e-2, d, 200 + p, b, round32=True)
        tv = max(1e-5, 3 * abs(vf - vo) / abs(vo))
        tg = np.maximum(1e-3, 3 * np.abs(gf - go) / np.abs(go))
        ev = abs(vb[p] - vo) / abs(vo)
        eg = np.abs(np.array(gb[p]) - go) / np.abs(go)
        print("problem %d (n=%d d=%d): NLL err %.2e (bar %.2e), grad err %s (bar %s)" % (p, len(x), d, ev, tv, eg, tg))
        assert ev <= tv
        assert np.all(eg <= tg)


def test_batched_graph_is_kept_and_relaunched(ctx):
    """A second call with the same problems (descriptors and input pointers) relaunches the
    kept graph: the same values, from the inputs' current contents."""
    specs = synth.batch_specs(4, seed=5, n_lo=4096, n_hi=8192)
    plans, kerns, pts, ys = _problems(specs)
    v1, g1 = ck.nll_grad_batched(ctx, plans, kerns, pts, ys)
    t0 = time.perf_counter()
    v2, g2 = ck.nll_grad_batched(ctx, plans, kerns, pts, ys)
    t_again = time.perf_counter() - t0
    assert v1 == v2 and g1 == g2
    ys[2].mul_(1.5)                                    # same pointer, new contents
    v3, g3 = ck.nll_grad_batched(ctx, plans, kerns, pts, ys)
    vs, gs = ck.nll_grad(ctx, plans[2], kerns[2], pts[2], ys[2])
    _compare(v3[2], g3[2], vs, gs)
    assert v3[0] == v1[0] and v3[2] != v1[2]
    print("relaunch of the kept graph: %.1f ms" % (1e3 * t_again))
