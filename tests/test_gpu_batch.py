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
