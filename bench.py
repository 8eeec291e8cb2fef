"""Benchmark of the low-rank K^-1 A path on GB300.

One step = one full solve of the workload: draw Omega (fresh seed each step), fused
sketch Y = K0 Omega, blocked TSQR with the FP64 core, low-rank solve of the n x m
right-hand side with one FP64 refinement step.  Default workload: the precision form
n = 262144 points in [0,1]^2, squared-exponential l = 0.1, nugget 1e-6, d = 512, m = 32,
BF16 sketch contraction (FP32 accumulation), FP32 Householder, FP64 tree combine and core.

Prints one JSON line (rank 0).  `--impl reference` times the FP64 CPU oracle instead on a
bounded sample of the same workload.
"""
import argparse
import json
import math
import os
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

import synth  # noqa: E402

METRIC = "low-rank K^-1A solves/s & TFLOP/s vs peak, n=262k d=512; BF16-refined vs FP32"
PEAKS_FALLBACK = {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0}


def load_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as fh:
            return json.load(fh), "measured"
    return dict(PEAKS_FALLBACK), "fallback"


KERNEL_NAMES = {0: "squared-exponential", 1: "matern-5/2"}


def measured_traffic(workload):
    """DRAM bytes (read + write) of one sketch launch from the committed ncu capture, if the
    capture was of this workload and the kernel source has not changed since; else None."""
    import hashlib
    if workload != "c3_bf16_n262144":
        return None
    here = os.path.dirname(os.path.abspath(__file__))
    try:
        with open(os.path.join(here, "profiles", "sketch_tc_bf16_pair_n262144_d512_traffic.json")) as fh:
            rec = json.load(fh)
        with open(os.path.join(here, rec["source"]), "rb") as fh:
            sha = hashlib.sha1(fh.read()).hexdigest()
    except (OSError, ValueError, KeyError):
        return None
    if sha != rec["source_sha1"]:
        return None
    return rec["dram_bytes_read"] + rec["dram_bytes_write"]


def workload_config(name):
    cfg = dict(synth.CONFIGS[name])
    cfg["workload"] = name
    return cfg


class ClockSampler:
    """nvidia-smi samples of SM clock and throttle reasons while the timed region runs."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), "--query-gpu=" + self.Q,
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except Exception:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": float(np.median(sm)) if sm else None,
                "sm_max_mhz": float(max(smax)) if smax else None,
                "samples": len(sm), "reasons": sorted(reasons)}


def sampled_sketch_error(ck, Y, pts, cfg, seed, rows):
    """Relative error of sampled rows of the GPU sketch against the FP64 oracle."""
    from oracle import omega as oom
    from oracle import sketch as osk
    n, d = cfg["n"], cfg["d"]
    O = oom.omega_matrix(n, d, seed)
    Yo = osk.sketch_rows(pts.astype(np.float64), rows, cfg["kind"], cfg["ell"], cfg["var"], O)
    Yg = Y[rows].double().cpu().numpy()
    return float(np.linalg.norm(Yg - Yo) / np.linalg.norm(Yo))


def job_rate(local_ms, steps, world, dist=None, device="cpu"):
    """Whole-job throughput of `steps` steps on each of `world` ranks: the slowest rank's
    time (max over ranks, behind a barrier) sets it.  Returns (units per second, ms per step
    of the slowest rank).  `dist` is torch.distributed (None for one process); `device` is
    where the reduction tensor lives (the rank's GPU under NCCL, "cpu" under gloo)."""
    total_ms = float(local_ms)
    if dist is not None and world > 1:
        import torch
        t = torch.tensor([total_ms], dtype=torch.float64, device=device)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        total_ms = float(t.item())
        dist.barrier()
    return world * steps / (total_ms / 1e3), total_ms / steps


def oracle_sample_time(cfg, rows_sample, seed):
    """FP64 CPU oracle on a bounded sample: Omega (built once per solve) and the sketch rows
    [0, rows_sample) of the workload.  Returns (seconds, extrapolated seconds per solve:
    Omega's time plus the rows' time scaled to all n rows)."""
    from oracle import omega as oom
    from oracle import sketch as osk
    n, d = cfg["n"], cfg["d"]
    pts = synth.points(n, cfg["dim"], 0).astype(np.float64)
    t0 = time.perf_counter()
    O = oom.omega_matrix(n, d, seed)
    t1 = time.perf_counter()
    for r0 in range(0, rows_sample, 256):         # 256 rows of K0 (0.5 GB at n = 262144) at a time
        osk.sketch_rows(pts, np.arange(r0, min(rows_sample, r0 + 256)), cfg["kind"], cfg["ell"], cfg["var"], O)
    t2 = time.perf_counter()
    return t2 - t0, (t1 - t0) + (t2 - t1) * n / rows_sample


def cpu_threads():
    try:
        import threadpoolctl
        info = threadpoolctl.threadpool_info()
        return max([i.get("num_threads", 1) for i in info] + [1])
    except Exception:
        return os.cpu_count() or 1


def run_reference(args, rank, world):
    cfg = workload_config(args.workload)
    if rank != 0:
        return
    rows = max(256, args.ref_rows // 4)            # a quarter of the bench's sample per step
    for _ in range(args.warmup):
        oracle_sample_time(cfg, 256, 0)
    per = []
    for s in range(args.steps):
        _, full = oracle_sample_time(cfg, rows, s)
        per.append(full)
    sps = 1.0 / float(np.mean(per))
    cores = cpu_threads()
    line = {"impl": "reference", "metric": METRIC, "value": sps, "unit": "solves/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * float(np.mean(per)),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic",
            "config": {"workload": cfg["workload"], "n": cfg["n"], "d": cfg["d"], "m": cfg["m"],
                       "kernel": KERNEL_NAMES[cfg["kind"]], "lengthscale": cfg["ell"], "nugget": cfg["tau"]},
            "cpu_baseline": {"value": sps, "unit": "solves/s", "cores": cores, "kind": "oracle",
                             "sample": "FP64 oracle per step: Omega, then sketch rows 0..%d of %d "
                                       "extrapolated to all rows; QR and solve not included"
                                       % (rows, cfg["n"])},
            "e2e": {"value": sps, "unit": "solves/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def run_extras(ck, ctx, dev, reps=3):
    """The other two workloads, timed once warm: the Gaussian likelihood and its gradient at
    n = 131072, d = 384 (one ckinv_nll_grad call), and the 64-problem batch (one
    ckinv_nll_grad_batched call: graph capture, instantiation and launch)."""
    import torch
    out = {}
    cfg = workload_config("c4_nll_n131072")
    n, d, dim = cfg["n"], cfg["d"], cfg["dim"]
    pts_np = synth.points(n, dim, seed=0)
    y_np = synth.gp_targets(pts_np, cfg["ell"], cfg["var"], cfg["tau"], seed=0)
    pts = torch.from_numpy(pts_np).to(dev)
    y = torch.from_numpy(y_np).to(dev)
    plan = ck.Plan(n=n, d=d, dim=dim, block_rows=cfg["block_rows"], prec=ck.BF16, seed=0, refine_steps=1,
                   tree_fp64_levels=-1)
    kern = ck.Kernel(cfg["kind"], cfg["ell"], cfg["var"], cfg["tau"])
    ck.nll_grad(ctx, plan, kern, pts, y)
    times = []
    for _ in range(reps):
        t0 = time.perf_counter()
        val, g = ck.nll_grad(ctx, plan, kern, pts, y)
        times.append(time.perf_counter() - t0)
    t = float(np.median(times))
    out["likelihood"] = {"workload": "c4_nll_n131072", "n": n, "d": d, "prec": "bf16",
                         "ms_per_eval": 1e3 * t, "evals_per_s": 1.0 / t, "nll": val, "grad": g,
                         "timing": "host wall clock around the call (it returns host scalars), median of %d" % reps}
    specs = synth.batch_specs(64, seed=0)
    plans, kerns, P, Ys = [], [], [], []
    for sp in specs:
        plans.append(ck.Plan(n=sp["n"], d=sp["d"], dim=sp["dim"], block_rows=sp["block_rows"], prec=ck.BF16,
                             seed=1000 + sp["seed"]))
        kerns.append(ck.Kernel(sp["kind"], sp["ell"], sp["var"], sp["tau"]))
        p_np = synth.points(sp["n"], sp["dim"], sp["seed"])
        P.append(torch.from_numpy(p_np).to(dev))
        Ys.append(torch.from_numpy(synth.gp_targets(p_np, 0.2, 1.0, sp["tau"], seed=sp["seed"])).to(dev))
    ck.nll_grad_batched(ctx, plans, kerns, P, Ys)
    torch.cuda.synchronize()
    times = []
    for _ in range(2):
        t0 = time.perf_counter()
        ck.nll_grad_batched(ctx, plans, kerns, P, Ys)
        times.append(time.perf_counter() - t0)
    tb = float(min(times))
    out["batched"] = {"workload": "c5_batch64", "problems": len(specs), "ms_per_batch": 1e3 * tb,
                      "problems_per_s": len(specs) / tb, "prec": "bf16",
                      "timing": "host wall clock around one ckinv_nll_grad_batched call (capture, instantiate, "
                                "launch, read back), best of 2"}
    return out


def run_ours(args, rank, world, local_rank):
    import torch
    import __graft_entry__
    __graft_entry__.build()
    from paper_1312_1869_gb300 import ckinv as ck

    torch.cuda.set_device(local_rank)
    dev = torch.device("cuda", local_rank)
    cfg = workload_config(args.workload)
    n, d, m, dim = cfg["n"], cfg["d"], cfg["m"], cfg["dim"]
    ctx = ck.Context(local_rank)
    prec = ck.PRECISIONS[args.prec]
    plan = ck.Plan(n=n, d=d, dim=dim, block_rows=cfg["block_rows"], prec=prec, seed=0,
                   refine_steps=args.refine, tree_fp64_levels=args.fp64_levels, leaf_fp64=0)
    kern = ck.Kernel(cfg["kind"], cfg["ell"], cfg["var"], cfg["tau"])
    pts_np = synth.points(n, dim, seed=rank)
    A_np = synth.rhs(n, m, seed=rank)
    pts = torch.from_numpy(pts_np).to(dev)
    A = torch.from_numpy(np.ascontiguousarray(A_np.T)).to(dev).t()
    Y = ck.colmajor(n, d, device=dev)
    X = ck.colmajor(n, m, device=dev)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)   # > L2 (129 MB)
    stream = torch.cuda.current_stream(dev)

    def step(i, ev=None):
        plan.seed = 1000 * rank + i        # a fresh Omega every step
        if ev:
            ev[0].record(stream)
        ck.sketch(ctx, plan, kern, pts, Y=Y)
        if ev:
            ev[1].record(stream)
        f = ck.tsqr(ctx, plan, kern, Y)
        ck.solve(ctx, f, A, X)
        f.free()

    for i in range(args.warmup):
        step(i)
    torch.cuda.synchronize()
    ck.check(ctx)

    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.barrier()
    torch.cuda.synchronize()
    clocks = ClockSampler(local_rank)
    clocks.start()
    launches0 = ck.kernel_launches()
    step_ms, sketch_ms = [], []
    for i in range(args.steps):
        flush.zero_()                      # evict L2 between steps
        e0, e1, e2, e3 = [torch.cuda.Event(enable_timing=True) for _ in range(4)]
        e0.record(stream)
        step(args.warmup + i, (e1, e2))
        e3.record(stream)
        e3.synchronize()
        step_ms.append(e0.elapsed_time(e3))
        sketch_ms.append(e1.elapsed_time(e2))
    torch.cuda.synchronize()
    launches = (ck.kernel_launches() - launches0) // max(1, args.steps)
    clk = clocks.stop()
    value, ms_step = job_rate(float(np.sum(step_ms)), args.steps, world, dist, dev)
    ck.check(ctx)

    # accuracy of the sketch on sampled rows (a fresh sketch: TSQR overwrites Y)
    y_err = None
    if rank == 0:
        plan.seed = 4242
        ck.sketch(ctx, plan, kern, pts, Y=Y)
        torch.cuda.synchronize()
        rows = np.linspace(0, n - 1, 48).astype(np.int64)
        y_err = sampled_sketch_error(ck, Y, pts_np, cfg, plan.seed, rows)

    # end to end through the one-call C ABI with host (pinned) buffers
    pts_h = torch.from_numpy(pts_np).pin_memory()
    A_h = torch.from_numpy(np.ascontiguousarray(A_np.T)).pin_memory().t()
    X_h = torch.empty((m, n), dtype=torch.float32).pin_memory().t()
    e2e_steps = max(1, min(args.steps, 3))
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for i in range(e2e_steps):
        plan.seed = 777 + i
        ck.kinv_a(ctx, plan, kern, pts_h, A_h, X_h)
    torch.cuda.synchronize()
    e2e_value, _ = job_rate(1e3 * (time.perf_counter() - t0), e2e_steps, world, dist, dev)
    h2d = pts_np.nbytes + A_np.nbytes
    d2h = X_h.numel() * 4

    peaks, src = load_peaks()
    traffic = measured_traffic(cfg["workload"])
    flops = 2.0 * n * n * d
    sk_s = float(np.mean(sketch_ms)) / 1e3
    achieved = flops / sk_s / 1e12
    peak = float(peaks.get("bf16_tflops_sustained", PEAKS_FALLBACK["bf16_tflops_sustained"]))
    roof = {"bound": "tensor", "kernel": "k_sketch_tc", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
            "frac": achieved / peak, "peak_source": src + " bf16 sustained", "traffic": traffic,
            "algorithmic_flops_per_launch": flops, "ms_per_launch": sk_s * 1e3}

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        dt, full = oracle_sample_time(cfg, args.ref_rows, 0)
        cpu = {"value": 1.0 / full, "unit": "solves/s", "cores": cpu_threads(), "kind": "oracle",
               "sample": "FP64 oracle: Omega, then sketch rows 0..%d of %d (%.1f s in all), the rows' time "
                         "extrapolated to all rows; QR and solve not included" % (args.ref_rows, n, dt)}

    forms = None
    if rank == 0 and not args.no_forms:
        # the other precision forms of the same solve (best of two, after one untimed run), and
        # the BF16 form with an FP32 tree combine for comparison
        forms = {"bf16": {"solves_per_s": value / world, "tree_fp64_levels": args.fp64_levels}}
        for name, prec, lv in [("bf16x2", "bf16x2", args.fp64_levels), ("bf16x3", "bf16x3", args.fp64_levels),
                               ("fp32", "fp32", args.fp64_levels), ("bf16_fp32_tree", args.prec, 0)]:
            plan2 = ck.Plan(n=n, d=d, dim=dim, block_rows=cfg["block_rows"], prec=ck.PRECISIONS[prec], seed=5,
                            refine_steps=args.refine, tree_fp64_levels=lv)
            best = None
            for rep_i in range(3):
                flush.zero_()
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                ck.sketch(ctx, plan2, kern, pts, Y=Y)
                f = ck.tsqr(ctx, plan2, kern, Y)
                ck.solve(ctx, f, A, X)
                f.free()
                e1.record(stream)
                e1.synchronize()
                if rep_i > 0:
                    t = e0.elapsed_time(e1)
                    best = t if best is None else min(best, t)
            forms[name] = {"solves_per_s": 1e3 / best, "tree_fp64_levels": lv}
        ck.check(ctx)

    extras = {}
    if rank == 0 and not args.no_extras:
        extras = run_extras(ck, ctx, dev)

    if rank == 0:
        line = {"metric": METRIC, "value": value, "unit": "solves/s", "n_gpus": world, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": ms_step, "higher_is_better": True, "scaling": "weak",
                "vs_baseline": None, "dtype": args.prec, "data": "synthetic",
                "config": {"workload": cfg["workload"], "n": n, "d": d, "m": m, "dim": dim,
                           "kernel": KERNEL_NAMES[cfg["kind"]], "lengthscale": cfg["ell"], "nugget": cfg["tau"],
                           "block_rows": cfg["block_rows"], "refine_steps": args.refine,
                           "tree_fp64_levels": args.fp64_levels, "parallelism": "replicas" if world > 1 else "1gpu",
                           "l2": "flushed between steps (256 MB write); Y and Q_hat (537 MB each) exceed L2"},
                "tflops": achieved, "sketch_ms": sk_s * 1e3, "sketch_rel_err_sampled": y_err,
                "kernel_evals_per_s": float(n) * float(n) / sk_s,
                "roofline": roof, "cpu_baseline": cpu,
                "e2e": {"value": e2e_value, "unit": "solves/s", "h2d_bytes_per_step": h2d,
                        "d2h_bytes_per_step": d2h},
                "gpu_launches": int(launches), "clocks": clk}
        if forms is not None:
            line["forms"] = forms
        line.update(extras)
        print(json.dumps(line), flush=True)
    ctx.close()


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="c3_bf16_n262144")
    ap.add_argument("--prec", default="bf16", choices=["fp32", "bf16", "bf16x2", "bf16x3"])
    ap.add_argument("--refine", type=int, default=1)
    ap.add_argument("--fp64-levels", type=int, default=-1, help="tree levels combined in FP64 (-1: all)")
    ap.add_argument("--ref-rows", type=int, default=2048, help="sketch rows in the oracle's timed sample")
    ap.add_argument("--no-forms", action="store_true", help="skip timing the BF16x2, BF16x3 and FP32 forms")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-extras", action="store_true", help="skip the likelihood and batched workloads")
    args = ap.parse_args()
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch
        import torch.distributed as dist
        if args.impl == "reference":
            dist.init_process_group("gloo")
        else:
            torch.cuda.set_device(local_rank)
            dist.init_process_group("nccl")
    if args.impl == "reference":
        run_reference(args, rank, world)
    else:
        run_ours(args, rank, world, local_rank)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
