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


def true_residual(X, A_np, pts_np, cfg, rows):
    """||(K0 + tau I) X - A|| / ||A|| over sampled rows: K0's rows from the FP64 oracle, X from
    the GPU.  X = K_tilde^-1 A solves the method's approximation K_tilde = tau I + K_N, so the
    residual measures K_N against K0 (plus the arithmetic), at any size."""
    from oracle import kernels as okk
    Xh = X.double().cpu().numpy()
    pts = pts_np.astype(np.float64)
    Kr = okk.kernel_matrix(pts[rows], pts, cfg["kind"], cfg["ell"], cfg["var"])
    R = Kr @ Xh + cfg["tau"] * Xh[rows] - A_np[rows].astype(np.float64)
    return float(np.linalg.norm(R) / np.linalg.norm(A_np[rows]))


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


def oracle_sample_time(cfg, rows_sample, seed, qr_rows=4096):
    """FP64 CPU oracle on a bounded sample of one solve of the workload.  Times (1) Omega,
    built once per solve; (2) the sketch rows [0, rows_sample), scaled by n / rows_sample
    (each row costs the same n kernel entries times Omega); (3) the TSQR with its tree, the
    core and the refined solve of the first qr_rows rows of that sketch (two-leaf TSQR), scaled
    by n / qr_rows (leaves, tree combines, B = Omega^T Q_hat, Q_hat^T A and the Q_hat products
    of the solve all grow linearly with the row count; the d x d LUs, counted once per
    sample, are over-counted by the scaling).  Returns (seconds spent, extrapolated seconds
    per solve, the parts)."""
    from oracle import lowrank as olr
    from oracle import omega as oom
    from oracle import sketch as osk
    n, d, b = cfg["n"], cfg["d"], cfg["block_rows"]
    pts = synth.points(n, cfg["dim"], 0).astype(np.float64)
    t0 = time.perf_counter()
    O = oom.omega_matrix(n, d, seed)
    t1 = time.perf_counter()
    Yrows = []
    # rows drawn at random from [0, n): the first rows alone, or evenly strided ones, see a
    # rank-deficient slice of Omega (its Walsh-Hadamard columns agree on those row indices)
    sample = np.sort(np.random.default_rng(seed).choice(n, rows_sample, replace=False))
    for r0 in range(0, rows_sample, 256):         # 256 rows of K0 (0.5 GB at n = 262144) at a time
        Yrows.append(osk.sketch_rows(pts, sample[r0:r0 + 256], cfg["kind"], cfg["ell"], cfg["var"], O))
    t2 = time.perf_counter()
    Ys = np.vstack(Yrows)
    qr_rows = min(qr_rows, Ys.shape[0])
    t3 = t4 = time.perf_counter()
    if qr_rows >= 2 * d:                          # two leaves of at least d rows
        Ys = Ys[:qr_rows]
        A = synth.rhs(qr_rows, cfg["m"], 0).astype(np.float64)
        t3 = time.perf_counter()
        f = olr.factorise(Ys, O[sample[:qr_rows]], cfg["tau"], min(b, qr_rows // 2))
        olr.solve_refined(f, A, 1)
        t4 = time.perf_counter()
    else:
        qr_rows = 1                               # not sampled
    parts = {"omega_s": t1 - t0, "sketch_rows_s": t2 - t1, "sketch_rows": rows_sample,
             "qr_core_solve_s": t4 - t3, "qr_rows": qr_rows}
    full = (t1 - t0) + (t2 - t1) * n / rows_sample + (t4 - t3) * n / qr_rows
    return (t2 - t0) + (t4 - t3), full, parts


def cpu_threads():
    """(threads the BLAS under numpy uses, logical CPUs of the host)."""
    blas = None
    try:
        import threadpoolctl
        info = threadpoolctl.threadpool_info()
        blas = max([i.get("num_threads", 1) for i in info] + [1])
    except Exception:
        pass
    cpus = os.cpu_count() or 1
    return (blas if blas else cpus), cpus


def run_reference(args, rank, world):
    """The reference arm: the FP64 oracle, as it stands, on this host's cores.  Each step is
    a bounded sample of one solve (see oracle_sample_time); ms_per_step is the time those
    samples took, `value` the solves/s they extrapolate to."""
    cfg = workload_config(args.workload)
    if rank != 0:
        return
    rows = max(2 * cfg["d"], args.ref_rows // 2)   # half the bench's sample per step
    qr_rows = rows
    for _ in range(args.warmup):
        oracle_sample_time(cfg, 256, 0, qr_rows=0)
    spent, per = [], []
    for s in range(args.steps):
        t, full, parts = oracle_sample_time(cfg, rows, s, qr_rows=qr_rows)
        spent.append(t)
        per.append(full)
    sps = 1.0 / float(np.mean(per))
    blas, cpus = cpu_threads()
    sample = ("FP64 oracle per step: Omega (%d columns of %d rows), %d random sketch rows of %d, and TSQR + core + "
              "refined solve of %d sketch rows; each part scaled to the whole solve by its row count"
              % (cfg["d"], cfg["n"], rows, cfg["n"], qr_rows))
    line = {"impl": "reference", "metric": METRIC, "value": sps, "unit": "solves/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * float(np.mean(spent)),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic",
            "config": {"workload": cfg["workload"], "n": cfg["n"], "d": cfg["d"], "m": cfg["m"],
                       "kernel": KERNEL_NAMES[cfg["kind"]], "lengthscale": cfg["ell"], "nugget": cfg["tau"]},
            "extrapolated_s_per_solve": float(np.mean(per)),
            "timing": "ms_per_step is the measured time of one step's bounded sample; value extrapolates the "
                      "sample to whole solves",
            "cpu_baseline": {"value": sps, "unit": "solves/s", "cores": blas, "host_cpus": cpus, "kind": "oracle",
                             "sample": sample},
            "e2e": {"value": sps, "unit": "solves/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def golden_likelihood():
    """The stored FP64 oracle likelihood of the 131072-point workload (written by
    tests/golden/make_likelihood_golden.py), or None."""
    p = os.path.join(ROOT, "tests", "golden", "likelihood_n131072_d384.json")
    try:
        with open(p) as fh:
            return json.load(fh)
    except (OSError, ValueError):
        return None


def run_likelihood(ck, ctx, dev, reps=3):
    """The likelihood workload: NLL and gradient at n = 131072, d = 384 (one ckinv_nll_grad
    call each; it returns host scalars, so it is timed by the host clock), in the
    FP32-accurate three-term form the workload names (kernel entries carried to 24 bits), with
    FP32 and with FP64 leaves, and in the one-term BF16 form; each against the stored oracle
    value."""
    cfg = workload_config("c4_nll_n131072")
    n, d, dim = cfg["n"], cfg["d"], cfg["dim"]
    pts_np = synth.points(n, dim, seed=0)
    y_np = synth.gp_targets(pts_np, cfg["ell"], cfg["var"], cfg["tau"], seed=0)
    pts = torch_from(pts_np, dev)
    y = torch_from(y_np, dev)
    kern = ck.Kernel(cfg["kind"], cfg["ell"], cfg["var"], cfg["tau"])
    gold = golden_likelihood()
    out = {"workload": "c4_nll_n131072", "n": n, "d": d,
           "timing": "host wall clock around the call (it returns host scalars), median of %d" % reps}
    for name, prec, leaf64 in [("bf16x3", ck.BF16X3, 0), ("bf16x3_fp64_leaves", ck.BF16X3, 1), ("bf16", ck.BF16, 0),
                               ("fp32_wht", ck.FP32_WHT, 0), ("fp32_wht_fp64_leaves", ck.FP32_WHT, 1)]:
        plan = ck.Plan(n=n, d=d, dim=dim, block_rows=cfg["block_rows"], prec=prec, seed=cfg["seed"], refine_steps=1,
                       tree_fp64_levels=-1, leaf_fp64=leaf64)
        ck.nll_grad(ctx, plan, kern, pts, y)
        times = []
        for _ in range(reps):
            t0 = time.perf_counter()
            val, g = ck.nll_grad(ctx, plan, kern, pts, y)
            times.append(time.perf_counter() - t0)
        t = float(np.median(times))
        rec = {"ms_per_eval": 1e3 * t, "evals_per_s": 1.0 / t, "nll": val, "grad": g}
        if gold and "exact" in gold:
            ex = gold["exact"]
            rec["nll_rel_err_vs_oracle"] = abs(val - ex["nll"]) / abs(ex["nll"])
            rec["grad_rel_err_vs_oracle"] = [abs(a - b) / abs(b) for a, b in zip(g, ex["grad"])]
        out[name] = rec
    if gold and "fp32_kernel_entries" in gold:
        ex, fl = gold["exact"], gold["fp32_kernel_entries"]
        out["oracle_floor_fp32_entries"] = {
            "nll_rel": abs(fl["nll"] - ex["nll"]) / abs(ex["nll"]),
            "grad_rel": [abs(a - b) / abs(b) for a, b in zip(fl["grad"], ex["grad"])],
            "note": "the oracle itself with every kernel entry rounded to FP32"}
    return out


def run_materialised(ck, ctx, dev, stream, peaks):
    """The plain method with K in HBM: n = 65536 points in [0, 1]^3, Matern-5/2 l = 0.15,
    d = 256.  K0 (17.2 GB FP32) is materialised by the library (untimed), then the sketch of
    the given matrix is timed with CUDA events (K read once: the HBM-bound step), in the FP32
    SIMT form, the one- and three-term tensor-core forms and the FP32 fast transform over K's
    columns, and the whole solve (sketch, TSQR, core, refined solve of m = 16 right-hand sides)
    in the FP32 forms the workload names (SIMT contraction and fast transform)."""
    import torch
    cfg = workload_config("c2_dense_n65536")
    n, d, dim, m = cfg["n"], cfg["d"], cfg["dim"], cfg["m"]
    pts_np = synth.points(n, dim, 0)
    A_np = synth.rhs(n, m, 0)
    pts = torch_from(pts_np, dev)
    A = torch.from_numpy(np.ascontiguousarray(A_np.T)).to(dev).t()
    kern = ck.Kernel(cfg["kind"], cfg["ell"], cfg["var"], cfg["tau"])
    dense = ck.Kernel(ck.DENSE, 0, 0, cfg["tau"])
    plan = ck.Plan(n=n, d=d, dim=dim, block_rows=cfg["block_rows"], prec=ck.FP32, seed=0, refine_steps=1)
    K = ck.kernel_matrix(ctx, plan, kern, pts)
    Y = ck.colmajor(n, d, device=dev)
    X = ck.colmajor(n, m, device=dev)
    bytes_k = 4.0 * n * n
    hbm = float(peaks.get("hbm_gbs", PEAKS_FALLBACK["hbm_gbs"]))
    out = {"workload": "c2_dense_n65536", "n": n, "d": d, "m": m, "K_bytes": bytes_k,
           "timing": "CUDA events on the launching stream, best of 3 after one untimed run"}
    for name, prec in [("fp32", ck.FP32), ("bf16", ck.BF16), ("bf16x3", ck.BF16X3), ("fp32_wht", ck.FP32_WHT)]:
        p2 = ck.Plan(n=n, d=d, dim=dim, block_rows=cfg["block_rows"], prec=prec, seed=0, refine_steps=1)
        best = None
        for r in range(4):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            ck.sketch(ctx, p2, dense, K=K, Y=Y)
            e1.record(stream)
            e1.synchronize()
            if r:
                t = e0.elapsed_time(e1)
                best = t if best is None else min(best, t)
        gbs = bytes_k / (best / 1e3) / 1e9
        out["sketch_" + name] = {"ms": best, "K_read_GBps": gbs, "frac_of_hbm": gbs / hbm}
    ck.check(ctx)
    rows = np.linspace(0, n - 1, 48).astype(np.int64)
    out["sketch_fp32"]["rel_err_sampled"] = sampled_sketch_error(ck, Y_of(ck, ctx, plan, dense, K, Y), pts_np, cfg, 0,
                                                                  rows)
    plan_w = ck.Plan(n=n, d=d, dim=dim, block_rows=cfg["block_rows"], prec=ck.FP32_WHT, seed=0, refine_steps=1)
    out["sketch_fp32_wht"]["rel_err_sampled"] = sampled_sketch_error(ck, Y_of(ck, ctx, plan_w, dense, K, Y), pts_np,
                                                                      cfg, 0, rows)
    # the whole solve in the workload's FP32 form: the SIMT contraction and the fast transform
    for name, pl in [("fp32", plan), ("fp32_wht", plan_w)]:
        best = None
        for r in range(3):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            ck.sketch(ctx, pl, dense, K=K, Y=Y)
            f = ck.tsqr(ctx, pl, dense, Y)
            ck.solve(ctx, f, A, X)
            f.free()
            e1.record(stream)
            e1.synchronize()
            if r:
                t = e0.elapsed_time(e1)
                best = t if best is None else min(best, t)
        ck.check(ctx)
        out["solve_" + name] = {"ms_per_solve": best, "solves_per_s": 1e3 / best,
                                "true_residual_sampled": true_residual(X, A_np, pts_np, cfg, rows)}
    del K
    torch.cuda.empty_cache()
    out["peak_hbm_GBps"] = hbm
    return out


def Y_of(ck, ctx, plan, dense, K, Y):
    ck.sketch(ctx, plan, dense, K=K, Y=Y)
    return Y


def torch_from(a, dev):
    import torch
    return torch.from_numpy(a).to(dev)


def run_projection(ck, ctx, dev, n_new=4096):
    """The paper's accuracy measure and prediction at the likelihood workload's size (n = 131072,
    d = 384, SE l = 0.12): the second pass S = Q_hat^T K0 Q_hat with the column-space error
    ||K0 - Q Q^T K0||_F / ||K0||_F (6 BF16 tensor-core products of the n x n x d contraction and
    one FP32 pass over the n^2 kernel entries), the two-pass solve, and the predictive mean at
    n_new new points (FP64 entries and sums).  Host wall clock around each call (the
    column-space error is returned to the host); best of 3 after one untimed call."""
    import torch
    cfg = workload_config("c4_nll_n131072")
    n, d, dim = cfg["n"], cfg["d"], cfg["dim"]
    pts = torch_from(synth.points(n, dim, 0), dev)
    y = torch_from(synth.gp_targets(synth.points(n, dim, 0), cfg["ell"], cfg["var"], cfg["tau"], seed=0), dev)
    xnew = torch_from(synth.points(n_new, dim, 1), dev)
    plan = ck.Plan(n=n, d=d, dim=dim, block_rows=cfg["block_rows"], prec=ck.BF16X3, seed=0, refine_steps=1)
    kern = ck.Kernel(cfg["kind"], cfg["ell"], cfg["var"], cfg["tau"])
    f = ck.tsqr(ctx, plan, kern, ck.sketch(ctx, plan, kern, pts))

    def best(fn, reps=3):
        fn()
        torch.cuda.synchronize()
        ts = []
        for _ in range(reps):
            t0 = time.perf_counter()
            r = fn()
            torch.cuda.synchronize()
            ts.append(time.perf_counter() - t0)
        return min(ts), r
    t_proj, (_, err) = best(lambda: ck.project(ctx, f, plan, kern, pts))
    alpha = ck.solve(ctx, f, y)
    t_pred, _ = best(lambda: ck.predict_mean(ctx, plan, kern, pts, alpha, xnew))
    ck.check(ctx)
    flops = 6 * 2.0 * n * n * d
    return {"workload": "c4_nll_n131072", "n": n, "d": d, "second_pass_ms": 1e3 * t_proj,
            "second_pass_tflops": flops / t_proj / 1e12, "second_pass_flops": flops,
            "colspace_rel_err": err, "predict_n_new": n_new, "predict_ms": 1e3 * t_pred,
            "predict_fp64_kernel_evals_per_s": n * n_new / t_pred,
            "timing": "host wall clock with a device synchronisation, best of 3 after one untimed call"}


def run_blocking_simulation(ck, ctx, dev, sizes=(1000, 5000, 10000, 50000), d=512, m=16, tau=1e-3):
    """The paper's blocking simulation (Sec. 5.1): K = E D E^T (E orthonormalised Gaussian,
    eigenvalues exp(-0.01 i)) at n = 1000 .. 50000, solved through the materialised path with
    each of the four Omega choices (Walsh-Hadamard - as the fast transform and as a dense
    contraction - scaled Gaussian, Hartley, cosine), FP32 forms.  K is built on the GPU from host-drawn factors (input generation, untimed; rank
    min(n, 1024): the eigenvalues beyond are below exp(-10.24) = 3.6e-5 of the largest).
    Per size and Omega: the solve (sketch, TSQR, core, refined solve of m right-hand sides)
    timed with CUDA events (best of 2 after an untimed run) and the residual of its X against
    that K on 48 sampled rows."""
    import torch
    stream = torch.cuda.current_stream(dev)
    out = {"d": d, "m": m, "nugget": tau, "rank": "min(n, 1024)",
           "timing": "CUDA events, best of 2 after one untimed run"}
    # the structured Walsh-Hadamard Omega applied as a fast transform (FP32), and as the
    # compensated dense contraction for comparison; the other three are dense Omega (SIMT GEMM)
    kinds = [("wht", ck.WHT, ck.FP32_WHT), ("wht_dense_contraction", ck.WHT, ck.FP32), ("gaussian", ck.GAUSSIAN, ck.FP32),
             ("hartley", ck.HARTLEY, ck.FP32), ("cosine", ck.COSINE, ck.FP32)]
    for n in sizes:
        E, D = synth.ede_factors(n, seed=0, rank=min(n, 1024))
        Et = torch.from_numpy(E.astype(np.float32)).to(dev)
        K = (Et * torch.from_numpy(D.astype(np.float32)).to(dev)[None, :]) @ Et.t()   # symmetric, n x n
        del Et
        A_np = synth.rhs(n, m, 0)
        A = torch.from_numpy(np.ascontiguousarray(A_np.T)).to(dev).t()
        rows = np.linspace(0, n - 1, 48).astype(np.int64)
        Krows = K[torch.from_numpy(rows).to(dev)].double().cpu().numpy()
        rec = {}
        for name, kind, prec in kinds:
            plan = ck.Plan(n=n, d=min(d, n // 2 // 16 * 16), block_rows=max(1024, 2 * d) if n >= 4 * d else 0,
                           prec=prec, seed=0, refine_steps=1, omega_kind=kind)
            dense = ck.Kernel(ck.DENSE, 0, 0, tau)
            best, X = None, None
            for r in range(3):
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                Y = ck.sketch(ctx, plan, dense, K=K.t())          # K is symmetric: its transpose view is column-major
                f = ck.tsqr(ctx, plan, dense, Y)
                X = ck.solve(ctx, f, A)
                f.free()
                e1.record(stream)
                e1.synchronize()
                if r:
                    t = e0.elapsed_time(e1)
                    best = t if best is None else min(best, t)
            ck.check(ctx)
            Xh = X.double().cpu().numpy()
            res = Krows @ Xh + tau * Xh[rows] - A_np[rows]
            rec[name] = {"ms_per_solve": best, "d": plan.d,
                         "true_residual_sampled": float(np.linalg.norm(res) / np.linalg.norm(A_np[rows]))}
        out["n%d" % n] = rec
        del K
        torch.cuda.empty_cache()
    return out


def run_batched(ck, ctx, dev):
    """The 64-problem batch: one ckinv_nll_grad_batched call (graph capture, instantiation,
    launch and read-back), timed by the host clock."""
    import torch
    specs = synth.batch_specs(64, seed=0)
    plans, kerns, P, Ys = [], [], [], []
    for sp in specs:
        plans.append(ck.Plan(n=sp["n"], d=sp["d"], dim=sp["dim"], block_rows=sp["block_rows"], prec=ck.BF16,
                             seed=1000 + sp["seed"]))
        kerns.append(ck.Kernel(sp["kind"], sp["ell"], sp["var"], sp["tau"]))
        p_np = synth.points(sp["n"], sp["dim"], sp["seed"])
        P.append(torch.from_numpy(p_np).to(dev))
        Ys.append(torch.from_numpy(synth.gp_targets(p_np, 0.2, 1.0, sp["tau"], seed=sp["seed"])).to(dev))
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    ck.nll_grad_batched(ctx, plans, kerns, P, Ys)          # capture, instantiate, launch
    t_first = time.perf_counter() - t0
    times = []
    for _ in range(3):
        t0 = time.perf_counter()
        ck.nll_grad_batched(ctx, plans, kerns, P, Ys)      # the kept graph, launched again
        times.append(time.perf_counter() - t0)
    tb = float(min(times))
    flops = sum(2.0 * 2.0 * sp["n"] * sp["n"] * sp["d"] for sp in specs)   # forward and derivative sketches
    return {"workload": "c5_batch64", "problems": len(specs), "ms_per_batch": 1e3 * tb,
            "problems_per_s": len(specs) / tb, "prec": "bf16", "ms_first_call": 1e3 * t_first,
            "sketch_dense_equiv_flops": flops, "sketch_tflops_over_batch": flops / tb / 1e12,
            "timing": "host wall clock around one ckinv_nll_grad_batched call that relaunches the kept graph "
                      "(launch and read-back of 64 likelihoods), best of 3; ms_first_call adds capture and "
                      "instantiation"}


def run_ours(args, rank, world, local_rank):
    import torch
    import __graft_entry__
    __graft_entry__.build()
    from paper_1312_1869_gb300 import ckinv as ck

    torch.cuda.set_device(local_rank)
    dev = torch.device("cuda", local_rank)
    cfg = workload_config(args.workload)
    if args.block_rows:
        cfg["block_rows"] = args.block_rows
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
        dt, full, parts = oracle_sample_time(cfg, args.ref_rows, 0)
        blas, cpus = cpu_threads()
        cpu = {"value": 1.0 / full, "unit": "solves/s", "cores": blas, "host_cpus": cpus, "kind": "oracle",
               "sample": "FP64 oracle: Omega, %d random sketch rows of %d, TSQR + core + refined solve of %d sketch "
                         "rows (%.1f s in all), each part scaled to the whole solve by its row count"
                         % (args.ref_rows, n, parts["qr_rows"], dt),
               "parts_s": parts}

    forms = None
    if rank == 0 and not args.no_forms:
        # every precision form of the same solve (same Omega, points and A; best of two timed
        # runs after an untimed one, one timed run for the slow SIMT FP32 form), each with the
        # residual of its X against the true kernel matrix on sampled rows
        rows = np.linspace(0, n - 1, 48).astype(np.int64)
        forms = {}
        for name, prec, lv in [("bf16", args.prec, args.fp64_levels), ("bf16x2", "bf16x2", args.fp64_levels),
                               ("bf16x3", "bf16x3", args.fp64_levels), ("fp32", "fp32", args.fp64_levels),
                               ("fp32_wht", "fp32_wht", args.fp64_levels), ("bf16_fp32_tree", args.prec, 0)]:
            plan2 = ck.Plan(n=n, d=d, dim=dim, block_rows=cfg["block_rows"], prec=ck.PRECISIONS[prec], seed=5,
                            refine_steps=args.refine, tree_fp64_levels=lv)
            best = None
            reps = 2 if prec == "fp32" else 3
            for rep_i in range(reps):
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
            ck.check(ctx)
            forms[name] = {"solves_per_s": 1e3 / best, "ms_per_solve": best, "tree_fp64_levels": lv,
                           "true_residual_sampled": true_residual(X, A_np, pts_np, cfg, rows)}
            if prec == "fp32_wht":
                # the fast-transform sketch alone (CUDA events, best of 3 after the runs above):
                # n^2 kernel entries, each evaluated, transformed and gathered in FP32
                sk = None
                for _ in range(3):
                    flush.zero_()
                    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                    e0.record(stream)
                    ck.sketch(ctx, plan2, kern, pts, Y=Y)
                    e1.record(stream)
                    e1.synchronize()
                    t = e0.elapsed_time(e1)
                    sk = t if sk is None else min(sk, t)
                forms[name]["sketch_ms"] = sk
                forms[name]["kernel_evals_per_s"] = float(n) * float(n) / (sk / 1e3)
                forms[name]["sketch_rel_err_sampled"] = sampled_sketch_error(ck, Y, pts_np, cfg, 5, rows)
        forms["residual_note"] = ("||(K0 + tau I) X - A|| / ||A|| on 48 sampled rows, K0 rows from the FP64 oracle: "
                                  "the method's approximation K_tilde of K0 + tau I, not the arithmetic, sets it")

    extras = {}
    if rank == 0 and not args.no_extras:
        extras["likelihood"] = run_likelihood(ck, ctx, dev)
        extras["materialised"] = run_materialised(ck, ctx, dev, stream, peaks)
        extras["batched"] = run_batched(ck, ctx, dev)
        extras["projection"] = run_projection(ck, ctx, dev)
        extras["blocking_simulation"] = run_blocking_simulation(ck, ctx, dev)

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
            line["accuracy"] = {
                "sketch_rel_err_sampled": y_err,
                "true_residual_sampled": forms[args.prec]["true_residual_sampled"] if args.prec in forms else None,
                "true_residual_sampled_bf16x3": forms["bf16x3"]["true_residual_sampled"],
                "true_residual_sampled_fp32": forms["fp32"]["true_residual_sampled"],
                "note": "||(K0 + tau I) X - A|| / ||A|| on 48 sampled rows for the timed form and for the FP32-level "
                        "forms; equal residuals mean the sketch's approximation, not the arithmetic, bounds the "
                        "accuracy here (kappa(Y) ~ 1e11: X itself is O(0.1) from the oracle's in every form)"}
        line.update(extras)
        print(json.dumps(line), flush=True)
    ctx.close()


def run_profile(args):
    """A bare loop over one part of the step (the fused sketch, the TSQR with its core, or
    the whole step) on the workload, or over the sketch of a materialised K (sketch_dense: the
    65536-point Matern workload, K built untimed), optionally at a smaller n: the command the
    ncu captures of profiles/ run."""
    import torch
    import __graft_entry__
    __graft_entry__.build()
    from paper_1312_1869_gb300 import ckinv as ck
    dense = args.profile_kernel == "sketch_dense"
    cfg = workload_config("c2_dense_n65536" if dense else args.workload)
    n = args.n or cfg["n"]
    d, m, dim = cfg["d"], cfg["m"], cfg["dim"]
    ctx = ck.Context(0)
    plan = ck.Plan(n=n, d=d, dim=dim, block_rows=cfg["block_rows"], prec=ck.PRECISIONS[args.prec], seed=0,
                   refine_steps=args.refine, tree_fp64_levels=args.fp64_levels)
    kern = ck.Kernel(cfg["kind"], cfg["ell"], cfg["var"], cfg["tau"])
    pts = torch.from_numpy(synth.points(n, dim, 0)).cuda()
    A = torch.from_numpy(np.ascontiguousarray(synth.rhs(n, m, 0).T)).cuda().t()
    Y = ck.colmajor(n, d)
    X = ck.colmajor(n, m)
    K = None
    if dense:
        K = ck.kernel_matrix(ctx, plan, kern, pts)
        kern = ck.Kernel(ck.DENSE, 0, 0, cfg["tau"])
        ck.sketch(ctx, plan, kern, K=K, Y=Y)
    else:
        ck.sketch(ctx, plan, kern, pts, Y=Y)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    for i in range(args.warmup + args.steps):
        if i == args.warmup:
            e0.record()
        if dense:
            ck.sketch(ctx, plan, kern, K=K, Y=Y)
        if args.profile_kernel in ("sketch", "step"):
            ck.sketch(ctx, plan, kern, pts, Y=Y)
        if args.profile_kernel in ("tsqr", "step"):
            f = ck.tsqr(ctx, plan, kern, Y)
            if args.profile_kernel == "step":
                ck.solve(ctx, f, A, X)
            f.free()
    e1.record()
    torch.cuda.synchronize()
    ck.check(ctx)
    print(json.dumps({"profile": args.profile_kernel, "n": n, "d": d, "prec": args.prec,
                      "launches": args.warmup + args.steps,
                      "ms_per_iteration": e0.elapsed_time(e1) / args.steps if args.steps else None}), flush=True)
    ctx.close()


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="c3_bf16_n262144")
    ap.add_argument("--prec", default="bf16", choices=["fp32", "bf16", "bf16x2", "bf16x3", "fp32_wht"])
    ap.add_argument("--refine", type=int, default=1)
    ap.add_argument("--fp64-levels", type=int, default=-1, help="tree levels combined in FP64 (-1: all)")
    ap.add_argument("--ref-rows", type=int, default=2048, help="sketch rows in the oracle's timed sample")
    ap.add_argument("--no-forms", action="store_true", help="skip timing the BF16x2, BF16x3 and FP32 forms")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-extras", action="store_true", help="skip the likelihood and batched workloads")
    ap.add_argument("--profile-kernel", default=None, choices=["sketch", "sketch_dense", "tsqr", "step"],
                    help="run only `steps` launches of one part of the step (for ncu captures): no JSON contract line")
    ap.add_argument("--n", type=int, default=None, help="override the workload's n (profiling a smaller case)")
    ap.add_argument("--block-rows", type=int, default=None, help="override the workload's TSQR leaf height")
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
    elif args.profile_kernel:
        run_profile(args)
    else:
        run_ours(args, rank, world, local_rank)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
