"""Writes the stored expected likelihood of the 131072-point workload (tests/golden/).

Calls only the FP64 oracle (oracle/) and the seeded input generators (synth/): the Gaussian
negative log-likelihood and its gradient with respect to (log l, log variance, log nugget)
of n = 131072 points uniform in [0, 1]^2 under the squared-exponential kernel l = 0.12,
variance 1, nugget 1e-4, through the method's K_tilde with a d = 384 sketch (Definition 1,
Sec. 3.2), a TSQR with 2048-row leaves (Sec. 3.3) and one refinement step.  With
--floor it also writes the same quantities with every kernel entry (and derivative entry)
rounded to FP32 before the sketch: the floor of a method whose kernel entries carry FP32
precision - and, from the same sketches, the floor of the library's FP32-level forms at their
working precision: the sketches Y and Y' rounded to FP32 (the arrays those forms store), the
leaf Householder factorisations in FP32 and alpha = K_tilde^-1 y rounded to FP32 before the
gradient.  Usage:
  python tests/golden/make_likelihood_golden.py [--floor] [--keep-exact] [--workers N]
(--keep-exact reuses the exact value already stored instead of recomputing it.)
The sketch row blocks are spread over N processes (default: all CPUs); each block is the
oracle's own computation.  The record is rewritten after each stage.  Takes tens of minutes
(two n x n x d sketches in FP64 per stage).
"""
import json
import multiprocessing
import os
import sys
import time

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

import synth  # noqa: E402
from oracle import kernels as okk  # noqa: E402
from oracle import lowrank as olr  # noqa: E402
from oracle import omega as oom  # noqa: E402

NAME = "c4_nll_n131072"
OUT = os.path.join(os.path.dirname(os.path.abspath(__file__)), "likelihood_n131072_d384.json")


_SHARED = {}


def _init(pts, kind, ell, var, O, round32):
    os.environ.setdefault("OMP_NUM_THREADS", "1")
    _SHARED.update(pts=pts, kind=kind, ell=ell, var=var, O=O, round32=round32)


def _block(r0, block=256):
    """Rows [r0, r0 + block) of Y = K0 Omega and Y' = dK0/dlog(l) Omega."""
    g = _SHARED
    n = g["pts"].shape[0]
    rows = slice(r0, min(n, r0 + block))
    Kb = okk.kernel_matrix(g["pts"][rows], g["pts"], g["kind"], g["ell"], g["var"])
    Db = okk.dkernel_matrix(g["pts"][rows], g["pts"], g["kind"], g["ell"], g["var"])
    if g["round32"]:
        Kb = Kb.astype(np.float32).astype(np.float64)
        Db = Db.astype(np.float32).astype(np.float64)
    return r0, Kb @ g["O"], Db @ g["O"]


def sketches(pts, kind, ell, var, O, round32, workers, block=256):
    """Y = K0 Omega and Y' = dK0/dlog(l) Omega, K0 built one block of rows at a time."""
    n = pts.shape[0]
    Y = np.empty((n, O.shape[1]))
    Yd = np.empty((n, O.shape[1]))
    ctx = multiprocessing.get_context("spawn")
    with ctx.Pool(workers, initializer=_init, initargs=(pts, kind, ell, var, O, round32)) as pool:
        for r0, yb, ydb in pool.imap_unordered(_block, range(0, n, block)):
            Y[r0:r0 + yb.shape[0]] = yb
            Yd[r0:r0 + ydb.shape[0]] = ydb
    return Y, Yd


def likelihood(cfg, y, O, Y, Yd, working32):
    """NLL, gradient and log-determinant from the two sketches (one refinement step); with
    working32 the FP32 storage of the sketches and of alpha and FP32 leaves."""
    r32 = lambda M: np.asarray(M, dtype=np.float32).astype(np.float64)
    if working32:
        Y, Yd = r32(Y), r32(Yd)
    f = olr.factorise(Y, O, cfg["tau"], cfg["block_rows"], np.float32 if working32 else np.float64)
    val, alpha = olr.nll(f, y, 1)
    g, _ = olr.grad(f, y, Y, Yd, r32(alpha) if working32 else alpha)
    return {"nll": float(val), "grad": [float(x) for x in g], "logdet": float(f.logdet())}


def evaluate(cfg, round32, workers):
    """The exact record (round32 False), or the two floors (round32 True) from one pair of
    sketches of FP32-rounded entries."""
    n, d = cfg["n"], cfg["d"]
    pts = synth.points(n, cfg["dim"], seed=0).astype(np.float64)
    y = synth.gp_targets(pts, cfg["ell"], cfg["var"], cfg["tau"], seed=0).astype(np.float64)
    O = oom.omega_matrix(n, d, cfg["seed"])
    Y, Yd = sketches(pts, cfg["kind"], cfg["ell"], cfg["var"], O, round32, workers)
    if not round32:
        return likelihood(cfg, y, O, Y, Yd, False)
    return likelihood(cfg, y, O, Y, Yd, False), likelihood(cfg, y, O, Y, Yd, True)


def main():
    cfg = synth.CONFIGS[NAME]
    rec = {"workload": NAME, "n": cfg["n"], "d": cfg["d"], "kernel": "squared-exponential",
           "lengthscale": cfg["ell"], "variance": cfg["var"], "nugget": cfg["tau"], "seed": cfg["seed"],
           "block_rows": cfg["block_rows"], "refine_steps": 1,
           "written_by": "tests/golden/make_likelihood_golden.py (FP64 oracle only)"}
    workers = os.cpu_count() or 1
    if "--workers" in sys.argv:
        workers = int(sys.argv[sys.argv.index("--workers") + 1])

    def save():
        with open(OUT, "w") as fh:
            json.dump(rec, fh, indent=1)

    t0 = time.time()
    if "--keep-exact" in sys.argv and os.path.exists(OUT):
        with open(OUT) as fh:
            rec["exact"] = json.load(fh)["exact"]
    else:
        rec["exact"] = evaluate(cfg, False, workers)
        print("exact", rec["exact"], "%.0f s" % (time.time() - t0), flush=True)
        save()
    if "--floor" in sys.argv:
        t0 = time.time()
        rec["fp32_kernel_entries"], rec["fp32_working_precision"] = evaluate(cfg, True, workers)
        print("fp32 entries", rec["fp32_kernel_entries"], "%.0f s" % (time.time() - t0), flush=True)
        print("fp32 working precision", rec["fp32_working_precision"], flush=True)
        save()


if __name__ == "__main__":
    main()
