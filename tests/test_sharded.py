"""The row-sharded solve's orchestration (paper_1312_1869_gb300/sharded.py) on CPU.

The product code decides the shard boundaries, which process computes what, and the order
and content of the three collectives; these tests run it over gloo ranks on 127.0.0.1 (world
size 2, one or two shards per process) and in one process holding three shards, with the
per-shard compute supplied by the FP64 oracle (a backend with the same six calls as the
CUDA library's row-shard entry points).  The sharded R and X must equal the single-process
oracle's: R is unique for a full-rank Y (diag(R) >= 0), so the shards' tree over R factors
gives the R of the leaves' tree over all rows (Sec. 3.3, Eqs. 1-4).
"""
import os
import socket
import sys

import numpy as np
import pytest
import torch
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import synth  # noqa: E402

N, D, ELL, TAU, B, SEED, M = 1536, 32, 0.2, 1e-3, 256, 3, 3


class OracleShard:
    def __init__(self, Q, R, row0):
        self.Q, self.R, self.row0 = Q, R, row0
        self.B = self.lu_B = self.lu_C = None


class OracleBackend:
    """The six row-shard calls, computed by the FP64 oracle (test infrastructure)."""

    def __init__(self, n, d, seed):
        from oracle import omega as oom
        self.O = oom.omega_matrix(n, d, seed)

    def zeros(self, shape):
        return torch.zeros(shape, dtype=torch.float64)

    def sketch_rows(self, plan, kern, points, row0, m):
        from oracle import sketch as osk
        return osk.sketch_rows(points, np.arange(row0, row0 + m), kern["kind"], kern["ell"], kern["var"], self.O)

    def tsqr_shard(self, plan, kern, Y, row0):
        from oracle import tsqr as ots
        t = ots.tsqr(Y, B)
        return OracleShard(t["Q"], t["R"], row0), torch.from_numpy(t["R"].copy())

    def combine(self, f, R_all, G, g):
        from oracle import tsqr as ots
        d = f.R.shape[0]
        stacked = R_all.numpy().reshape(G * d, d)
        top = ots.tsqr(stacked, d)                   # one leaf per shard R, then the tree
        f.Q = f.Q @ top["Q"][g * d:(g + 1) * d]
        f.R = top["R"]
        return torch.from_numpy(self.O[f.row0:f.row0 + f.Q.shape[0]].T @ f.Q)

    def core(self, f, B_):
        from oracle import lowrank as olr
        f.B = B_.numpy()
        f.lu_B = olr.lu_factor(f.B)
        f.lu_C = olr.lu_factor(f.R.T + TAU * f.B)

    def solve_begin(self, f, A):
        return torch.from_numpy(f.Q.T @ A)

    def solve_end(self, f, Z, A):
        from oracle import lowrank as olr
        V = olr.lu_solve(f.lu_C, f.R.T @ Z.numpy())
        return (A - f.Q @ V) / TAU

    def r(self, f):
        return f.R


def _problem():
    pts = synth.points(N, 2, SEED).astype(np.float64)
    A = synth.rhs(N, M, SEED).astype(np.float64)
    return pts, A


def _reference():
    from oracle import lowrank as olr
    pts, A = _problem()
    X, f, _ = olr.kinv_a(pts, A, 0, ELL, 1.0, TAU, D, SEED, B, refine_steps=0)
    return X, f.R


def _run(comm, shards, G):
    from paper_1312_1869_gb300 import sharded
    pts, A = _problem()
    bounds = sharded.shard_bounds(N, G, D)
    A_rows = {g: A[bounds[g]:bounds[g + 1]] for g in shards}
    plan = type("P", (), {"n": N, "d": D})()
    kern = {"kind": 0, "ell": ELL, "var": 1.0}
    return sharded.kinv_a_sharded(OracleBackend(N, D, SEED), comm, plan, kern, pts, A_rows, shards, G)


def _check(X, R, bounds, Xo, Ro):
    assert np.abs(R - Ro).max() <= 1e-10 * np.abs(Ro).max()
    for g, Xg in X.items():
        ref = Xo[bounds[g]:bounds[g + 1]]
        assert np.linalg.norm(Xg - ref) <= 1e-8 * np.linalg.norm(ref)


def test_shard_bounds_cover_the_rows():
    from paper_1312_1869_gb300 import sharded
    for n, G, d in [(1536, 2, 32), (1536, 3, 32), (100000, 8, 512), (4096, 4, 1024)]:
        b = sharded.shard_bounds(n, G, d)
        assert b[0] == 0 and b[-1] == n and len(b) == G + 1
        assert all(b[k + 1] - b[k] >= d for k in range(G))
    with pytest.raises(ValueError):
        sharded.shard_bounds(100, 4, 32)


def test_one_process_three_shards_equals_the_oracle():
    from paper_1312_1869_gb300 import sharded
    Xo, Ro = _reference()
    X, R, bounds = _run(sharded.LocalComm(), [0, 1, 2], 3)
    _check(X, R, bounds, Xo, Ro)


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, per_rank, out):
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        from paper_1312_1869_gb300 import sharded
        G = world * per_rank
        shards = list(range(rank * per_rank, (rank + 1) * per_rank))
        X, R, bounds = _run(sharded.TorchComm(dist), shards, G)
        out.put((rank, {g: x for g, x in X.items()}, R, bounds))
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("per_rank", [1, 2])
def test_two_gloo_ranks_equal_the_oracle(per_rank):
    world = 2
    ctx = mp.get_context("spawn")
    out = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, world, port, per_rank, out)) for r in range(world)]
    for p in procs:
        p.start()
    res = [out.get(timeout=300) for _ in range(world)]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    Xo, Ro = _reference()
    for rank, X, R, bounds in res:
        assert len(X) == per_rank
        _check(X, R, bounds, Xo, Ro)
