"""Row-sharded K^-1 A over several GPUs, one process per GPU (the tree of Sec. 3.3 across
units: every shard's blocks are factored where they live, Eq. 1, and the shards' R factors
are combined pairwise, Eqs. 2-3).

The rows of Y = K0 Omega are split into G contiguous shards; the points and Omega's seed are
on every process.  Per solve there are three collectives, all sums over processes:
  * the shards' d x d R factors (each process contributes its own shards, zeros elsewhere:
    an all-gather written as a sum, exact because every slot has one non-zero contributor);
  * B = Omega^T Q_hat from the shards' parts;
  * Z = Q_hat^T A from the shards' parts.
The top of the tree over the G R factors, the core and its LUs run redundantly on every
process.  The compute of each step is a backend object with the six row-shard calls of the C
ABI (LibraryBackend: the CUDA library on this process's GPU); the communicator is any object
with `sum(tensor) -> tensor` (TorchComm: torch.distributed, NCCL between GPUs).  A process may
hold several shards, so one process can also run all G shards of a problem, one after the
other, with a communicator that returns its argument.
"""
import torch

from . import ckinv as ck


def shard_bounds(n, G, d, align=64):
    """Row boundaries of G contiguous shards of n rows: as equal as the alignment allows
    (boundaries on multiples of `align`), every shard at least d rows."""
    if G < 1 or n < G * d:
        raise ValueError("need G >= 1 and n >= G * d")
    b = [0]
    for k in range(1, G):
        x = (k * n) // G
        x = max(b[-1] + d, min(n - (G - k) * d, (x // align) * align))
        b.append(x)
    b.append(n)
    return b


class LocalComm:
    """The communicator of a process that holds every shard: sums over one process."""

    def sum(self, t):
        return t


class TorchComm:
    """Sums over the processes of a torch.distributed group (NCCL for CUDA tensors, gloo for
    CPU tensors)."""

    def __init__(self, dist, group=None):
        self.dist, self.group = dist, group

    def sum(self, t):
        t = t.contiguous()
        self.dist.all_reduce(t, op=self.dist.ReduceOp.SUM, group=self.group)
        return t


class LibraryBackend:
    """The six row-shard calls of the C ABI on this process's GPU."""

    def __init__(self, ctx):
        self.ctx = ctx

    def zeros(self, shape):
        return torch.zeros(shape, dtype=torch.float64, device="cuda")

    def sketch_rows(self, plan, kern, points, row0, m):
        return ck.sketch_rows(self.ctx, plan, kern, row0, m, points=points)

    def tsqr_shard(self, plan, kern, Y, row0):
        return ck.tsqr_shard(self.ctx, plan, kern, Y, row0)

    def combine(self, f, R_all, G, g):
        return ck.shard_combine(self.ctx, f, R_all, G, g)

    def core(self, f, B):
        ck.shard_core(self.ctx, f, B)

    def solve_begin(self, f, A):
        return ck.shard_solve_begin(self.ctx, f, A)

    def solve_end(self, f, Z, A):
        return ck.shard_solve_end(self.ctx, f, Z, A)

    def r(self, f):
        return f.r()


def kinv_a_sharded(backend, comm, plan, kern, points, A_rows, shards, G):
    """X = K_tilde^-1 A for the rows of the shards this process holds.

    points: all n points (as the backend takes them); A_rows: {shard: that shard's rows of A};
    shards: the global indices of this process's shards; G: the number of shards of the
    problem.  Returns ({shard: its rows of X}, the root R, the shard boundaries)."""
    bounds = shard_bounds(plan.n, G, plan.d)
    d = plan.d
    fac, R_all = {}, backend.zeros((G, d, d))
    for g in shards:                                   # Eq. 1 on every shard's leaves
        r0, r1 = bounds[g], bounds[g + 1]
        Y = backend.sketch_rows(plan, kern, points, r0, r1 - r0)
        fac[g], R = backend.tsqr_shard(plan, kern, Y, r0)
        R_all[g] = R
    R_all = comm.sum(R_all)                            # every shard's R, in shard order
    B = backend.zeros((d, d))
    for g in shards:                                   # Eqs. 2-3 over the shards, redundantly
        B += backend.combine(fac[g], R_all, G, g)
    B = comm.sum(B)
    for g in shards:
        backend.core(fac[g], B)
    Z = None
    for g in shards:
        Zp = backend.solve_begin(fac[g], A_rows[g])
        Z = Zp if Z is None else Z + Zp
    Z = comm.sum(Z)
    X = {g: backend.solve_end(fac[g], Z, A_rows[g]) for g in shards}
    root_R = backend.r(fac[shards[0]]) if shards else None
    return X, root_R, bounds
