"""Seeded synthetic inputs shared by the tests, the benchmark and the oracle checks.

This module holds no arithmetic of the method: it draws points, right-hand sides,
Gaussian-process targets and batch descriptions, and names the workloads.  Every array
is generated on the host with numpy's PCG64 seeded by (seed, stream) and returned in the
precision the library consumes (float32); the oracle upcasts the same values to float64,
so both sides see bit-identical inputs.

Input recipe (the paper's own workloads use a sky-survey dataset that is not available;
these stand in for it):
  points   i.i.d. uniform in [0, 1]^D                       stream 2
  A        i.i.d. N(0, 1), n x m, column-major              stream 3
  y        a squared-exponential GP draw through M random Fourier features
           (omega_j ~ N(0, l^-2 I), b_j ~ U[0, 2 pi)), f = sqrt(2 var / M) sum cos(.),
           plus sqrt(tau) N(0, 1) noise                      streams 4, 5
  batch    n_p log-uniform in [4096, 65536], D_p in {2, 3}, kernel in {SE, Matern-5/2},
           l_p ~ U[0.05, 0.3], d_p in {64, 128, 256}        stream 6
  K = EDE^T  the blocking simulation's covariance: E orthonormalised i.i.d. Gaussian,
           eigenvalues exp(-0.01 i)                          stream 7
"""
import math

import numpy as np

SE = 0
MATERN52 = 1

# The five workloads (sizes and hyper-parameters of each).
CONFIGS = {
    "c1_plain_n2048": dict(n=2048, dim=2, kind=SE, ell=0.2, var=1.0, tau=1e-6, d=64,
                           m=4, block_rows=512, seed=0, leaf_fp64=1),
    "c2_dense_n65536": dict(n=65536, dim=3, kind=MATERN52, ell=0.15, var=1.0, tau=1e-5,
                            d=256, m=16, block_rows=1024, seed=0),
    "c3_bf16_n262144": dict(n=262144, dim=2, kind=SE, ell=0.1, var=1.0, tau=1e-6, d=512,
                            m=32, block_rows=3008, seed=0),
    "c4_nll_n131072": dict(n=131072, dim=2, kind=SE, ell=0.12, var=1.0, tau=1e-4, d=384,
                           m=1, block_rows=2048, seed=0),
    "c5_batch64": dict(nprob=64, m=8, seed=0),
}


def _rng(seed, stream):
    return np.random.Generator(np.random.PCG64([int(seed), int(stream)]))


def points(n, dim, seed=0):
    """n x dim points uniform in [0, 1]^dim, float32, row-major."""
    return _rng(seed, 2).random((n, dim)).astype(np.float32)


def rhs(n, m, seed=0):
    """n x m standard normal right-hand sides, float32, column-major (Fortran order)."""
    return np.asfortranarray(_rng(seed, 3).standard_normal((n, m)).astype(np.float32))


def gp_targets(pts, ell, var, tau, n_features=384, seed=0):
    """Targets from a squared-exponential GP, drawn through random Fourier features."""
    pts = np.asarray(pts, dtype=np.float64)
    n, dim = pts.shape
    r = _rng(seed, 4)
    w = r.standard_normal((dim, n_features)) / ell
    b = r.uniform(0.0, 2.0 * math.pi, n_features)
    z = r.standard_normal(n_features)
    f = math.sqrt(2.0 * var / n_features) * (np.cos(pts @ w + b) @ z)
    eps = _rng(seed, 5).standard_normal(n)
    return (f + math.sqrt(tau) * eps).astype(np.float32)


def batch_specs(nprob=64, seed=0, n_lo=4096, n_hi=65536):
    """Descriptions of the independent GP problems of the batched workload."""
    r = _rng(seed, 6)
    specs = []
    for p in range(nprob):
        n = int(math.floor(math.exp(r.uniform(math.log(n_lo), math.log(n_hi)))))
        dim = int(r.integers(2, 4))
        kind = int(r.integers(0, 2))
        ell = float(r.uniform(0.05, 0.3))
        d = int(r.choice([64, 128, 256]))
        specs.append(dict(n=n, dim=dim, kind=kind, ell=ell, var=1.0, tau=1e-4, d=d,
                          block_rows=max(1024, 2 * d), seed=p))
    return specs


def ede_factors(n, seed=0, rank=None, rate=0.01):
    """The covariance of the paper's blocking simulation, K = E D E^T with E an orthonormalised
    matrix of i.i.d. Gaussian entries and D exponentially decaying eigenvalues of scale 1 and
    rate `rate` (d_ii = exp(-rate i)), returned as (E, D).  rank (default min(n, 2048)) keeps
    the leading columns: beyond 2048 the eigenvalues are below exp(-20.48) = 1.3e-9 of the
    largest, under the FP32 rounding of K's entries.  Stream 7."""
    r = min(n, 2048) if rank is None else rank
    G = _rng(seed, 7).standard_normal((n, r))
    E, _ = np.linalg.qr(G)
    D = np.exp(-rate * np.arange(r, dtype=np.float64))
    return E, D


def ede_matrix(n, seed=0, rank=None, rate=0.01):
    """K = E D E^T as a dense float64 matrix (for sizes a host builds in seconds)."""
    E, D = ede_factors(n, seed, rank, rate)
    return (E * D[None, :]) @ E.T
