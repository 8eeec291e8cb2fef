"""Structured random matrices Omega = c R T P (Definition 1, Sec. 3.2) with the other
orthogonal transforms the paper names for T: the discrete Hartley and the discrete cosine
matrix (Sec. 3.2; the paper's simulations and data example use both, Sec. 5).  Unlike the
Walsh-Hadamard matrix they exist for every order, so T is n x n and no padding is needed.
Test infrastructure (see the package docstring).

Readings (the paper fixes none of these):
  * Hartley: T[k, p] = cas(2 pi k p / n) = cos(2 pi k p / n) + sin(2 pi k p / n), which
    satisfies T^T T = n I; c = n^(-1/2) makes Omega's columns orthonormal.
  * Cosine: T[k, p] = s_p cos(pi (2k + 1) p / (2n)), s_0 = n^(-1/2), s_p = (2/n)^(1/2)
    otherwise (the orthonormal DCT-II basis vectors as columns); c = 1.
  * R as for the Walsh-Hadamard form (Philox stream 0); P by the same smallest-key rule
    (Philox stream 1) over the candidates [0, n).
"""
import numpy as np

from .omega import rademacher_signs
from .philox import philox4x32_10


def subsample_columns_n(n, d, seed):
    """d distinct column indices of [0, n), ascending: the d smallest Philox keys."""
    if not (0 < d <= n):
        raise ValueError("need 0 < d <= n")
    cand = np.arange(n, dtype=np.uint64)
    w0, w1, _, _ = philox4x32_10(cand, 1, seed)
    keys = (w0 << np.uint64(32)) | w1
    order = np.lexsort((cand, keys))
    return np.sort(order[:d]).astype(np.int64)


def hartley_entries(k, p, n):
    """cas(2 pi k p / n), broadcasting.  k p is reduced mod n first (exact in integers)."""
    kp = (np.asarray(k, dtype=np.int64) * np.asarray(p, dtype=np.int64)) % int(n)
    a = 2.0 * np.pi * kp / float(n)
    return np.cos(a) + np.sin(a)


def cosine_entries(k, p, n):
    """s_p cos(pi (2k + 1) p / (2n)), broadcasting."""
    k = np.asarray(k, dtype=np.int64)
    p = np.asarray(p, dtype=np.int64)
    m = ((2 * k + 1) * p) % (4 * int(n))          # the angle's period is 4n in these units
    s = np.where(p == 0, np.sqrt(1.0 / n), np.sqrt(2.0 / n))
    return s * np.cos(np.pi * m / (2.0 * n))


def omega_matrix_t(n, d, seed, transform):
    """Omega = c R T P (n x d, float64) for transform in {"hartley", "cosine"}."""
    rows = np.arange(n, dtype=np.int64)
    cols = subsample_columns_n(n, d, seed)
    r = rademacher_signs(n, seed)
    if transform == "hartley":
        T = hartley_entries(rows[:, None], cols[None, :], n)
        c = 1.0 / np.sqrt(float(n))
    elif transform == "cosine":
        T = cosine_entries(rows[:, None], cols[None, :], n)
        c = 1.0
    else:
        raise ValueError("transform must be 'hartley' or 'cosine'")
    return c * r[:, None] * T
