"""The structured random matrix Omega = c R T P of Definition 1 (Sec. 3.2) with T the
Walsh-Hadamard matrix of the Sylvester recursion H_n = [[H, H], [H, -H]], H_2 = [[1, 1],
[1, -1]] (Sec. 3.2).  Test infrastructure (see the package docstring).

Readings (the paper fixes none of these):
  * T = H_N unnormalised and c = N^(-1/2), so that for N = n the columns of Omega are
    orthonormal as Definition 1 requires.
  * H_N[k, p] = (-1)^popcount(k & p) with 0-based indices: the entry pattern that the
    recursion produces (pinned against the recursion itself in the tests).
  * The Walsh-Hadamard matrix exists only for powers of two (Sec. 3.2).  For other n,
    N = 2^ceil(log2 n) and Omega is rows 0..n-1 of N^(-1/2) R H_N P (the kernel matrix
    zero-padded to order N); its columns are then only nearly orthonormal.
  * R: r_k = +1 when bit 0 of Philox word 0 at (index k, stream 0) is 0, else -1.
  * P: for every candidate column c < N draw key_c = (word0 << 32) | word1 of Philox at
    (index c, stream 1); P holds the d candidates with the smallest keys (ties go to the
    smaller c), in ascending order of c.  This is a uniform d-subset of [0, N).
"""
import numpy as np

from .philox import philox4x32_10


def padded_order(n):
    """N = the smallest power of two >= n."""
    n = int(n)
    return 1 << max(0, (n - 1).bit_length())


def rademacher_signs(n, seed):
    """Diagonal of R as +-1 (float64), Definition 1."""
    w0, _, _, _ = philox4x32_10(np.arange(n, dtype=np.uint64), 0, seed)
    return np.where((w0 & np.uint64(1)) == 0, 1.0, -1.0)


def subsample_columns(n, d, seed):
    """Column subsample P of Definition 1: d distinct indices in [0, N), ascending."""
    N = padded_order(n)
    if not (0 < d <= N):
        raise ValueError("need 0 < d <= N")
    cand = np.arange(N, dtype=np.uint64)
    w0, w1, _, _ = philox4x32_10(cand, 1, seed)
    keys = (w0 << np.uint64(32)) | w1
    order = np.lexsort((cand, keys))        # primary key: keys, ties: smaller c
    return np.sort(order[:d]).astype(np.int64)


def hadamard_entries(k, p):
    """H_N[k, p] = (-1)^popcount(k & p)  (broadcasting)."""
    k = np.asarray(k, dtype=np.uint64)
    p = np.asarray(p, dtype=np.uint64)
    par = np.bitwise_count(k & p) & np.uint8(1)
    return np.where(par == 0, 1.0, -1.0)


def omega_scale(n):
    return 1.0 / np.sqrt(float(padded_order(n)))


def omega_rows(rows, n, d, seed, signs=None, cols=None):
    """Rows `rows` of Omega (len(rows) x d, float64)."""
    rows = np.asarray(rows, dtype=np.int64)
    if signs is None:
        signs = rademacher_signs(n, seed)
    if cols is None:
        cols = subsample_columns(n, d, seed)
    H = hadamard_entries(rows[:, None].astype(np.uint64), cols[None, :].astype(np.uint64))
    return omega_scale(n) * signs[rows][:, None] * H


def omega_matrix(n, d, seed):
    """Omega = c R H_N P restricted to rows 0..n-1 (n x d, float64)."""
    return omega_rows(np.arange(n), n, d, seed)


def gaussian_omega(n, d, seed):
    """The scaled Gaussian projection the paper compares with (Sec. 2 and Sec. 5.1: "a matrix
    with scaled iid standard Gaussian entries"): Omega[k, j] = z_kj / sqrt(n), z_kj standard
    normal.  Reading (the paper fixes neither the generator nor the scale): z_kj by the
    Box-Muller transform of the Philox4x32-10 words 0 and 1 at counter (k d + j, stream 8):
    u = (w + 1/2) / 2^32, z = sqrt(-2 ln u_0) cos(2 pi u_1); the scale 1/sqrt(n) gives columns of
    about unit norm (Omega's scale changes neither Q_hat nor K_N)."""
    idx = np.arange(n * d, dtype=np.uint64)
    w0, w1, _, _ = philox4x32_10(idx, 8, seed)
    u0 = (w0.astype(np.float64) + 0.5) / 4294967296.0
    u1 = (w1.astype(np.float64) + 0.5) / 4294967296.0
    z = np.sqrt(-2.0 * np.log(u0)) * np.cos(2.0 * np.pi * u1)
    return (z / np.sqrt(float(n))).reshape(n, d)
