"""Householder QR, FP64, unblocked.  Test infrastructure (see the package docstring).

The paper factors every block with a QR decomposition (Sec. 3.3, Eq. 1) and names
Householder-based QR as its tool (Sec. 1).  This is the textbook column-by-column
Householder triangularisation (Golub & Van Loan, Alg. 5.2.1; Trefethen & Bau,
Alg. 10.1).  Reflector convention (reading): for the column x below the diagonal,
v = x + sign(x_1) ||x|| e_1 with sign(0) = +1, scaled so that v_1 = 1, and
tau = 2 / (v^T v); then H x = -sign(x_1) ||x|| e_1.  R is upper triangular (the paper
calls it lower at Sec. 1 and upper at Sec. 3.3; upper is used).  `normalise` makes
diag(R) >= 0 by flipping rows of R and the matching columns of Q, which makes a
full-rank QR unique.
"""
import numpy as np


def house(x, dtype=np.float64):
    """Return (v, tau, r) with (I - tau v v^T) x = r e_1 and v[0] = 1."""
    x = np.asarray(x, dtype=dtype)
    normx = np.sqrt(np.dot(x, x))
    v = np.zeros_like(x)
    v[0] = 1.0
    if normx == 0.0:
        return v, dtype(0.0), dtype(0.0)
    s = dtype(1.0) if x[0] >= 0.0 else dtype(-1.0)
    head = x[0] + s * normx
    v[1:] = x[1:] / head
    tau = dtype(2.0) / np.dot(v, v)
    return v, tau, -s * normx


def householder_qr(A, dtype=np.float64):
    """QR of an m x k matrix (m >= k).  Returns (V, tau, R): V is m x k unit lower
    trapezoidal (the reflectors), tau the k scalars, R the k x k upper triangle.
    `dtype` is the working precision (FP64 unless a floor of a lower-precision
    factorisation is wanted: float32 runs the same steps with every operation rounded
    to FP32)."""
    A = np.array(A, dtype=dtype, copy=True)
    m, k = A.shape
    if m < k:
        raise ValueError("householder_qr needs at least as many rows as columns")
    V = np.zeros((m, k), dtype=dtype)
    tau = np.zeros(k, dtype=dtype)
    for j in range(k):
        v, t, r = house(A[j:, j], dtype)
        w = v @ A[j:, j:]
        A[j:, j:] -= t * np.outer(v, w)
        A[j, j] = r
        A[j + 1:, j] = 0.0
        V[j:, j] = v
        tau[j] = t
    return V, tau, np.triu(A[:k, :k])


def apply_q(V, tau, B):
    """Q B with Q = H_0 H_1 ... H_{k-1} (B has m rows), in the reflectors' precision."""
    B = np.array(B, dtype=V.dtype, copy=True)
    for j in reversed(range(V.shape[1])):
        v = V[j:, j]
        B[j:] -= tau[j] * np.outer(v, v @ B[j:])
    return B


def apply_qt(V, tau, B):
    """Q^T B."""
    B = np.array(B, dtype=np.float64, copy=True)
    for j in range(V.shape[1]):
        v = V[j:, j]
        B[j:] -= tau[j] * np.outer(v, v @ B[j:])
    return B


def thin_q(V, tau):
    """The first k columns of Q (m x k)."""
    m, k = V.shape
    return apply_q(V, tau, np.eye(m, k, dtype=V.dtype))


def normalise(Q, R):
    """Flip signs so that diag(R) >= 0 (a zero diagonal entry counts as +)."""
    s = np.where(np.diag(R) < 0.0, -1.0, 1.0)
    return Q * s[None, :], R * s[:, None]


def qr(A):
    """Direct (unblocked) QR with diag(R) >= 0: returns thin Q and R."""
    V, tau, R = householder_qr(A)
    return normalise(thin_q(V, tau), R)
