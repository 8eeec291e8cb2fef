"""Column-space sketch K_hat = K Omega (Sec. 3.1, Sec. 3.3), FP64.  Test infrastructure.

The sketch uses the noise-free kernel matrix K0 = var * rho(X, X): the nugget tau enters
only through the low-rank solve (reading; the paper never writes a nugget).  K0 is built
explicitly, one block of rows at a time, and multiplied by the explicit Omega with a
plain matmul.
"""
import numpy as np

from .kernels import kernel_matrix, dkernel_matrix


def sketch_rows(points, rows, kind, ell, var, omega, derivative=False):
    """Rows `rows` of Y = K0 Omega (or of dK0/dlog(l) Omega when derivative=True)."""
    pts = np.asarray(points, dtype=np.float64)
    f = dkernel_matrix if derivative else kernel_matrix
    Krows = f(pts[np.asarray(rows)], pts, kind, ell, var)
    return Krows @ omega


def sketch(points, kind, ell, var, omega, derivative=False, row_block=512):
    pts = np.asarray(points, dtype=np.float64)
    n = pts.shape[0]
    Y = np.empty((n, omega.shape[1]))
    for r0 in range(0, n, row_block):
        rows = np.arange(r0, min(n, r0 + row_block))
        Y[rows] = sketch_rows(pts, rows, kind, ell, var, omega, derivative)
    return Y


def sketch_dense(K, omega):
    """Y = K Omega for an explicitly given kernel matrix."""
    return np.asarray(K, dtype=np.float64) @ omega
