"""The paper's accuracy measure and the Gaussian-process prediction, FP64.  Test
infrastructure (see the package docstring).

  * Column-space error (Sec. 3.1, Sec. 4 Theorem 3): ||K - Q Q^T K||_F / ||K||_F, Q an
    orthonormal basis of the sketch K Omega (here K = K0, the noise-free kernel matrix).
    Evaluated as written, one column block of K0 at a time.
  * Predictive mean at new points X* (the prediction task of the data example, Sec. 5):
    mu* = K0(X*, X) K_tilde^-1 y, with K_tilde^-1 y from the method's low-rank solve.
"""
import numpy as np

from .kernels import kernel_matrix
from .lowrank import factorise, solve_refined
from .omega import omega_matrix
from .sketch import sketch


def colspace_error(points, kind, ell, var, Q, col_block=512):
    """||K0 - Q Q^T K0||_F / ||K0||_F for K0 = var * rho(points, points)."""
    pts = np.asarray(points, dtype=np.float64)
    Q = np.asarray(Q, dtype=np.float64)
    n = pts.shape[0]
    num = 0.0
    den = 0.0
    for c0 in range(0, n, col_block):
        Kb = kernel_matrix(pts, pts[c0:c0 + col_block], kind, ell, var)     # n x b column block
        E = Kb - Q @ (Q.T @ Kb)
        num += float(np.sum(E * E))
        den += float(np.sum(Kb * Kb))
    return np.sqrt(num / den)


def predictive_mean(points, y, new_points, kind, ell, var, tau, d, seed, block_rows, refine_steps=1,
                    omega=None):
    """mu* = K0(X*, X) K_tilde^-1 y, the method's K_tilde (sketch, TSQR, low-rank solve)."""
    pts = np.asarray(points, dtype=np.float64)
    n = pts.shape[0]
    O = omega_matrix(n, d, seed) if omega is None else omega
    Y = sketch(pts, kind, ell, var, O)
    f = factorise(Y, O, tau, block_rows)
    alpha = solve_refined(f, np.asarray(y, dtype=np.float64).reshape(n, 1), refine_steps)[:, 0]
    Ks = kernel_matrix(np.asarray(new_points, dtype=np.float64), pts, kind, ell, var)
    return Ks @ alpha
