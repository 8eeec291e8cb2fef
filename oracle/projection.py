"""The paper's accuracy measure and the Gaussian-process prediction, FP64.  Test
infrastructure (see the package docstring).

  * Column-space error (Sec. 3.1, Sec. 4 Theorem 3): ||K - Q Q^T K||_F / ||K||_F, Q an
    orthonormal basis of the sketch K Omega (here K = K0, the noise-free kernel matrix).
    Evaluated as written, one column block of K0 at a time.
  * Predictive mean at new points X* (the prediction task of the data example, Sec. 5):
    mu* = K0(X*, X) K_tilde^-1 y, with K_tilde^-1 y from the method's low-rank solve.
  * Two-pass core (reading: the projection P_Khat K = Q Q^T K of the proof of Theorem 3,
    made symmetric): S = Q^T K0 Q from a second pass over K0, K0 ~ Q S Q^T, and the solve
    with tau I + Q S Q^T by Woodbury.  Unlike the single-pass core it needs no inverse of
    Omega^T Y and stays positive semi-definite.
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


def two_pass_core(points, kind, ell, var, Q, col_block=512):
    """S = Q^T K0 Q (d x d), the projection of K0 onto the sketch's column space (the second
    pass over K0 that the paper's P_Khat K of Theorem 3's proof implies), with K0 built one
    column block at a time.  K0 ~ Q S Q^T is then the two-pass low-rank approximation."""
    pts = np.asarray(points, dtype=np.float64)
    Q = np.asarray(Q, dtype=np.float64)
    n = pts.shape[0]
    W = np.empty_like(Q)
    for c0 in range(0, n, col_block):
        Kb = kernel_matrix(pts, pts[c0:c0 + col_block], kind, ell, var)   # n x b column block
        W[c0:c0 + col_block] = Kb.T @ Q                                    # rows of K0 Q (K0 symmetric)
    return Q.T @ W


def two_pass_solve(Q, S, tau, A):
    """(tau I + Q S Q^T)^-1 A for orthonormal Q (Woodbury):
    tau^-1 (A - Q (tau I + S)^-1 S Q^T A)."""
    A = np.asarray(A, dtype=np.float64)
    Z = Q.T @ A
    d = S.shape[0]
    V = np.linalg.solve(tau * np.eye(d) + S, S @ Z)
    return (A - Q @ V) / tau


def two_pass_logdet(S, tau, n):
    """log det (tau I + Q S Q^T) = (n - d) ln tau + ln det (tau I + S)."""
    d = S.shape[0]
    sign, ld = np.linalg.slogdet(tau * np.eye(d) + S)
    return (n - d) * np.log(tau) + ld
