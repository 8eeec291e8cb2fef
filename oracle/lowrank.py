"""Low-rank solve, likelihood and gradient, FP64.  Test infrastructure.

The paper evaluates K^-1 A through a QR decomposition as R^-1 Q^T A (Sec. 1) and
projects K onto the sketch's column space, P_Khat K = R_k^-1 Q_k^T K (proof of
Theorem 3).  It writes no nugget, no likelihood and no gradient; the readings below
complete it for the Gaussian-likelihood use it targets (Abstract, Sec. 1):

  K0 = var * rho(X, X),  K = K0 + tau I,  Y = K0 Omega = Q R (TSQR),  W = Omega^T Y.
  K_N = Y W^-1 Y^T (single-pass Nystrom); with B = Omega^T Q one has W = B R, so
  K_N = Q C Q^T with C = B^-1 R^T, and K_tilde = tau I + K_N.
  Woodbury with Q^T Q = I:  K_tilde^-1 A = tau^-1 (A - Q C'^-1 R^T Q^T A),
  C' = R^T + tau B.  Neither R nor W is ever inverted.
  logdet K_tilde = (n - d) ln tau + ln|det C'| - ln|det B|.
  NLL = 1/2 y^T alpha + 1/2 logdet K_tilde + n/2 ln(2 pi),  alpha = K_tilde^-1 y.
  Gradient: dNLL = 1/2 tr(P dK_tilde), P = K_tilde^-1 - alpha alpha^T; through
  K_N = Y W^-1 Y^T this is <Ybar, dY> with
  Ybar = P Q B^-1 - 1/2 Omega B^-T (Q^T P Q) B^-1,
  d/dlog(l) = <Ybar, dK0/dlog(l) Omega>, d/dlog(var) = <Ybar, Y>,
  d/dlog(tau) = 1/2 tau (tr K_tilde^-1 - alpha^T alpha),
  tr K_tilde^-1 = (n - d)/tau + tr(C'^-1 B).
  Refinement: X <- X + K_tilde^-1 (A - K_tilde X), K_tilde X = tau X + Q B^-1 R^T Q^T X.
"""
import numpy as np

from .omega import omega_matrix
from .sketch import sketch
from .tsqr import tsqr


# ---------------------------------------------------------------- dense LU (own code)
def lu_factor(M):
    """LU with partial pivoting: M[piv] = L U (L unit lower, packed with U)."""
    A = np.array(M, dtype=np.float64, copy=True)
    n = A.shape[0]
    piv = np.arange(n)
    for j in range(n):
        p = j + int(np.argmax(np.abs(A[j:, j])))
        if p != j:
            A[[j, p]] = A[[p, j]]
            piv[[j, p]] = piv[[p, j]]
        if A[j, j] == 0.0:
            raise np.linalg.LinAlgError("singular matrix in lu_factor")
        A[j + 1:, j] /= A[j, j]
        A[j + 1:, j + 1:] -= np.outer(A[j + 1:, j], A[j, j + 1:])
    return A, piv


def _forward_unit(L, B):
    X = np.array(B, dtype=np.float64, copy=True)
    for i in range(L.shape[0]):
        X[i] -= L[i, :i] @ X[:i]
    return X


def _backward(U, B):
    X = np.array(B, dtype=np.float64, copy=True)
    for i in reversed(range(U.shape[0])):
        X[i] = (X[i] - U[i, i + 1:] @ X[i + 1:]) / U[i, i]
    return X


def lu_solve(lu, B):
    """Solve M X = B."""
    A, piv = lu
    return _backward(A, _forward_unit(A, np.asarray(B, dtype=np.float64)[piv]))


def lu_solve_t(lu, B):
    """Solve M^T X = B  (M^T = U^T L^T P)."""
    A, piv = lu
    B = np.asarray(B, dtype=np.float64)
    n = A.shape[0]
    Z = np.array(B, copy=True)
    for i in range(n):                              # U^T z = B (lower triangular)
        Z[i] = (Z[i] - A[:i, i] @ Z[:i]) / A[i, i]
    for i in reversed(range(n)):                    # L^T w = z (unit upper)
        Z[i] -= A[i + 1:, i] @ Z[i + 1:]
    X = np.empty_like(Z)
    X[piv] = Z
    return X


def lu_logabsdet(lu):
    return float(np.sum(np.log(np.abs(np.diag(lu[0])))))


# ---------------------------------------------------------------- factorisation
class Factor:
    """Q_hat, R, B = Omega^T Q, C' = R^T + tau B and their LUs."""

    def __init__(self, Q, R, omega, tau):
        self.Q, self.R, self.omega, self.tau = Q, R, omega, float(tau)
        self.n, self.d = Q.shape
        self.B = omega.T @ Q
        self.Cp = R.T + self.tau * self.B
        self.lu_B = lu_factor(self.B)
        self.lu_C = lu_factor(self.Cp)

    def logdet(self):
        return ((self.n - self.d) * np.log(self.tau) + lu_logabsdet(self.lu_C)
                - lu_logabsdet(self.lu_B))


def factorise(Y, omega, tau, block_rows, leaf_dtype=np.float64):
    t = tsqr(Y, block_rows, leaf_dtype)
    return Factor(t["Q"], t["R"], omega, tau)


def solve(f, A):
    """K_tilde^-1 A = tau^-1 (A - Q C'^-1 R^T Q^T A)."""
    A = np.asarray(A, dtype=np.float64)
    Z = f.Q.T @ A
    V = lu_solve(f.lu_C, f.R.T @ Z)
    return (A - f.Q @ V) / f.tau


def apply_ktilde(f, X):
    """K_tilde X = tau X + Q B^-1 R^T Q^T X."""
    X = np.asarray(X, dtype=np.float64)
    return f.tau * X + f.Q @ lu_solve(f.lu_B, f.R.T @ (f.Q.T @ X))


def solve_refined(f, A, steps=1):
    X = solve(f, A)
    for _ in range(steps):
        X = X + solve(f, np.asarray(A, dtype=np.float64) - apply_ktilde(f, X))
    return X


def nll(f, y, refine_steps=1):
    y = np.asarray(y, dtype=np.float64).reshape(-1)
    alpha = solve_refined(f, y[:, None], refine_steps)[:, 0]
    return 0.5 * y @ alpha + 0.5 * f.logdet() + 0.5 * f.n * np.log(2.0 * np.pi), alpha


def grad(f, y, Y, Yprime, alpha):
    """Gradient of the NLL with respect to (log l, log var, log tau)."""
    y = np.asarray(y, dtype=np.float64).reshape(-1)
    Q, tau = f.Q, f.tau
    KiQ = solve(f, Q)                                   # K_tilde^-1 Q
    PQ = KiQ - np.outer(alpha, alpha @ Q)
    QtPQ = Q.T @ PQ
    PQBi = lu_solve_t(f.lu_B, PQ.T).T                   # P Q B^-1
    M = lu_solve_t(f.lu_B, lu_solve_t(f.lu_B, QtPQ.T).T)  # B^-T (Q^T P Q) B^-1
    Ybar = PQBi - 0.5 * f.omega @ M
    g_ell = float(np.sum(Ybar * Yprime))
    g_var = float(np.sum(Ybar * Y))
    tr_ki = (f.n - f.d) / tau + float(np.trace(lu_solve(f.lu_C, f.B)))
    g_tau = 0.5 * tau * (tr_ki - alpha @ alpha)
    return np.array([g_ell, g_var, g_tau]), Ybar


# ---------------------------------------------------------------- full pipelines
def kinv_a(points, A, kind, ell, var, tau, d, seed, block_rows, refine_steps=1):
    """K_tilde^-1 A by sketch, TSQR and low-rank solve (Sec. 3, end to end)."""
    pts = np.asarray(points, dtype=np.float64)
    omega = omega_matrix(pts.shape[0], d, seed)
    Y = sketch(pts, kind, ell, var, omega)
    f = factorise(Y, omega, tau, block_rows)
    return solve_refined(f, A, refine_steps), f, Y


def nll_grad(points, y, kind, ell, var, tau, d, seed, block_rows, refine_steps=1):
    pts = np.asarray(points, dtype=np.float64)
    omega = omega_matrix(pts.shape[0], d, seed)
    Y = sketch(pts, kind, ell, var, omega)
    Yp = sketch(pts, kind, ell, var, omega, derivative=True)
    f = factorise(Y, omega, tau, block_rows)
    val, alpha = nll(f, y, refine_steps)
    g, _ = grad(f, y, Y, Yp, alpha)
    return val, g
