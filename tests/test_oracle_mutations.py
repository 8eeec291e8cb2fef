"""Planted mistakes in the oracle must be caught by its pins (CPU only).

Each case patches one plausible error into a copy of an oracle routine and checks that
the corresponding pin of test_oracle_pins.py then fails.
"""
import math

import numpy as np
import pytest

import synth
from oracle import householder as hh
from oracle import kernels as kk
from oracle import lowrank as lr
from oracle import omega as om
from oracle import sketch as sk
from oracle import tsqr as ts


def _dense_check(f, O, Y, tau):
    n = Y.shape[0]
    A = synth.rhs(n, 2, 1).astype(np.float64)
    Kt = tau * np.eye(n) + Y @ np.linalg.solve(O.T @ Y, Y.T)
    Xd = np.linalg.solve(Kt, A)
    return np.linalg.norm(lr.solve(f, A) - Xd) / np.linalg.norm(Xd) < 1e-6


def _setup(n=256, d=32, tau=1e-4):
    pts = synth.points(n, 2, 0).astype(np.float64)
    O = om.omega_matrix(n, d, 0)
    Y = sk.sketch(pts, kk.SE, 0.2, 1.0, O)
    return O, Y, tau


def test_unmutated_factor_passes():
    O, Y, tau = _setup()
    assert _dense_check(lr.factorise(Y, O, tau, 64), O, Y, tau)


def test_dropped_nugget_term_in_core_is_caught():
    O, Y, tau = _setup()
    f = lr.factorise(Y, O, tau, 64)
    f.Cp = f.R.T.copy()                       # mistake: C' = R^T (tau B dropped)
    f.lu_C = lr.lu_factor(f.Cp)
    assert not _dense_check(f, O, Y, tau)


def test_transposed_b_is_caught():
    O, Y, tau = _setup()
    f = lr.factorise(Y, O, tau, 64)
    f.B = f.Q.T @ O                           # mistake: Q^T Omega instead of Omega^T Q
    f.Cp = f.R.T + tau * f.B
    f.lu_B, f.lu_C = lr.lu_factor(f.B), lr.lu_factor(f.Cp)
    assert not _dense_check(f, O, Y, tau)


def test_wrong_hadamard_pattern_is_caught(monkeypatch):
    def bad(k, p):
        k = np.asarray(k, dtype=np.uint64)
        p = np.asarray(p, dtype=np.uint64)
        return np.where((np.bitwise_count(k | p) & np.uint8(1)) == 0, 1.0, -1.0)
    monkeypatch.setattr(om, "hadamard_entries", bad)
    k = np.arange(8, dtype=np.uint64)
    H = om.hadamard_entries(k[:, None], k[None, :])
    Hs = np.array([[1.0, 1.0], [1.0, -1.0]])
    while Hs.shape[0] < 8:
        Hs = np.block([[Hs, Hs], [Hs, -Hs]])
    assert not np.array_equal(H, Hs)


def test_swapped_tree_children_are_caught(monkeypatch):
    real = hh.householder_qr

    def swapped(A, *dtype):
        m = A.shape[0]
        if m == 2 * A.shape[1]:               # a tree combine: stack in the wrong order
            d = A.shape[1]
            return real(np.vstack([A[d:], A[:d]]), *dtype)
        return real(A, *dtype)
    monkeypatch.setattr(ts, "householder_qr", swapped)
    Y = np.random.default_rng(0).standard_normal((256, 16))
    t = ts.tsqr(Y, 64)
    Q, R = hh.qr(Y)
    assert np.abs(t["Q"] - Q).max() > 1e-3


def test_dropped_half_in_gradient_is_caught(monkeypatch):
    n, d = 256, 24
    pts = synth.points(n, 2, 1).astype(np.float64)
    y = synth.gp_targets(pts, 0.2, 1.0, 1e-3, seed=1).astype(np.float64)

    def bad_grad(f, yy, Y, Yp, alpha):
        Q = f.Q
        KiQ = lr.solve(f, Q)
        PQ = KiQ - np.outer(alpha, alpha @ Q)
        QtPQ = Q.T @ PQ
        PQBi = lr.lu_solve_t(f.lu_B, PQ.T).T
        M = lr.lu_solve_t(f.lu_B, lr.lu_solve_t(f.lu_B, QtPQ.T).T)
        Ybar = PQBi - f.omega @ M                 # mistake: the 1/2 is missing
        return np.array([np.sum(Ybar * Yp), np.sum(Ybar * Y), 0.0]), Ybar
    monkeypatch.setattr(lr, "grad", bad_grad)

    def F(a):
        return lr.nll_grad(pts, y, kk.SE, math.exp(a), 1.0, 1e-3, d, 3, 64)
    h = 1e-4
    _, g = F(math.log(0.25))
    fd = (F(math.log(0.25) + h)[0] - F(math.log(0.25) - h)[0]) / (2 * h)
    assert abs(g[0] - fd) > 1e-3 * abs(fd)


# ------------------------------------------------------------------ transforms, projection
def test_wrong_cosine_normalisation_is_caught(monkeypatch):
    """s_0 = (2/n)^(1/2) like the other columns (a plausible slip) breaks orthonormality."""
    from oracle import transforms as tr

    def bad(k, p, n):
        k = np.asarray(k, dtype=np.int64)
        p = np.asarray(p, dtype=np.int64)
        return np.sqrt(2.0 / n) * np.cos(np.pi * (((2 * k + 1) * p) % (4 * n)) / (2.0 * n))

    monkeypatch.setattr(tr, "cosine_entries", bad)
    n = 500
    x = np.random.default_rng(0).standard_normal(n)
    k = np.arange(n)
    scipy_fft = pytest.importorskip("scipy.fft")
    assert not np.allclose(bad(k[:, None], k[None, :], n).T @ x, scipy_fft.dct(x, type=2, norm="ortho"))


def test_wrong_hartley_scale_is_caught(monkeypatch):
    """c = 1/n instead of n^(-1/2) breaks the orthonormal columns of Definition 1."""
    from oracle import transforms as tr
    real = tr.hartley_entries
    monkeypatch.setattr(tr, "hartley_entries", lambda k, p, n: real(k, p, n) / np.sqrt(float(n)))
    O = tr.omega_matrix_t(300, 20, 2, "hartley")
    assert np.abs(O.T @ O - np.eye(20)).max() > 1e-3


def test_unsquared_colspace_error_is_caught():
    """Reporting num/den without the square root disagrees with the dense definition."""
    from oracle import projection as pr
    n = 200
    pts = np.random.default_rng(1).random((n, 2))
    K = kk.kernel_matrix(pts, pts, kk.SE, 0.2, 1.0)
    Q, _ = hh.qr(K @ om.omega_matrix(n, 16, 3))
    e = pr.colspace_error(pts, kk.SE, 0.2, 1.0, Q, col_block=50)
    dense = np.linalg.norm(K - Q @ Q.T @ K) / np.linalg.norm(K)
    assert abs(e - dense) <= 1e-12 * dense
    assert abs(e * e - dense) > 1e-6 * dense         # the planted slip would be visible
