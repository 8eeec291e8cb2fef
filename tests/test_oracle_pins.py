"""Pins of the FP64 oracle to facts the paper and the mathematics fix (CPU only).

Each test checks the oracle against something other than itself: numbers printed in
the paper, a different construction of the same object, a library routine for a
special case, brute force on tiny inputs, or finite differences.
"""
import math
import os

import numpy as np
import pytest

import synth
from oracle import householder as hh
from oracle import kernels as kk
from oracle import lowrank as lr
from oracle import omega as om
from oracle import sketch as sk
from oracle import tsqr as ts

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _read_table(name):
    rows = []
    with open(os.path.join(GOLDEN, name)) as fh:
        for line in fh:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            parts = line.split()
            rows.append((int(parts[0]), parts[1:]))
    return rows


def _cond_numbers(K, ms):
    ev = np.sort(np.linalg.eigvalsh(K))[::-1]
    return {m: ev[0] / ev[m - 1] for m in ms}


def _check_entry(value, printed):
    if printed.startswith("E"):
        k = int(printed[1:])
        # O(10^k): the paper truncates; one entry (SE theta2 = 0.05, m = 10) is rounded up
        assert 10.0 ** (k - 1) <= value < 10.0 ** (k + 1), (value, printed)
    else:
        assert abs(value - float(printed)) < 0.0101, (value, printed)


GRID = np.linspace(0.0, 1.0, 100)
R100 = np.abs(GRID[:, None] - GRID[None, :])


def test_table1_squared_exponential():
    """Table 1 (Sec. 5.1): SE condition numbers, incl. the exact 29.89 at theta2 = 10."""
    thetas = [0.05, 0.5, 1.0, 1.5, 2.0, 10.0]
    rows = _read_table("table1_se_condition_numbers.txt")
    for ci, t2 in enumerate(thetas):
        cn = _cond_numbers(kk.se_theta(R100, 1.0, t2), [m for m, _ in rows])
        for m, entries in rows:
            _check_entry(cn[m], entries[ci])


def test_table2_matern():
    """Table 2 (Sec. 5.1), with the 2 sqrt(nu) Bessel argument (exact 38.18 at nu = 1/2)."""
    nus = [0.5, 1.0, 1.5, 2.0, 2.5, 3.0]
    rows = _read_table("table2_matern_condition_numbers.txt")
    for ci, nu in enumerate(nus):
        K = kk.matern_bessel(R100, 1.0, 1.0, nu, arg_scale=2.0 * math.sqrt(nu))
        cn = _cond_numbers(K, [m for m, _ in rows])
        for m, entries in rows:
            _check_entry(cn[m], entries[ci])


def test_table2_printed_argument_does_not_reproduce():
    """The printed sqrt(2 nu) argument gives 59.34, not 38.18 (the reading is needed)."""
    K = kk.matern_bessel(R100, 1.0, 1.0, 0.5)
    assert abs(_cond_numbers(K, [5])[5] - 59.34) < 0.01


def test_matern52_closed_form_is_the_bessel_family_member():
    """Matern-5/2 closed form == theta1/(Gamma(nu) 2^(nu-1)) z^nu K_nu(z), nu = 5/2."""
    r = np.linspace(0.0, 2.0, 301)
    for ell in (0.05, 0.15, 1.0):
        a = kk.rho(r, kk.MATERN52, ell, 1.7)
        b = kk.matern_bessel(r, 1.7, ell, 2.5)
        assert np.allclose(a, b, rtol=1e-12, atol=1e-15)


def test_se_lengthscale_form_matches_theta_form():
    r = np.linspace(0.0, 1.5, 101)
    for ell in (0.1, 0.2, 0.7):
        assert np.allclose(kk.rho(r, kk.SE, ell, 2.0), kk.se_theta(r, 2.0, 1.0 / (2 * ell * ell)),
                           rtol=1e-12, atol=0)


def test_kernel_derivatives_by_finite_differences():
    r = np.linspace(0.0, 1.0, 57)
    for kind in (kk.SE, kk.MATERN52):
        ell, h = 0.3, 1e-5
        fd = (kk.rho(r, kind, ell * math.exp(h), 1.3) - kk.rho(r, kind, ell * math.exp(-h), 1.3)) / (2 * h)
        assert np.allclose(kk.drho_dlogell(r, kind, ell, 1.3), fd, rtol=1e-7, atol=1e-10)


def _sylvester(N):
    H = np.array([[1.0, 1.0], [1.0, -1.0]])          # H_2 of Sec. 3.2
    while H.shape[0] < N:
        H = np.block([[H, H], [H, -H]])
    return H


@pytest.mark.parametrize("N", [2, 4, 8, 32, 128])
def test_hadamard_entries_follow_the_sylvester_recursion(N):
    k = np.arange(N, dtype=np.uint64)
    H = om.hadamard_entries(k[:, None], k[None, :])
    assert np.array_equal(H, _sylvester(N))
    assert np.array_equal(H, H.T)
    assert np.array_equal(H @ H.T, N * np.eye(N))


@pytest.mark.parametrize("n,d", [(64, 16), (1024, 64), (4096, 128)])
def test_omega_columns_orthonormal_for_powers_of_two(n, d):
    O = om.omega_matrix(n, d, seed=3)
    assert np.abs(O.T @ O - np.eye(d)).max() < 1e-13          # Definition 1
    assert set(np.unique(np.abs(O))) == {1.0 / math.sqrt(n)}


def test_omega_non_power_of_two_is_the_truncated_padded_matrix():
    n, d = 1000, 32
    cols = om.subsample_columns(n, d, 5)
    assert cols.max() < 1024 and len(np.unique(cols)) == d and np.all(np.diff(cols) > 0)
    full_signs = om.rademacher_signs(1024, 5)
    Ofull = (1.0 / 32.0) * full_signs[:, None] * om.hadamard_entries(
        np.arange(1024, dtype=np.uint64)[:, None], cols[None, :].astype(np.uint64))
    assert np.array_equal(om.omega_matrix(n, d, 5), Ofull[:n])


def test_philox_matches_the_published_known_answers():
    """The generator behind R and P (Definition 1 draws them at random; Philox4x32-10 is the
    reading) reproduces the known-answer vectors published with it, word for word."""
    from oracle.philox import philox4x32_10, philox4x32_10_block
    path = os.path.join(GOLDEN, "philox4x32_10_kat.txt")
    rows = [ln.split() for ln in open(path) if ln.strip() and not ln.startswith("#")]
    assert len(rows) == 3
    for r in rows:
        w = [int(x, 16) for x in r]
        out = philox4x32_10_block(w[0], w[1], w[2], w[3], w[4], w[5])
        assert [int(o) for o in out] == w[6:10]
    # the counter layout used for the draws: (index_lo, index_hi, stream, 0), key = seed
    c = philox4x32_10_block(5, 0, 1, 0, 7, 0)
    d = philox4x32_10(np.array([5], dtype=np.uint64), 1, 7)
    assert [int(x) for x in c] == [int(x[0]) for x in d]


def test_rademacher_signs_are_balanced_and_stream_independent():
    n = 1 << 18
    s = om.rademacher_signs(n, 11)
    assert abs(s.sum()) < 5 * math.sqrt(n)                    # binomial, 5 sigma
    s2 = om.rademacher_signs(n, 12)
    assert abs(np.dot(s, s2)) < 5 * math.sqrt(n)              # different seeds uncorrelated
    assert abs(np.dot(s[:-1], s[1:])) < 5 * math.sqrt(n)      # no lag-1 correlation
    assert np.array_equal(s, om.rademacher_signs(n, 11))      # deterministic


def test_subsample_is_a_uniform_subset():
    N, d, trials = 256, 16, 4000
    counts = np.zeros(N)
    for t in range(trials):
        c = om.subsample_columns(N, d, 1000 + t)
        assert len(np.unique(c)) == d
        counts[c] += 1
    expected = trials * d / N
    chi2 = np.sum((counts - expected) ** 2 / expected)
    # chi-square with 255 degrees of freedom: mean 255, sd ~22.6; 6 sd margin
    assert chi2 < 255 + 6 * 22.6


def test_sketch_matches_brute_force():
    n, d = 16, 4
    pts = synth.points(n, 2, 7).astype(np.float64)
    O = om.omega_matrix(n, d, 9)
    Y = sk.sketch(pts, kk.SE, 0.3, 1.5, O, row_block=5)
    for i in range(n):
        for j in range(d):
            acc = 0.0
            for k in range(n):
                r2 = sum((pts[i, t] - pts[k, t]) ** 2 for t in range(2))
                acc += 1.5 * math.exp(-r2 / (2 * 0.3 ** 2)) * O[k, j]
            assert abs(Y[i, j] - acc) < 1e-13


def _rand(m, k, seed=0):
    return np.random.default_rng(seed).standard_normal((m, k))


@pytest.mark.parametrize("m,k", [(40, 40), (200, 17), (333, 64)])
def test_householder_matches_lapack_up_to_signs(m, k):
    A = _rand(m, k, m + k)
    Q, R = hh.qr(A)
    Ql, Rl = np.linalg.qr(A)
    s = np.where(np.diag(Rl) < 0, -1.0, 1.0)
    assert np.allclose(R, Rl * s[:, None], rtol=0, atol=1e-12 * np.abs(R).max())
    assert np.allclose(Q, Ql * s[None, :], atol=1e-12)
    assert np.abs(Q.T @ Q - np.eye(k)).max() < 1e-12
    assert np.abs(Q @ R - A).max() < 1e-13 * np.abs(A).max() * 10
    assert np.all(np.diag(R) >= 0) and np.allclose(R, np.triu(R))


def test_householder_apply_q_and_qt_are_inverse():
    A = _rand(100, 20, 1)
    V, tau, _ = hh.householder_qr(A)
    B = _rand(100, 3, 2)
    assert np.allclose(hh.apply_q(V, tau, hh.apply_qt(V, tau, B)), B, atol=1e-13)


@pytest.mark.parametrize("n,d,b", [(512, 16, 64), (520, 16, 64), (700, 32, 96), (96, 32, 32), (64, 16, 128)])
def test_tsqr_r_equals_direct_r(n, d, b):
    """Sec. 3.3 / Eq. 4: the tree of block QRs yields the QR of the whole matrix."""
    Y = _rand(n, d, n + d + b)
    t = ts.tsqr(Y, b)
    Q, R = hh.qr(Y)
    assert np.abs(t["R"] - R).max() < 1e-12 * np.abs(R).max()
    assert np.abs(t["Q"] - Q).max() < 1e-12
    assert np.abs(t["Q"].T @ t["Q"] - np.eye(d)).max() < 1e-12


def test_tsqr_leaf_ranges_merge_short_tail_and_odd_levels():
    assert ts.leaf_ranges(520, 16, 64)[-1] == (448, 520)      # 8-row tail merged
    assert ts.leaf_ranges(528, 16, 64)[-1] == (512, 528)      # 16-row tail kept
    r = ts.leaf_ranges(130, 16, 64)
    assert r == [(0, 64), (64, 130)]
    t = ts.tsqr(_rand(5 * 64, 16, 3), 64)           # 5 leaves: odd nodes pass up
    assert [len(l) for l in t["levels"]] == [5, 3, 2, 1]


def test_lu_matches_library_solve():
    M = _rand(60, 60, 4) + 3 * np.eye(60)
    lu = lr.lu_factor(M)
    A, piv = lu
    L = np.tril(A, -1) + np.eye(60)
    U = np.triu(A)
    assert np.allclose(M[piv], L @ U, atol=1e-12)
    B = _rand(60, 5, 5)
    assert np.allclose(lr.lu_solve(lu, B), np.linalg.solve(M, B), atol=1e-11)
    assert np.allclose(lr.lu_solve_t(lu, B), np.linalg.solve(M.T, B), atol=1e-11)
    assert abs(lr.lu_logabsdet(lu) - np.linalg.slogdet(M)[1]) < 1e-10


def _problem(n=512, d=48, ell=0.2, kind=kk.SE, tau=1e-6, seed=0):
    pts = synth.points(n, 2, seed).astype(np.float64)
    O = om.omega_matrix(n, d, seed)
    Y = sk.sketch(pts, kind, ell, 1.0, O)
    return pts, O, Y


@pytest.mark.parametrize("kind,tau", [(kk.SE, 1e-6), (kk.MATERN52, 1e-4)])
def test_lowrank_solve_and_logdet_equal_dense_nystrom(kind, tau):
    """tau I + Y W^-1 Y^T built densely and solved by LAPACK == the Woodbury/LU form."""
    pts, O, Y = _problem(kind=kind, tau=tau)
    f = lr.factorise(Y, O, tau, 128)
    A = synth.rhs(512, 4, 1).astype(np.float64)
    W = O.T @ Y
    Kt = tau * np.eye(512) + Y @ np.linalg.solve(W, Y.T)
    Xd = np.linalg.solve(Kt, A)
    X = lr.solve(f, A)
    assert np.linalg.norm(X - Xd) / np.linalg.norm(Xd) < 1e-6
    assert abs(f.logdet() - np.linalg.slogdet(Kt)[1]) < 1e-6 * abs(f.logdet())
    Xr = lr.solve_refined(f, A, 1)
    assert np.linalg.norm(Xr - Xd) / np.linalg.norm(Xd) < 1e-6
    assert np.linalg.norm(lr.apply_ktilde(f, Xr) - A) / np.linalg.norm(A) < 1e-7


@pytest.mark.parametrize("r", [48, 20])
def test_exact_rank_recovery(r):
    """K0 = E D E^T of rank r <= d (the construction of Sec. 5.1) is recovered exactly."""
    n, d, tau = 512, 48, 1e-3
    E, _ = np.linalg.qr(_rand(n, r, 17))
    D = np.exp(-0.01 * np.arange(r)) * 5.0           # exponential decay, Sec. 5.1
    K0 = (E * D) @ E.T
    O = om.omega_matrix(n, d, 2)
    Y = sk.sketch_dense(K0, O)
    f = lr.factorise(Y, O, tau, 128)
    Q = f.Q
    if r == d:
        assert np.linalg.norm(K0 - Q @ (Q.T @ K0)) / np.linalg.norm(K0) < 1e-12
    A = synth.rhs(n, 3, 4).astype(np.float64)
    L = np.linalg.cholesky(K0 + tau * np.eye(n))
    Xc = np.linalg.solve(L.T, np.linalg.solve(L, A))
    X = lr.solve(f, A)
    assert np.linalg.norm(X - Xc) / np.linalg.norm(Xc) < 1e-10


@pytest.mark.parametrize("kind", [kk.SE, kk.MATERN52])
def test_gradient_matches_central_differences(kind):
    n, d = 384, 32
    pts = synth.points(n, 2, 1).astype(np.float64)
    y = synth.gp_targets(pts, 0.2, 1.0, 1e-3, seed=1).astype(np.float64)
    le, lv, lt = math.log(0.25), math.log(1.3), math.log(1e-3)

    def F(a, b, c):
        return lr.nll_grad(pts, y, kind, math.exp(a), math.exp(b), math.exp(c), d, 3, 128)

    v0, g = F(le, lv, lt)
    h = 1e-4
    fd = np.array([(F(le + h, lv, lt)[0] - F(le - h, lv, lt)[0]) / (2 * h),
                   (F(le, lv + h, lt)[0] - F(le, lv - h, lt)[0]) / (2 * h),
                   (F(le, lv, lt + h)[0] - F(le, lv, lt - h)[0]) / (2 * h)])
    assert np.all(np.abs(g - fd) <= 1e-5 * np.maximum(np.abs(fd), 1.0)), (g, fd)


def test_nll_matches_dense_gaussian_density():
    n, d, tau = 256, 32, 1e-3
    pts, O, Y = _problem(n=n, d=d)
    y = synth.gp_targets(pts, 0.2, 1.0, tau, seed=2).astype(np.float64)
    f = lr.factorise(Y, O, tau, 64)
    val, _ = lr.nll(f, y)
    Kt = tau * np.eye(n) + Y @ np.linalg.solve(O.T @ Y, Y.T)
    dense = 0.5 * y @ np.linalg.solve(Kt, y) + 0.5 * np.linalg.slogdet(Kt)[1] + 0.5 * n * math.log(2 * math.pi)
    assert abs(val - dense) < 1e-7 * abs(dense)


def test_projection_error_decreases_with_d():
    """Theorem 3 is qualitative here (its constants are unstated): more columns, less error."""
    n = 512
    pts = synth.points(n, 2, 0).astype(np.float64)
    K0 = kk.kernel_matrix(pts, pts, kk.SE, 0.15, 1.0)
    errs = []
    for d in (8, 16, 32, 64):
        O = om.omega_matrix(n, d, 1)
        Q, _ = hh.qr(K0 @ O)
        errs.append(np.linalg.norm(K0 - Q @ (Q.T @ K0)) / np.linalg.norm(K0))
    assert all(b < a for a, b in zip(errs, errs[1:]))


def test_fp32_householder_matches_lapack_single_precision():
    """The oracle's Householder QR run in FP32 (the floor of FP32 leaves) is the textbook
    algorithm in single precision: its R agrees with LAPACK's single-precision QR up to row
    signs at FP32 accuracy, and its Q is orthonormal to FP32 accuracy, not better."""
    A = np.random.default_rng(4).standard_normal((512, 64))
    V, tau, R = hh.householder_qr(A, np.float32)
    assert V.dtype == np.float32 and R.dtype == np.float32
    R_l = np.linalg.qr(A.astype(np.float32))[1]
    s = np.sign(np.diag(R_l)) * np.sign(np.diag(R))
    err = np.linalg.norm(R.astype(np.float64) - s[:, None] * R_l) / np.linalg.norm(R_l)
    assert err < 1e-5
    R64 = hh.householder_qr(A)[2]
    assert 1e-9 < np.linalg.norm(R.astype(np.float64) - R64) / np.linalg.norm(R64) < 1e-5
    Q = hh.thin_q(V, tau).astype(np.float64)
    orth = np.abs(Q.T @ Q - np.eye(64)).max()
    assert 1e-9 < orth < 1e-5


def test_tsqr_with_fp32_leaves_is_near_the_fp64_tsqr():
    Y = np.random.default_rng(8).standard_normal((2048, 32))
    t64 = ts.tsqr(Y, 512)
    t32 = ts.tsqr(Y, 512, np.float32)
    e = np.linalg.norm(t32["R"] - t64["R"]) / np.linalg.norm(t64["R"])
    assert 1e-9 < e < 1e-5
