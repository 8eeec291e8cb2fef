"""Pins of the oracle's Hartley and cosine forms of Omega (Definition 1, Sec. 3.2) and of the
column-space error and predictive mean (Sec. 3.1, Sec. 4, Sec. 5), all on CPU.

Each pin is something other than the oracle itself: a library transform (numpy FFT, scipy
DCT), an identity the definition forces (orthonormal columns for every n), or a result the
mathematics fixes (exact recovery when rank(K0) <= d; the exact GP mean when K_tilde = K).
"""
import numpy as np
import pytest

from oracle import kernels as okk
from oracle import omega as oom
from oracle import projection as opr
from oracle import transforms as otr
from oracle import householder as ohh


@pytest.mark.parametrize("n", [7, 64, 1000])
def test_hartley_matrix_is_the_fft_combination(n):
    """sum_k x_k cas(2 pi k p / n) = Re(FFT x)_p - Im(FFT x)_p (numpy's FFT uses e^{-i...})."""
    rng = np.random.default_rng(n)
    x = rng.standard_normal(n)
    k = np.arange(n)
    T = otr.hartley_entries(k[:, None], k[None, :], n)
    F = np.fft.fft(x)
    assert np.allclose(T.T @ x, F.real - F.imag, atol=1e-10 * np.abs(x).sum())


@pytest.mark.parametrize("n", [5, 64, 1000])
def test_cosine_matrix_is_the_orthonormal_dct2(n):
    scipy_fft = pytest.importorskip("scipy.fft")
    rng = np.random.default_rng(n + 1)
    x = rng.standard_normal(n)
    k = np.arange(n)
    T = otr.cosine_entries(k[:, None], k[None, :], n)
    assert np.allclose(T.T @ x, scipy_fft.dct(x, type=2, norm="ortho"), atol=1e-12 * np.abs(x).sum())


@pytest.mark.parametrize("transform", ["hartley", "cosine"])
@pytest.mark.parametrize("n,d", [(1000, 48), (777, 272), (64, 64)])
def test_structured_omega_has_orthonormal_columns_for_any_n(transform, n, d):
    """Definition 1 asks for orthonormal columns; these transforms give them without padding."""
    O = otr.omega_matrix_t(n, d, 5, transform)
    assert O.shape == (n, d)
    assert np.abs(O.T @ O - np.eye(d)).max() <= 1e-12


def test_subsample_is_a_uniform_subset_of_the_transform_order():
    n, d = 1000, 100
    hits = np.zeros(n)
    for s in range(200):
        c = otr.subsample_columns_n(n, d, s)
        assert len(np.unique(c)) == d and c.min() >= 0 and c.max() < n and np.all(np.diff(c) > 0)
        hits[c] += 1
    expected = 200 * d / n
    chi2 = float(np.sum((hits - expected) ** 2 / expected))
    assert chi2 < n + 5 * np.sqrt(2 * n)             # about 1 +- 0.22 per degree of freedom


def _exact_rank_points_kernel(n, r, seed):
    """K0 = E D E^T with E an orthonormalised Gaussian n x r and exponentially decaying D
    (the construction of the blocking simulation, Sec. 5)."""
    rng = np.random.default_rng(seed)
    E, _ = np.linalg.qr(rng.standard_normal((n, r)))
    D = np.exp(-0.01 * np.arange(r))
    return (E * D) @ E.T


@pytest.mark.parametrize("transform", ["wht", "hartley", "cosine"])
def test_exact_recovery_of_the_column_space(transform):
    """rank(K0) = r <= d: the sketch's Q spans K0's column space, so ||K - QQ^T K|| = 0."""
    n, r, d = 512, 20, 32
    K = _exact_rank_points_kernel(n, r, 3)
    O = oom.omega_matrix(n, d, 1) if transform == "wht" else otr.omega_matrix_t(n, d, 1, transform)
    Q, _ = ohh.qr(K @ O)
    err = np.linalg.norm(K - Q @ (Q.T @ K)) / np.linalg.norm(K)
    assert err <= 1e-12


def test_colspace_error_matches_its_definition_and_decreases_with_d():
    n = 400
    pts = np.random.default_rng(0).random((n, 2))
    K = okk.kernel_matrix(pts, pts, okk.SE, 0.2, 1.0)
    errs = []
    for d in (8, 16, 32, 64):
        Q, _ = ohh.qr(K @ oom.omega_matrix(n, d, 2))
        e = opr.colspace_error(pts, okk.SE, 0.2, 1.0, Q, col_block=64)
        dense = np.linalg.norm(K - Q @ Q.T @ K) / np.linalg.norm(K)
        assert abs(e - dense) <= 1e-12 * max(dense, 1e-300) + 1e-15
        errs.append(e)
    assert all(a > b for a, b in zip(errs, errs[1:]))    # more columns, smaller error


def test_predictive_mean_is_exact_when_the_kernel_has_rank_at_most_d():
    """With a kernel whose K0 has rank <= d the method's K_tilde is K0 + tau I exactly, so
    mu* = K0(X*, X) (K0 + tau I)^-1 y (the textbook GP mean, by Cholesky)."""
    n, m_new, d, tau = 256, 17, 64, 1e-3
    rng = np.random.default_rng(4)
    pts = rng.random((n, 1)) * 0.02                  # points this close: K0 numerically rank-1-ish
    new = rng.random((m_new, 1)) * 0.02
    ell = 50.0                                        # SE with a huge lengthscale: rank(K0) <= d in FP64
    y = rng.standard_normal(n)
    mu = opr.predictive_mean(pts, y, new, okk.SE, ell, 1.0, tau, d, 0, 128)
    K = okk.kernel_matrix(pts, pts, okk.SE, ell, 1.0) + tau * np.eye(n)
    L = np.linalg.cholesky(K)
    alpha = np.linalg.solve(L.T, np.linalg.solve(L, y))
    mu_exact = okk.kernel_matrix(new, pts, okk.SE, ell, 1.0) @ alpha
    assert np.allclose(mu, mu_exact, rtol=1e-6, atol=1e-6 * np.abs(mu_exact).max())


def test_a_planted_sign_error_in_the_hartley_kernel_is_caught():
    """cos - sin instead of cos + sin (a plausible slip) breaks the FFT pin."""
    n = 64
    rng = np.random.default_rng(9)
    x = rng.standard_normal(n)
    k = np.arange(n)
    a = 2.0 * np.pi * ((k[:, None] * k[None, :]) % n) / n
    wrong = np.cos(a) - np.sin(a)
    F = np.fft.fft(x)
    assert not np.allclose(wrong.T @ x, F.real - F.imag, atol=1e-8)


@pytest.mark.parametrize("A,B", [(4, 8), (16, 2), (1, 32)])
def test_kronecker_split_of_the_walsh_hadamard_product(A, B):
    """H_N = H_A (x) H_B in Sylvester order, so (H_N v)[p_a B + p_b] =
    sum_{k_a} H_A[k_a, p_a] (H_B v_{k_a})[p_b]: the identity a structured fast sketch uses to
    replace the dense Omega by B-point transforms and a signed gather."""
    N = A * B
    rng = np.random.default_rng(A * 100 + B)
    v = rng.standard_normal(N)
    k = np.arange(N)
    dense = oom.hadamard_entries(k[:, None], k[None, :]) @ v
    HB = oom.hadamard_entries(np.arange(B)[:, None], np.arange(B)[None, :])
    HA = oom.hadamard_entries(np.arange(A)[:, None], np.arange(A)[None, :])
    U = v.reshape(A, B) @ HB.T                         # row k_a: the B-point transform of block k_a
    split = (HA.T @ U).reshape(N)                      # output p = p_a * B + p_b
    assert np.allclose(split, dense, atol=1e-12 * np.abs(v).sum())


def test_two_pass_core_equals_dense_projection_and_solves():
    """S = Q^T K0 Q against the dense product; the Woodbury solve and log-determinant against
    LAPACK on the dense tau I + Q S Q^T; exact recovery of (K0 + tau I)^-1 A when
    rank(K0) <= d (the projection then loses nothing)."""
    from oracle import householder as hh
    from oracle import kernels as kk
    from oracle import omega as om
    from oracle import projection as pr
    n, d, tau = 300, 24, 1e-3
    pts = np.random.default_rng(2).random((n, 2))
    K = kk.kernel_matrix(pts, pts, kk.SE, 0.2, 1.3)
    Q, _ = hh.qr(K @ om.omega_matrix(n, d, 5))
    S = pr.two_pass_core(pts, kk.SE, 0.2, 1.3, Q, col_block=64)
    assert np.allclose(S, Q.T @ K @ Q, rtol=0, atol=1e-12 * np.abs(S).max())
    assert np.allclose(S, S.T, atol=1e-12 * np.abs(S).max())
    assert np.linalg.eigvalsh(S).min() > -1e-12 * np.abs(S).max()
    A = np.random.default_rng(3).standard_normal((n, 3))
    Kt = tau * np.eye(n) + Q @ S @ Q.T
    X = pr.two_pass_solve(Q, S, tau, A)
    assert np.linalg.norm(X - np.linalg.solve(Kt, A)) <= 1e-9 * np.linalg.norm(X)
    assert abs(pr.two_pass_logdet(S, tau, n) - np.linalg.slogdet(Kt)[1]) <= 1e-9 * abs(np.linalg.slogdet(Kt)[1])
    # exact rank r <= d: K0 = E D E^T, the two-pass solve is the dense solve of K0 + tau I
    E, _ = np.linalg.qr(np.random.default_rng(4).standard_normal((n, d)))
    K0 = E @ np.diag(np.exp(-0.3 * np.arange(d))) @ E.T
    Q2, _ = hh.qr(K0 @ om.omega_matrix(n, d, 6))
    S2 = Q2.T @ K0 @ Q2
    X2 = pr.two_pass_solve(Q2, S2, tau, A)
    Xd = np.linalg.solve(K0 + tau * np.eye(n), A)
    assert np.linalg.norm(X2 - Xd) <= 1e-8 * np.linalg.norm(Xd)


def test_two_pass_with_transposed_product_is_caught():
    """A slip that uses S Q^T A's transpose order (Q^T A S) breaks the dense check."""
    from oracle import householder as hh
    from oracle import kernels as kk
    from oracle import omega as om
    from oracle import projection as pr
    n, d, tau = 200, 16, 1e-2
    pts = np.random.default_rng(7).random((n, 2))
    K = kk.kernel_matrix(pts, pts, kk.SE, 0.25, 1.0)
    Q, _ = hh.qr(K @ om.omega_matrix(n, d, 1))
    S = Q.T @ K @ Q
    A = np.random.default_rng(8).standard_normal((n, d))
    V = np.linalg.solve(tau * np.eye(d) + S, (Q.T @ A) @ S)
    bad = (A - Q @ V) / tau
    good = pr.two_pass_solve(Q, S, tau, A)
    assert np.linalg.norm(bad - good) > 1e-3 * np.linalg.norm(good)


def test_gaussian_omega_is_standard_normal_and_scaled():
    """The Gaussian projection's entries pass a Kolmogorov-Smirnov test against the standard
    normal (after the 1/sqrt(n) scale is undone), are independent across entries (lag-1
    correlation), and its columns are nearly orthonormal for large n."""
    from scipy import stats
    from oracle import omega as om
    n, d = 4000, 64
    O = om.gaussian_omega(n, d, 5)
    z = (O * np.sqrt(n)).ravel()
    assert stats.kstest(z, "norm").pvalue > 1e-3
    assert abs(np.corrcoef(z[:-1], z[1:])[0, 1]) < 0.02
    G = O.T @ O
    assert np.abs(np.diag(G) - 1.0).max() < 0.1 and np.abs(G - np.diag(np.diag(G))).max() < 0.1
    assert not np.array_equal(O, om.gaussian_omega(n, d, 6))
