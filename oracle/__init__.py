"""FP64 CPU oracle for the low-rank K^-1 A method of "Parallel inversion of huge
covariance matrices" (Banerjee, Vogelstein & Dunson, arXiv:1312.1869).

TEST INFRASTRUCTURE ONLY.  This package is a plain, slow, obviously correct restatement of
what the method computes: the structured random sketch Y = K Omega (Sec. 3.1-3.2,
Definition 1), the blocked tall-skinny Householder QR with its binary tree of R
combines (Sec. 3.3, Eqs. 1-4), and the low-rank solve R^-1 Q^T A (Sec. 1, Sec. 3.3)
in its Nystrom/Woodbury form with a nugget, plus the Gaussian negative log-likelihood
and its gradient (the likelihood evaluation that motivates the method, Abstract and
Sec. 1).  Only the tests, `__graft_entry__.smoke()` and the CPU-baseline leg of
`bench.py` may import it.  It shares no code with the CUDA library and imports
nothing from it; the seeded input generators in `synth/` are the only code both sides
use.

Everything is float64 numpy.  Library primitives (matmul, sort, eigvalsh) serve as steps
where noted; there is no blocking or fusion beyond what the paper states.

Parity status per function (pins live in tests/test_oracle_*.py):
  philox        pinned by the published known-answer vectors of Philox4x32-10, plus
                uniformity and independence of the streams it draws
  kernels       pinned by Tables 1-2 (29.89, 38.18 and the order-of-magnitude rows)
                and by the Bessel form of the Matern kernel at nu = 5/2
  omega         pinned by the Sylvester recursion of Sec. 3.2 and Omega^T Omega = I
  householder   pinned by LAPACK QR (uniqueness up to row signs) and Q^T Q = I
  tsqr          pinned by equality with the direct QR's R
  lowrank       pinned by dense Cholesky/LU solves of tau I + K_N, exact-rank recovery,
                and central finite differences of the NLL
  transforms    (Hartley and cosine forms of Omega, for the structured fast sketch that
                comes next) pinned by numpy's FFT, scipy's orthonormal DCT-II and
                Omega^T Omega = I at orders that are not powers of two
  projection    (column-space error, predictive mean) pinned by the dense definition,
                exact recovery for rank(K0) <= d, and the textbook GP mean by Cholesky
  theory bounds (Theorems 3-4): parity unpinned, constants are not stated in the paper
"""
