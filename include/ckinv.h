/*
 * ckinv.h -- C ABI of the GB300 (sm_103a) library for low-rank K^-1 A with a huge,
 * nearly rank-deficient covariance matrix K, after Banerjee, Vogelstein & Dunson,
 * "Parallel inversion of huge covariance matrices" (arXiv:1312.1869).
 *
 * The paper's problem statement (Sec. 1): evaluate K^-1 A for a symmetric positive
 * definite K of huge order n without forming K^-1, through a QR decomposition,
 * R^-1 Q^T A.  Its method (Sec. 3) has three steps, each an entry point here:
 *   ckinv_sketch  Y = K0 Omega with the structured random Omega = c R T P of
 *                 Definition 1 (Sec. 3.2), T the Walsh-Hadamard matrix (Sec. 3.2);
 *   ckinv_tsqr    blocked tall-skinny QR of Y: per-block Householder QR (Eq. 1) and a
 *                 binary tree of QRs of stacked R factors (Eqs. 2-4);
 *   ckinv_solve   the low-rank solve that applies Q_hat and R to A.
 * ckinv_nll_grad evaluates the Gaussian negative log-likelihood and its gradient, the
 * application the paper names first (Abstract and Sec. 1: Gaussian likelihoods of many points).
 *
 * Conventions shared by every entry point:
 *   - Matrices are column-major; "ld" is the leading dimension in elements.
 *   - Array arguments are DEVICE pointers unless the comment says "host"; the caller
 *     owns them.  ckinv_kinv_a also accepts host pointers (it stages them).
 *   - Calls are asynchronous on `stream` (NULL = the legacy default stream) unless they
 *     return host scalars, which they do after synchronising that stream.
 *   - Every call returns a ckinv_status and never aborts; ckinv_last_error() gives a
 *     one-line description of the last failure on that context.
 *   - A context is not thread-safe: use one per host thread.
 *
 * Definitions used throughout (the paper writes no nugget; tau enters only the solve):
 *   K0 = variance * rho(x_i, x_k)      noise-free kernel matrix,  rho(0) = 1
 *   Omega[k, j] = c r_k (-1)^popcount(k & p_j),  c = N^-1/2, N = 2^ceil(log2 n)
 *   Y = K0 Omega = Q_hat R  (diag(R) >= 0),  B = Omega^T Q_hat,  C' = R^T + tau B
 *   K_tilde = tau I + Y (Omega^T Y)^-1 Y^T        (tau = nugget)
 *   ckinv_solve returns K_tilde^-1 A = tau^-1 (A - Q_hat C'^-1 R^T Q_hat^T A).
 */
#ifndef CKINV_H
#define CKINV_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Same object as cudaStream_t; declared here so that the header needs no CUDA headers. */
typedef struct CUstream_st *ckinv_stream;

typedef enum {
  CKINV_OK = 0,
  CKINV_EINVAL = 1,        /* invalid argument (sizes, null pointers, enum values) */
  CKINV_ENOMEM = 2,        /* device allocation failed */
  CKINV_ECUDA = 3,         /* a CUDA runtime/driver call failed */
  CKINV_ESINGULAR = 4,     /* a zero pivot in an LU factorisation */
  CKINV_ETIMEOUT = 5,      /* a bounded device-side wait ran out */
  CKINV_EUNSUPPORTED = 6   /* valid but unsupported here (device, size limit) */
} ckinv_status;

typedef enum {
  CKINV_SE = 0,            /* rho = exp(-r^2 / (2 l^2)) */
  CKINV_MATERN52 = 1,      /* rho = (1 + sqrt5 r/l + 5 r^2/(3 l^2)) exp(-sqrt5 r/l) */
  CKINV_DENSE = 2          /* K0 is given as a materialised n x n matrix */
} ckinv_kernel_kind;

typedef enum {
  CKINV_FP32 = 0,          /* kernel tile x Omega in FP32 FMA (SIMT) */
  CKINV_BF16 = 1,          /* one BF16 tensor-core product, FP32 accumulation */
  CKINV_BF16X2 = 2,        /* kernel tile split in two BF16 terms (two products) */
  CKINV_BF16X3 = 3,        /* three BF16 terms: FP32-accurate on tensor cores */
  CKINV_FP32_WHT = 4       /* FP32 on the CUDA cores through the fast Walsh-Hadamard transform
                              (Sec. 3.2's structured Omega applied as a transform: per kernel
                              entry log2(1024) additions instead of 2d multiply-adds); needs
                              omega_kind 0 and N >= 1024, else the same as CKINV_FP32 */
} ckinv_precision;

typedef struct {
  int32_t kind;            /* ckinv_kernel_kind */
  int32_t reserved;        /* must be 0 */
  double lengthscale;      /* l > 0 (ignored for CKINV_DENSE) */
  double variance;         /* sigma^2 > 0 (ignored for CKINV_DENSE) */
  double nugget;           /* tau > 0 */
} ckinv_kernel;

typedef struct {
  int64_t n;               /* number of points, n >= d */
  int32_t dim;             /* point dimension, 1..3 (ignored for CKINV_DENSE) */
  int32_t d;               /* sketch width r of Sec. 3, 16 <= d <= 512, d % 16 == 0 */
  int32_t block_rows;      /* TSQR leaf height b (>= d); 0 = automatic */
  int32_t prec;            /* ckinv_precision of the sketch contraction */
  uint64_t seed;           /* seed of the counter-based generator drawing R and P */
  int32_t refine_steps;    /* FP64 iterative-refinement steps of the final solve (0..4) */
  int32_t tree_fp64_levels;/* top levels of the R tree combined in FP64; -1 = all.  Q_hat
                              is formed in the leaves' precision either way */
  int32_t leaf_fp64;       /* 1: per-block Householder (and so the whole tree) in FP64 */
  int32_t omega_kind;      /* T of Omega = c R T P (Definition 1): 0 Walsh-Hadamard (the default,
                              generated from bits on the fly); 1 the scaled Gaussian projection,
                              2 discrete Hartley, 3 discrete cosine (Sec. 5.1's three choices;
                              dense, materialised, for ckinv_sketch / ckinv_tsqr / ckinv_solve /
                              ckinv_kinv_a only) */
} ckinv_plan_desc;

typedef struct ckinv_ctx ckinv_ctx;       /* workspaces, cached Omega, error string */
typedef struct ckinv_factor ckinv_factor; /* R, Q_hat, LU(B), LU(C'), reflectors */

/* Library version string (static storage). */
const char *ckinv_version(void);

/* Number of CUDA kernel launches the library has issued since it was loaded (all
 * contexts and threads); a diagnostic for counting the work of a call. */
unsigned long long ckinv_kernel_launches(void);

/* Create a context on CUDA device `device` (must be sm_103).  *ctx receives the
 * handle; on failure *ctx is NULL and the status says why. */
ckinv_status ckinv_create(ckinv_ctx **ctx, int device);

/* Synchronise the context's device and free everything it owns.  NULL is allowed. */
ckinv_status ckinv_destroy(ckinv_ctx *ctx);

/* One-line description of the last error on this context (static if ctx is NULL). */
const char *ckinv_last_error(const ckinv_ctx *ctx);

/* Synchronise `stream` and report device-detected failures of earlier asynchronous
 * calls on this context as a status, then clear the device error word:
 *   CKINV_ETIMEOUT      a bounded device-side wait ran out (see ckinv_set_wait_limit);
 *   CKINV_EINVAL        a NaN or infinity in the points, A or y (checked on the device);
 *   CKINV_ESINGULAR     a zero, infinite or NaN pivot in LU(B) or LU(C');
 *   CKINV_EUNSUPPORTED  an on-device list overflowed (Omega draw).
 * The paper has no counterpart (error handling of this library). */
ckinv_status ckinv_check(ckinv_ctx *ctx, ckinv_stream stream);

/* Limit, in nanoseconds, of every device-side wait of the tensor-core kernels launched
 * afterwards from this context on another role's progress (a pipeline stage's data, the
 * peer CTA, the accumulator).  When a wait runs out the CTA gives up its tile, waits (one
 * second at most) for its own copies and tensor-core products still in flight, frees its
 * tensor memory and exits; the failure surfaces as CKINV_ETIMEOUT from ckinv_check or from
 * the next call that returns host scalars, and the context stays usable.  0 restores the
 * default of one second; at most 60 s.  Outputs of a call that timed out are undefined.
 * The paper has no counterpart (error handling of this library). */
ckinv_status ckinv_set_wait_limit(ckinv_ctx *ctx, uint64_t nanoseconds);

/* Omega of Definition 1 (Sec. 3.2) as drawn from `seed`:
 *   sign_bits: ceil(n/32) uint32 words; bit (k % 32) of word k/32 is 1 iff r_k = -1;
 *   cols:      d int32 column indices p_0 < ... < p_{d-1} in [0, N).
 * Both device, caller-owned.  Pass NULL for an output that is not wanted.  1 <= n <= 2^31,
 * 1 <= d <= min(N, 4096); P is drawn by a two-level radix select over the N keys. */
ckinv_status ckinv_omega(ckinv_ctx *ctx, int64_t n, int32_t d, uint64_t seed,
                         uint32_t *sign_bits, int32_t *cols, ckinv_stream stream);

/* Omega as a dense n x d FP32 matrix (device, column-major, ldo >= n) of the given kind
 * (0 Walsh-Hadamard, 1 scaled Gaussian, 2 discrete Hartley, 3 discrete cosine; see
 * ckinv_plan_desc.omega_kind), each entry evaluated in FP64 and rounded once:
 *   0: c r_k (-1)^popcount(k & p_j), c = N^-1/2, P over the N = 2^ceil(log2 n) columns;
 *   1: z_kj / sqrt(n), z by Box-Muller from Philox words 0, 1 at (k d + j, stream 8);
 *   2: n^-1/2 r_k cas(2 pi k p_j / n);   3: r_k s_p cos(pi (2k + 1) p_j / (2n)),
 *      s_0 = n^-1/2, s_p = (2/n)^1/2; for 2 and 3 P is drawn over the n columns.
 * Definition 1 (Sec. 3.2) and Sec. 5.1. */
ckinv_status ckinv_omega_matrix(ckinv_ctx *ctx, int64_t n, int32_t d, uint64_t seed, int32_t kind,
                                float *Omega, int64_t ldo, ckinv_stream stream);

/* The same draw as ckinv_omega for callers that cannot allocate device memory (for
 * example a program that reserves all device memory for its own pool up front, or code
 * that must not take the implicit device synchronisation of an allocation).  The paper has
 * no counterpart: this is an interface variant, not part of the method.
 *   Runs on the calling thread's current device; needs no context; calls no allocator.
 *   Its scratch is one fixed device array of about 304 KB per device (a 65536-bin key
 *   histogram, reused by both levels of the column select, room for 4096 candidate
 *   columns, counters), kept until the process exits.
 *   The first call on a device resolves that array's device address (set-up).
 *   Limits: 1 <= n <= 2^31, 1 <= d <= min(512, N); larger sizes return CKINV_EINVAL with a
 *   message in ckinv_last_error(NULL).  The two-level select keeps the candidate list near
 *   d entries (about N / 2^32 keys share its last bin), so the 4096 slots suffice at every
 *   n in range; an overflow would still be reported as CKINV_EUNSUPPORTED.
 *   Every call on a device shares the array: calls whose GPU work overlaps (other streams,
 *   other host threads) race on it and must be serialised by the caller.
 *   Outputs as in ckinv_omega (device, caller-owned).  The call synchronises `stream`
 *   before returning, to report a candidate-list overflow as CKINV_EUNSUPPORTED. */
ckinv_status ckinv_omega_noalloc(int64_t n, int32_t d, uint64_t seed, uint32_t *sign_bits,
                                 int32_t *cols, ckinv_stream stream);

/* Sketch Y = K0 Omega (Sec. 3.1-3.2; Sec. 3.3's K_hat), computed matrix-free from the
 * points: kernel tiles are evaluated on the fly and contracted with Omega.
 *   points: n x dim FP32 row-major (x_i at points[i*dim]); NULL for CKINV_DENSE.  The
 *           tensor-core forms need them 16-byte aligned (CKINV_EINVAL otherwise).  A NaN or
 *           infinity among them is reported by the next ckinv_check as CKINV_EINVAL.
 *   K, ldk: n x n FP32 column-major kernel matrix for CKINV_DENSE (ldk >= n), else NULL.
 *   Y, ldy: n x d FP32 column-major output (ldy >= n).
 * No nugget enters the sketch.  plan->prec selects the contraction precision. */
ckinv_status ckinv_sketch(ckinv_ctx *ctx, const ckinv_plan_desc *plan,
                          const ckinv_kernel *kern, const float *points,
                          const float *K, int64_t ldk, float *Y, int64_t ldy,
                          ckinv_stream stream);

/* The kernel matrix K0 = variance * rho(x_i, x_k) materialised in device memory (n x n
 * FP32, column-major, ldk >= n; each entry evaluated in FP64 from the FP32 points and
 * rounded once): the input of the plain method with K held explicitly (Sec. 3.1 sketches a
 * given K), which ckinv_sketch then contracts as CKINV_DENSE.  4 n^2 bytes. */
ckinv_status ckinv_kernel_matrix(ckinv_ctx *ctx, const ckinv_plan_desc *plan,
                                 const ckinv_kernel *kern, const float *points, float *K,
                                 int64_t ldk, ckinv_stream stream);

/* Derivative sketch dK0/dlog(l) Omega (same layout as ckinv_sketch); used by the
 * gradient.  Not defined for CKINV_DENSE. */
ckinv_status ckinv_sketch_dlogl(ckinv_ctx *ctx, const ckinv_plan_desc *plan,
                                const ckinv_kernel *kern, const float *points,
                                float *Yd, int64_t ldy, ckinv_stream stream);

/* Blocked TSQR of Y (Sec. 3.3, Eqs. 1-4) and the low-rank core B = Omega^T Q_hat,
 * C' = R^T + tau B with their LU factorisations (FP64).  Y is read, not modified.
 * *out receives a library-owned factor (free with
 * ckinv_factor_free) holding Q_hat (n x d FP32) and six d x d FP64 matrices; it records
 * plan->refine_steps for ckinv_solve.  The factor is usable once `stream` reaches this
 * point.  A zero pivot in LU(B) or LU(C') is reported by the next ckinv_check. */
ckinv_status ckinv_tsqr(ckinv_ctx *ctx, const ckinv_plan_desc *plan,
                        const ckinv_kernel *kern, float *Y, int64_t ldy,
                        ckinv_factor **out, ckinv_stream stream);

/* Free a factor without host synchronisation: its memory is released in the order of the
 * stream it was created on, so work on other streams that reads it must be complete (or
 * ordered before that stream's current point).  NULL is allowed. */
ckinv_status ckinv_factor_free(ckinv_factor *f);

/* Copy the factor's R (d x d FP64, column-major, ld = d, diag(R) >= 0) to device R. */
ckinv_status ckinv_factor_r(const ckinv_factor *f, double *R, ckinv_stream stream);

/* Copy the explicit Q_hat (n x d FP32) to device Q (column-major, ldq >= n). */
ckinv_status ckinv_factor_q(const ckinv_factor *f, float *Q, int64_t ldq,
                            ckinv_stream stream);

/* Copy B = Omega^T Q_hat and C' = R^T + tau B (d x d FP64, ld = d) to device buffers
 * (either may be NULL) and write log det K_tilde = (n-d) ln tau + ln|det C'| -
 * ln|det B| to host *logdet (synchronises `stream`; may be NULL). */
ckinv_status ckinv_factor_core(const ckinv_factor *f, double *B, double *Cp,
                               double *logdet, ckinv_stream stream);

/* ---------------------------------------------------------------- row shards (several GPUs)
 * The paper's tree of QRs runs across "units" (Sec. 3.3: the blocks of Eq. 1 are factored
 * in parallel, then pairs of R factors are combined, Eqs. 2-3).  Across GPUs the rows of Y
 * are split into G contiguous shards, one per GPU; the points and Omega's seed are on every
 * GPU.  One solve takes these calls, with the collectives between them made by the caller
 * (for example over NCCL; no call here communicates):
 *   1. ckinv_sketch_rows      this shard's rows of Y (the contraction runs over all n points)
 *   2. ckinv_tsqr_shard       local TSQR: a shard factor and its d x d R  -> all-gather the R's
 *   3. ckinv_shard_combine    the top of the tree over the G R's (redundantly on every GPU),
 *                             the shard's rows of Q_hat, and its part of B  -> all-reduce B
 *   4. ckinv_shard_core       C' = R^T + tau B and the LUs (redundantly)
 *   5. ckinv_shard_solve_begin  Q_hat_shard^T A_shard                  -> all-reduce Z
 *   6. ckinv_shard_solve_end    the shard's rows of X = K_tilde^-1 A
 * The shard factor's solve takes no refinement step.  R, B and X equal those of one GPU
 * holding all rows up to rounding (the tree's pairing differs unless every shard holds the
 * same power-of-two number of leaves; R and Q_hat are unique for a full-rank Y). */

/* Rows row0 .. row0 + m - 1 of Y = K0 Omega (as ckinv_sketch, which is row0 = 0, m = n):
 * points (all n, as in ckinv_sketch), or the columns row0 .. row0 + m - 1 of a materialised
 * K (= its rows, K being symmetric).  Y: m x d FP32 column-major, ldy >= m. */
ckinv_status ckinv_sketch_rows(ckinv_ctx *ctx, const ckinv_plan_desc *plan,
                               const ckinv_kernel *kern, const float *points, const float *K,
                               int64_t ldk, int64_t row0, int64_t m, float *Y, int64_t ldy,
                               ckinv_stream stream);

/* Local TSQR of a shard's m rows of Y (rows row0 .. row0 + m - 1 of the problem that
 * plan->n describes; d <= m).  *out receives a shard factor (free with ckinv_factor_free);
 * R_local (device, d x d FP64, ld = d) receives the shard's R (diag >= 0). */
ckinv_status ckinv_tsqr_shard(ckinv_ctx *ctx, const ckinv_plan_desc *plan,
                              const ckinv_kernel *kern, float *Y, int64_t ldy, int64_t row0,
                              int64_t m, ckinv_factor **out, double *R_local, ckinv_stream stream);

/* Top of the tree over the G shards' R factors (R_all: device, G blocks of d x d FP64, block
 * k = shard k's R), combined pairwise in FP64 as Eqs. 2-3; the shard factor's R becomes the
 * root R and its Q_hat the shard's rows of the whole Q_hat.  B_partial (device d x d FP64)
 * receives Omega[rows of this shard]^T Q_hat_shard, whose sum over the shards is B. */
ckinv_status ckinv_shard_combine(ckinv_ctx *ctx, ckinv_factor *f, const double *R_all, int32_t G,
                                 int32_t g, double *B_partial, ckinv_stream stream);

/* B (device d x d FP64, the sum of the shards' B_partial): C' = R^T + tau B and the FP64 LUs
 * of B and C' in the shard factor. */
ckinv_status ckinv_shard_core(ckinv_ctx *ctx, ckinv_factor *f, const double *B, ckinv_stream stream);

/* Z_partial (device d x m FP64, ld = d) = Q_hat_shard^T A_shard; A_shard: the shard's m_rows x m
 * rows of A (FP32, lda >= the shard's rows).  The sum over the shards is Q_hat^T A. */
ckinv_status ckinv_shard_solve_begin(ckinv_ctx *ctx, const ckinv_factor *f, const float *A, int64_t lda,
                                     int32_t m, double *Z_partial, ckinv_stream stream);

/* The shard's rows of X = tau^-1 (A - Q_hat C'^-1 R^T Z), Z = Q_hat^T A (device d x m FP64,
 * the sum of the shards' Z_partial).  X may equal A. */
ckinv_status ckinv_shard_solve_end(ckinv_ctx *ctx, const ckinv_factor *f, const double *Z, const float *A,
                                   int64_t lda, int32_t m, float *X, int64_t ldx, ckinv_stream stream);

/* Second pass over K0 (the projection Q Q^T K of the proof of Theorem 3, made symmetric):
 * S = Q_hat^T K0 Q_hat (d x d FP64), computed matrix-free from the points on the tensor
 * cores (Q_hat split into three BF16 terms, kernel entries into three, the products of order
 * at most two, partial sums over 4096-point ranges folded in FP64).  Afterwards the factor's
 * core is the two-pass one: ckinv_solve applies K_tilde = tau I + Q_hat S Q_hat^T, solved
 * through the FP64 LU of S + tau I (no inverse of Omega^T Y, and positive semi-definite).
 *   plan, kern, points: as given to ckinv_sketch for this factor (plan->n and d must match).
 *   S: device d x d (ld = d) copy of S, or NULL.
 *   colspace_err: host; if not NULL receives ||K0 - Q Q^T K0||_F / ||K0||_F, the paper's
 *     accuracy measure (Sec. 3.1, Theorem 3), evaluated as sqrt(1 - ||K0 Q||^2 / ||K0||^2)
 *     with ||K0||_F^2 from FP64 kernel entries (n^2 of them; errors below ~1e-3 are not
 *     resolved by that difference); the call then synchronises `stream`.
 * Must run on the stream the factor was created on. */
ckinv_status ckinv_factor_project(ckinv_ctx *ctx, ckinv_factor *f, const ckinv_plan_desc *plan,
                                  const ckinv_kernel *kern, const float *points, double *S,
                                  double *colspace_err, ckinv_stream stream);

/* Gaussian-process predictive mean at n_new points (the prediction task of Sec. 5's data
 * example): mean[i] = sum_k K0(x*_i, x_k) alpha_k, alpha = K_tilde^-1 y as ckinv_solve gives
 * it.  Kernel entries and sums in FP64 (alpha's terms reach |y| / tau and cancel).
 *   points: n x dim FP32 (the plan's), alpha: n FP32, new_points: n_new x dim FP32 row-major,
 *   mean: n_new FP64, all device. */
ckinv_status ckinv_predict_mean(ckinv_ctx *ctx, const ckinv_plan_desc *plan, const ckinv_kernel *kern,
                                const float *points, const float *alpha, const float *new_points,
                                int64_t n_new, double *mean, ckinv_stream stream);

/* X = K_tilde^-1 A (Sec. 1's R^-1 Q^T A in Woodbury form), then plan->refine_steps
 * steps of FP64 iterative refinement X += K_tilde^-1 (A - K_tilde X).
 *   A: n x m FP32 (lda >= n);  X: n x m FP32 (ldx >= n); X may equal A.  1 <= m <= 256.
 * A NaN or infinity in A is reported by the next ckinv_check as CKINV_EINVAL. */
ckinv_status ckinv_solve(ckinv_ctx *ctx, const ckinv_factor *f, const float *A,
                         int64_t lda, int32_t m, float *X, int64_t ldx,
                         ckinv_stream stream);

/* One call for the whole path: sketch, TSQR, core and solve.  points, A and X may be
 * host or device pointers (host buffers are staged through device memory inside the
 * call, which then synchronises `stream`). */
ckinv_status ckinv_kinv_a(ckinv_ctx *ctx, const ckinv_plan_desc *plan,
                          const ckinv_kernel *kern, const float *points,
                          const float *A, int64_t lda, int32_t m, float *X,
                          int64_t ldx, ckinv_stream stream);

/* Gaussian negative log-likelihood of targets y (n FP32, device) under K_tilde,
 *   NLL = 1/2 y^T K_tilde^-1 y + 1/2 log det K_tilde + n/2 ln(2 pi),
 * and its gradient with respect to (log l, log variance, log nugget), written to
 * host *nll and host grad[3] after synchronising `stream`. */
ckinv_status ckinv_nll_grad(ckinv_ctx *ctx, const ckinv_plan_desc *plan,
                            const ckinv_kernel *kern, const float *points,
                            const float *y, double *nll, double *grad,
                            ckinv_stream stream);

/* Leaf-height autotuner of the TSQR (the block_rows of a plan).  Times the TSQR of an
 * n x d pseudo-random matrix at the candidate heights 256 .. 4096 (at least d, at most
 * n / 2) with the plan's tree_fp64_levels and leaf_fp64, and records the fastest for the
 * shape class (device, d, ceil(log2 n), tree_fp64_levels, leaf_fp64).  Every later call
 * on any context whose plan has block_rows = 0 and the same shape class uses it.  Writes
 * the chosen height to *block_rows; synchronises `stream`.  No counterpart in the paper,
 * which fixes the height by a formula in n and r (Sec. 3.3).  Without tuning the
 * library uses 2048 rows, or n / 2 for small n. */
ckinv_status ckinv_autotune(ckinv_ctx *ctx, const ckinv_plan_desc *plan, int32_t *block_rows,
                            ckinv_stream stream);

/* Batched form over nprob independent problems (uneven n, d, kernels): plans[p],
 * kerns[p], points[p], y[p] as above (device pointers in HOST arrays); nll[p] and
 * grad[3p..3p+2] are host outputs, written after `stream` is synchronised.  Each problem
 * runs the same pipeline as ckinv_nll_grad; the pipelines of all problems are captured
 * into one CUDA graph (on 8 forked streams, so that small problems overlap on the SMs)
 * and the graph is launched once.  A problem whose block_rows is 0 gets the leaf height
 * the autotuner (ckinv_autotune) picks for its shape class, tuned on first sight.
 * Device-side errors name the problem index in ckinv_last_error.  The paper motivates the
 * method by likelihoods of many points (Abstract, Sec. 1); batching many independent
 * problems has no counterpart there. */

ckinv_status ckinv_nll_grad_batched(ckinv_ctx *ctx, int32_t nprob,
                                    const ckinv_plan_desc *plans,
                                    const ckinv_kernel *kerns,
                                    const float *const *points, const float *const *y,
                                    double *nll, double *grad, ckinv_stream stream);

#ifdef __cplusplus
}
#endif
#endif /* CKINV_H */
