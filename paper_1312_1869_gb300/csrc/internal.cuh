// Internal declarations of the ckinv CUDA library (sm_103a).  Not part of the C ABI.
#pragma once
#include <cuda_runtime.h>
#include <cuda_bf16.h>
#include <stdint.h>
#include <algorithm>
#include <string>
#include <vector>

#include "../../include/ckinv.h"

namespace ckinv {

// ----------------------------------------------------------------------------- errors
struct Error {
  ckinv_status st;
  std::string msg;
};

#define CK_CUDA(call)                                                              \
  do {                                                                             \
    cudaError_t e_ = (call);                                                       \
    if (e_ != cudaSuccess) {                                                       \
      return ::ckinv::Error{e_ == cudaErrorMemoryAllocation ? CKINV_ENOMEM         \
                                                            : CKINV_ECUDA,          \
                            std::string(#call) + ": " + cudaGetErrorString(e_)};   \
    }                                                                              \
  } while (0)

#define CK_TRY(expr)                                                               \
  do {                                                                             \
    ::ckinv::Error er_ = (expr);                                                   \
    if (er_.st != CKINV_OK) return er_;                                            \
  } while (0)

inline Error ok() { return Error{CKINV_OK, std::string()}; }

// Message returned by ckinv_last_error(NULL) for calls that have no context.
void set_static_error(const std::string &msg);

// Host-side count of kernel launches issued by the library (diagnostics).
unsigned long long &launch_counter();
inline void note_launch() { __atomic_add_fetch(&launch_counter(), 1ull, __ATOMIC_RELAXED); }
inline Error fail(ckinv_status s, const std::string &m) { return Error{s, m}; }

// Device error word bits (ctx->d_err); the host maps them to a status.
enum : int {
  DERR_TIMEOUT = 1,      // a bounded mbarrier / flag wait ran out
  DERR_SINGULAR = 2,     // zero pivot in an LU
  DERR_CAPACITY = 4,     // an on-device list overflowed its buffer
  DERR_NONFINITE = 8,    // a non-finite value in the points, A or y
};

// Limit of a device-side wait for another role's progress (ns), unless the context sets
// another one (ckinv_set_wait_limit).  Waits for the library's own copies and MMAs to drain
// after a timeout always keep the default, so that nothing is left in flight.
constexpr uint64_t kDefaultWaitNs = 1000000000ull;

// Stream-ordered device allocation from the library's own memory pool (one per device,
// created on first use, freed memory kept for reuse), or from the device's default pool
// while `st` is being captured into a CUDA graph.  Free with cudaFreeAsync.
cudaError_t dev_alloc(void **p, size_t bytes, cudaStream_t st);
template <typename T>
inline cudaError_t dev_alloc(T **p, size_t bytes, cudaStream_t st) {
  return dev_alloc(reinterpret_cast<void **>(p), bytes, st);
}

// ----------------------------------------------------------------------------- context
// The last Omega drawn on a context; buffers only grow, so that a context whose capacity
// was reserved up front never allocates inside a captured graph.
struct OmegaCache {
  int64_t n = -1;
  int32_t d = -1;
  uint64_t seed = 0;
  uint32_t *bits = nullptr;     // ceil(n/32) words
  size_t bits_cap = 0;          // words
  int32_t *cols = nullptr;      // d
  size_t cols_cap = 0;
  __nv_bfloat16 *omegaT = nullptr;  // d x kpad, row j = Omega column j (unscaled +-1)
  size_t omegaT_cap = 0;        // bytes
  int64_t kpad = 0;
  bool omegaT_valid = false;
};

// Pinned host memory for descriptor uploads made while a stream is being captured: each
// upload gets its own bytes, alive until the graph has run.
struct UploadArena {
  unsigned char *host = nullptr;
  size_t cap = 0, used = 0;
};

}  // namespace ckinv

struct ckinv_batch_graph;

struct ckinv_ctx {
  // pinned host staging ring for small descriptor uploads (no host synchronisation)
  struct Stage {
    void *host = nullptr;
    size_t cap = 0;
    cudaEvent_t done = nullptr;
  } stage[8];
  int stage_next = 0;
  int device = 0;
  int sm_count = 0;
  std::string err;
  ckinv::OmegaCache om;
  int *d_err = nullptr;               // device error word
  // scratch of the Omega draw
  uint32_t *hist = nullptr;           // 65536 bins
  unsigned long long *cand = nullptr; // candidate (key) list
  uint32_t *cand_idx = nullptr;
  uint32_t *small = nullptr;          // small counters
  size_t cand_cap = 0;
  // set while the context's work is being captured into a CUDA graph
  ckinv::UploadArena *capture_arena = nullptr;
  // the last batched likelihood's instantiated CUDA graph and what it refers to
  struct ckinv_batch_graph *batch = nullptr;
  // FP32 GEMMs on the tensor cores (split BF16) rather than the CUDA cores; set by
  // tsqr_factor for the duration of one factorization
  bool gemm_tc = false;
  // limit of the device-side waits of kernels launched from this context (ns)
  uint64_t wait_ns = ckinv::kDefaultWaitNs;
};

struct ckinv_factor {
  ckinv_ctx *ctx = nullptr;
  int device = 0;
  cudaStream_t stream = nullptr;   // creation stream: memory is released in its order
  int64_t n = 0;
  int32_t d = 0;
  double tau = 0;
  float *Q = nullptr;        // n x d explicit Q_hat (ld = n)
  double *R = nullptr;       // d x d, diag >= 0
  double *B = nullptr;       // d x d  Omega^T Q_hat
  double *Cp = nullptr;      // d x d  R^T + tau B
  double *luB = nullptr;     // packed LU of B
  double *luC = nullptr;     // packed LU of C'
  int32_t *pivB = nullptr;
  int32_t *pivC = nullptr;
  double *logdet_parts = nullptr;  // [ln|det B|, ln|det C'|]
  uint32_t *bits = nullptr;  // Omega signs (copy)
  int32_t *cols = nullptr;   // Omega columns (copy)
  double omega_scale = 0;
  int refine_steps = 0;
  int prec = 0;              // plan precision: FP32 keeps every contraction FP32-accurate
  // two-pass core (ckinv_factor_project): S = Q_hat^T K0 Q_hat and the LU of S + tau I
  bool two_pass = false;
  double *S2 = nullptr;      // d x d S, then d x d packed LU of S + tau I
  int32_t *pivS = nullptr;
  double *logdet2 = nullptr; // ln|det(S + tau I)|
  // row shard (ckinv_tsqr_shard): this factor holds rows row0 .. row0 + n - 1 of a problem of
  // n_total points; Omega's signs and columns are those of the whole problem
  int64_t row0 = 0;
  int64_t n_total = 0;
  // Omega of a kind other than the bit-generated Walsh-Hadamard one: dense n x d FP32 copy
  int omega_kind = 0;
  float *omega_dense = nullptr;
};

namespace ckinv {

// ----------------------------------------------------------------------------- helpers
inline int64_t padded_order(int64_t n) {
  int64_t N = 1;
  while (N < n) N <<= 1;
  return N;
}
inline int64_t ceil_div(int64_t a, int64_t b) { return (a + b - 1) / b; }

// Kernel parameters as the device code consumes them.
struct KernelParams {
  int kind;          // CKINV_SE / CKINV_MATERN52
  float inv_l;       // 1/l
  float c_se;        // log2(e) / (2 l^2): SE value = exp2(-r^2 c_se)
  float coord_scale; // sqrt(c_se) for SE (points pre-scaled), 1 for Matern
  double scale;      // variance * omega scale c, applied in the epilogue
  double ell;        // lengthscale (FP64 evaluation of the FP32 form)
  double var;        // variance
};

// Upload `bytes` of host data to device memory `dst` on `st` through the pinned staging
// ring: the host does not wait for the stream unless the ring slot is still in flight.
Error stage_upload(ckinv_ctx *ctx, const void *src, size_t bytes, void *dst, cudaStream_t st);

// ----------------------------------------------------------------------------- Omega
Error omega_draw(ckinv_ctx *ctx, int64_t n, int32_t d, uint64_t seed, cudaStream_t st);
Error omega_materialise_bf16(ckinv_ctx *ctx, cudaStream_t st);   // ctx->om.omegaT
// Omega as a dense n x d FP32 matrix (ld n) of kind 0 Walsh-Hadamard, 1 scaled Gaussian,
// 2 discrete Hartley, 3 discrete cosine (T of Definition 1, or Sec. 5.1's Gaussian projection).
Error omega_dense(ckinv_ctx *ctx, int64_t n, int32_t d, uint64_t seed, int kind, float *Om, cudaStream_t st);
// Y = var * K0 Omega for a dense Omega (n x d FP32): the fused tensor-core sketch with Omega in
// three BF16 terms and kernel entries in three, the six term products of order <= 2, partial
// sums over 4096-point ranges folded in FP64.
Error sketch_dense_omega(ckinv_ctx *ctx, int64_t n, int dim, int d, const KernelParams &kp, const float *points,
                         const float *Om, float *Y, int64_t ldy, cudaStream_t st);
// Grows the context's Omega buffers and draw scratch to hold an (n, d) draw (no draw).
Error omega_reserve(ckinv_ctx *ctx, int64_t n, int32_t d, cudaStream_t st);

// ----------------------------------------------------------------------------- sketch
// Rows row0 .. row0 + m - 1 of Y = K0 Omega (m < 0: all n rows); with a materialised K its
// rows (columns, K being symmetric) row0 .. row0 + m - 1 are read.
Error sketch_simt(ckinv_ctx *ctx, int64_t n, int dim, int d, const KernelParams &kp,
                  const float *points, const float *K, int64_t ldk, bool deriv,
                  float *Y, int64_t ldy, cudaStream_t st, int64_t row0 = 0, int64_t m = -1);
// K (n x n FP32, column-major, ld ldk) = var * rho(x_i, x_k), each entry evaluated in FP64
// from the FP32 points and rounded once.
Error kernel_matrix(ckinv_ctx *ctx, int64_t n, int dim, const KernelParams &kp, const float *points, float *K,
                    int64_t ldk, cudaStream_t st);
// Rows row0 .. row0 + m - 1 of Y = K0 Omega through the fast Walsh-Hadamard transform, FP32 on
// the CUDA cores (needs N = 2^ceil(log2 n) >= 1024 and d <= 512).
bool sketch_wht_supported(int64_t n, int d);
Error sketch_wht(ckinv_ctx *ctx, int64_t n, int dim, int d, const KernelParams &kp, const float *points, bool deriv,
                 float *Y, int64_t ldy, cudaStream_t st, int64_t row0 = 0, int64_t m = -1);
// The same transform over a materialised K0 (n x n, column-major, ld ldk; symmetric, so row i
// is read as column i).
Error sketch_wht_dense(ckinv_ctx *ctx, int64_t n, int d, const KernelParams &kp, const float *K, int64_t ldk, float *Y,
                       int64_t ldy, cudaStream_t st, int64_t row0 = 0, int64_t m = -1,
                       const uint32_t *bits = nullptr, const int32_t *cols = nullptr);
// Whether a form applies the Walsh-Hadamard Omega to an n x d matrix (Omega^T X) by the fast
// transform: the BF16 and fast-transform forms, where N >= 1024.
inline bool omega_by_transform(int prec, int64_t n, int d) {
  return (prec == CKINV_BF16 || prec == CKINV_FP32_WHT) && sketch_wht_supported(n, d);
}
// B (d x d, FP64, ld d) = scale Omega^T X for X n x d (FP32, ld ldx), with Omega's signs and
// columns given: the fast transform over X's d columns in FP32, transposed and widened.
Error omega_t_times_wht(ckinv_ctx *ctx, int64_t n, int d, const float *X, int64_t ldx, const uint32_t *bits,
                        const int32_t *cols, double scale, double *B, cudaStream_t st);
Error sketch_tc(ckinv_ctx *ctx, int64_t n, int dim, int d, int nsplit,
                const KernelParams &kp, const float *points, bool deriv, float *Y,
                int64_t ldy, cudaStream_t st, int64_t row0 = 0, int64_t m = -1);
// Tensor-core contraction of a dense FP32 matrix with Omega (the context's current draw):
// rows i < m of A (row i at A + i*lda, contiguous over the n-long contraction), split into
// nsplit BF16 terms.  Either Y (column-major, store) = scale * A Omega, or
// G[i*si + j*sj] = scale * (A Omega)[i][j] reduced in FP64 (split contraction).
Error dense_tc(ckinv_ctx *ctx, int64_t m, int64_t n, int d, int nsplit, const float *A, int64_t lda,
               double scale, float *Y, int64_t ldy, double *G, int64_t si, int64_t sj, cudaStream_t st);

// ----------------------------------------------------------------------------- TSQR
struct TsqrOut {
  float *Q;     // n x d (ld n), explicit, column signs folded in
  double *R;    // d x d, diag >= 0
};
Error tsqr_factor(ckinv_ctx *ctx, int64_t n, int d, int b, int fp64_levels, bool leaf_fp64, bool tc_gemm,
                  const float *Y, int64_t ldy, float *Qout, double *Rout, cudaStream_t st);
// One problem of a joint factorization: Y (n x d, ld ldy) -> Q_hat (ld ldq) and R (d x d).
struct TsqrProblem {
  int64_t n;
  const float *Y;
  int64_t ldy;
  float *Q;
  int64_t ldq;
  double *R;
};
// Several problems of the same d factored together (one leaf stage and one stage per tree
// level for all of them); each problem's results are those of its own factorization.
Error tsqr_factor_multi(ckinv_ctx *ctx, const std::vector<TsqrProblem> &probs, int d, int b, int fp64_levels,
                        bool leaf_fp64, bool tc_gemm, cudaStream_t st);
int auto_block_rows(int64_t n, int d, int sm_count);
// Tallest TSQR leaf (a multiple of 16) whose panels fit in shared memory at this d.
int max_leaf_rows(int d, bool leaf_fp64);
// Tree combine of G given R factors (FP64, strided d x d): root R (diag >= 0) and each leaf's
// d x d block of the combined Q factor.
Error tsqr_combine_r(ckinv_ctx *ctx, int G, int d, const double *Rin, double *Rout, double *Xout, cudaStream_t st);

// ----------------------------------------------------------------------------- GEMM
// C_b = alpha op(A_b) B_b + beta C_b for b < batch (column-major, strided batches).
// FP32 batched GEMM on the tensor cores (three BF16 terms per operand, six products).
Error gemm_tc_f32(const ckinv_ctx *ctx, bool transA, int M, int N, int K, float alpha, const float *A, int64_t lda,
                  int64_t sA, const float *B, int64_t ldb, int64_t sB, float beta, float *C, int64_t ldc, int64_t sC,
                  int batch, cudaStream_t st);
template <typename T>
Error gemm_batched(const ckinv_ctx *ctx, bool transA, int M, int N, int K, T alpha, const T *A, int64_t lda,
                   int64_t sA, const T *B, int64_t ldb, int64_t sB, T beta, T *C, int64_t ldc, int64_t sC,
                   int batch, cudaStream_t st);
// Two-level batch on the CUDA cores: b = b1 + nb1 * b2, operand offset b1 * s + b2 * s2.
template <typename T>
Error gemm_batched2(const ckinv_ctx *ctx, bool transA, int M, int N, int K, T alpha, const T *A, int64_t lda,
                    int64_t sA, int64_t sA2, const T *B, int64_t ldb, int64_t sB, int64_t sB2, T beta, T *C,
                    int64_t ldc, int64_t sC, int64_t sC2, int nb1, int nb2, cudaStream_t st);

// ----------------------------------------------------------------------------- low rank
// G (d1 x d2, FP64, ld d1) = L^T M over n rows.  L = explicit FP32 (ldl) or, when
// L == nullptr, Omega generated from bits/cols/scale.
Error tsprod(ckinv_ctx *ctx, int64_t n, int d1, int d2, const float *L, int64_t ldl,
             const uint32_t *bits, const int32_t *cols, double oscale, const float *M,
             int64_t ldm, double *G, cudaStream_t st, int64_t orow0 = 0);
Error lu_factor_f64(ckinv_ctx *ctx, int n, double *A, int32_t *piv, double *logabsdet,
                    cudaStream_t st);
Error lowrank_solve(ckinv_ctx *ctx, const ckinv_factor *f, const float *A, int64_t lda,
                    int m, float *X, int64_t ldx, int refine_steps, cudaStream_t st);
Error lowrank_core(ckinv_ctx *ctx, ckinv_factor *f, cudaStream_t st);
// C' = R^T + tau B and the LUs of B and C' from the factor's R and B (B already in f->B).
Error core_from_b(ckinv_ctx *ctx, ckinv_factor *f, cudaStream_t st);
// X = tau^-1 (A - Q_hat C'^-1 R^T Z) for a given Z = Q_hat^T A (row shards: Z all-reduced).
Error solve_from_z(ckinv_ctx *ctx, const ckinv_factor *f, const double *Z, const float *A, int64_t lda, int m,
                   float *X, int64_t ldx, cudaStream_t st);
// Second pass over K0: S = Q_hat^T K0 Q_hat (tensor cores, Q_hat in three BF16 terms, partial
// sums folded in FP64), the factor switched to the two-pass core, and (if colspace is not
// null) the column-space error ||K0 - Q Q^T K0||_F / ||K0||_F written to host *colspace.
Error two_pass_core(ckinv_ctx *ctx, ckinv_factor *f, int dim, const KernelParams &kp, const float *points,
                    double *colspace, cudaStream_t st);
// mean[i] = K0(x*_i, X) alpha (FP64 entries and sums; mean device FP64).
Error predict_mean(ckinv_ctx *ctx, int64_t n, int dim, const KernelParams &kp, const float *points, const float *alpha,
                   const float *xnew, int64_t n_new, double *mean, cudaStream_t st);
// X (d x m FP64) <- op(A)^-1 X for a packed LU with LAPACK interchanges.
Error lu_solve_dev(int d, int m, const double *LU, const int32_t *piv, double *X, int trans, cudaStream_t st);
// C (d x m) = op(A) Bm, FP64, ld = d.
Error gemm_small_dev(int d, int m, const double *A, const double *Bm, double *C, int transA, cudaStream_t st);

}  // namespace ckinv

// ----------------------------------------------------------------------------- device
#ifdef __CUDACC__
namespace ckinv {
namespace dev {

__device__ __forceinline__ uint4 philox4x32_10(uint32_t c0, uint32_t c1, uint32_t c2,
                                               uint32_t c3, uint32_t k0, uint32_t k1) {
  // Philox4x32-10 (Salmon et al., SC'11): 10 rounds of the 4x32 S-box, key bumped by
  // the Weyl constants between rounds.
  const uint32_t M0 = 0xD2511F53u, M1 = 0xCD9E8D57u;
  const uint32_t W0 = 0x9E3779B9u, W1 = 0xBB67AE85u;
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    if (r) {
      k0 += W0;
      k1 += W1;
    }
    uint32_t hi0 = __umulhi(M0, c0), lo0 = M0 * c0;
    uint32_t hi1 = __umulhi(M1, c2), lo1 = M1 * c2;
    uint32_t n0 = hi1 ^ c1 ^ k0, n2 = hi0 ^ c3 ^ k1;
    c0 = n0;
    c1 = lo1;
    c2 = n2;
    c3 = lo0;
  }
  return make_uint4(c0, c1, c2, c3);
}

__device__ __forceinline__ float ex2_approx(float x) {
  float y;
  asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}

// Unit-variance kernel value (or its d/dlog(l)) from the squared distance r2 computed
// in pre-scaled coordinates (SE: coordinates scaled by sqrt(c_se), so r2s = r^2 c_se;
// Matern: unscaled, r2s = r^2).
__device__ __forceinline__ float kernel_value(int kind, float r2s, float inv_l, bool deriv) {
  if (kind == CKINV_SE) {
    float v = ex2_approx(-r2s);
    // d/dlog l of exp(-r^2/(2l^2)) = exp(.) * r^2/l^2 = exp(.) * r2s * 2 ln2
    return deriv ? v * (r2s * 1.3862943611198906f) : v;
  } else {
    float r = sqrtf(r2s);
    float u = 2.2360679774997896f * r * inv_l;
    float e = ex2_approx(-u * 1.4426950408889634f);
    return deriv ? (u * u * (1.0f / 3.0f)) * (1.0f + u) * e
                 : (1.0f + u + u * u * (1.0f / 3.0f)) * e;
  }
}

}  // namespace dev
}  // namespace ckinv
#endif
