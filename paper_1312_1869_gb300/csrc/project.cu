// The paper's accuracy measure and prediction on the GPU, and the two-pass core:
//   * S = Q_hat^T K0 Q_hat from a second pass over K0 (the projection Q Q^T K of the proof of
//     Theorem 3, made symmetric), with the column-space error ||K0 - Q Q^T K0||_F / ||K0||_F
//     (Sec. 3.1, Theorem 3; the Frobenius error of Sec. 5's Table 3) and the solve with
//     tau I + Q_hat S Q_hat^T;
//   * the Gaussian-process predictive mean mu* = K0(X*, X) alpha at new points (the prediction
//     task of Sec. 5's data example).
//
// W = K0 Q_hat is the fused sketch kernel with Q_hat in place of Omega: Q_hat's columns are
// split into three BF16 terms (Bt_t, row j = term t of column j), and three launches take the
// products of order at most two (3-term kernel entries x Bt_0, 2-term x Bt_1, 1-term x Bt_2),
// each with its contraction split into ranges of at most kMaxBlocksPerSplit point blocks
// whose FP32 partial sums are kept apart and added in FP64 afterwards: the tensor cores'
// FP32 accumulation loses up to 2^-23 per K = 16 step, so a long accumulation (thousands of
// steps) is cut into short ones.
#include <cmath>

#include "internal.cuh"

namespace ckinv {
Error sketch_tc_rhs(ckinv_ctx *ctx, int64_t n, int dim, int d, int nsplit, const KernelParams &kp, const float *points,
                    const __nv_bfloat16 *Bt, int64_t kpad, int splits, float *part, int64_t ldp, bool accumulate,
                    cudaStream_t st);

namespace {

constexpr int kMaxBlocksPerSplit = 64;   // 4096 points per partial accumulation

// Bt[t][j * kpad + k] = BF16 term t of Q[k + j * ldq] (k < n; zero for n <= k < kpad): each
// term the BF16 rounding of what the terms before it left of the FP32 value.
__global__ void k_split_terms(int64_t n, int d, const float *__restrict__ Q, int64_t ldq, int64_t kpad,
                             __nv_bfloat16 *__restrict__ Bt) {
  const int j = blockIdx.y;
  for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < kpad; k += (int64_t)gridDim.x * blockDim.x) {
    float r = k < n ? Q[k + (int64_t)j * ldq] : 0.0f;
#pragma unroll
    for (int t = 0; t < 3; ++t) {
      const __nv_bfloat16 b = __float2bfloat16_rn(r);
      Bt[(int64_t)t * d * kpad + (int64_t)j * kpad + k] = b;
      r -= __bfloat162float(b);
    }
  }
}

// W[i + j * ldw] = scale * sum_s part[s][i + j * ldp], summed in FP64 in split order.
__global__ void k_fold_parts_f32(int64_t n, int d, int splits, const float *__restrict__ part, int64_t ldp, double scale,
                                 float *__restrict__ W, int64_t ldw) {
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < n * d; e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = e % n, j = e / n;
    double acc = 0.0;
    for (int s = 0; s < splits; ++s) acc += (double)part[(int64_t)s * ldp * d + i + j * ldp];
    W[i + j * ldw] = (float)(scale * acc);
  }
}

// Unit-variance kernel value in FP64 from the squared distance.
__device__ __forceinline__ double rho_f64(int kind, double r2, double ell) {
  if (kind == CKINV_SE) return exp(-0.5 * r2 / (ell * ell));
  const double u = 2.2360679774997896964 * sqrt(r2) / ell;
  return (1.0 + u + u * u / 3.0) * exp(-u);
}

// Per-block partial sums of rho(x_i, x_k)^2 over all pairs: one thread per row i, the points
// x_k read by every lane of a warp at once (broadcast loads); entries in FP32 (expf, about one
// unit of FP32 rounding), their squares summed in FP32 over 256 consecutive k and those
// chunk sums added in FP64.  ||K0||_F^2 then carries ~1e-6 relative error, which resolves
// column-space errors down to ~1e-3.
constexpr int kSqThreads = 256;
__global__ void __launch_bounds__(kSqThreads) k_kernel_sqnorm(int64_t n, int dim, int kind, float ell,
                                                              const float *__restrict__ pts, double *partial) {
  __shared__ double red[kSqThreads];
  double acc = 0.0;
  const float inv_l = 1.0f / ell;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i - threadIdx.x < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    const bool live = i < n;
    float x[3] = {0.f, 0.f, 0.f};
    if (live)
      for (int t = 0; t < dim; ++t) x[t] = pts[i * dim + t];
    for (int64_t k0 = 0; k0 < n; k0 += 256) {
      const int64_t k1 = k0 + 256 < n ? k0 + 256 : n;
      float chunk = 0.0f;
      for (int64_t k = k0; k < k1; ++k) {
        float r2 = 0.0f;
        for (int t = 0; t < dim; ++t) {
          const float df = x[t] - __ldg(pts + k * dim + t);
          r2 = fmaf(df, df, r2);
        }
        float v;
        if (kind == CKINV_SE) {
          v = expf(-0.5f * r2 * inv_l * inv_l);
        } else {
          const float u = 2.2360679774997896f * sqrtf(r2) * inv_l;
          v = (1.0f + u + u * u * (1.0f / 3.0f)) * expf(-u);
        }
        chunk = fmaf(v, v, chunk);
      }
      if (live) acc += (double)chunk;
    }
  }
  red[threadIdx.x] = acc;
  __syncthreads();
  for (int o = kSqThreads / 2; o > 0; o >>= 1) {
    if ((int)threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x == 0) partial[blockIdx.x] = red[0];
}

// out[0] = sum of partial[0..count) in order; out[1] = sum of W's squares (FP64), one block.
__global__ void __launch_bounds__(1024) k_finish_norms(int count, const double *partial, int64_t nw, const float *W,
                                                       double *out) {
  __shared__ double red[1024];
  double s = 0.0;
  for (int64_t e = threadIdx.x; e < nw; e += blockDim.x) s = fma((double)W[e], (double)W[e], s);
  red[threadIdx.x] = s;
  __syncthreads();
  for (int o = 512; o > 0; o >>= 1) {
    if ((int)threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    double k2 = 0.0;
    for (int b = 0; b < count; ++b) k2 += partial[b];
    out[0] = k2;
    out[1] = red[0];
  }
}

// A = S + tau I (copy of S, FP64 d x d) for the two-pass LU.
__global__ void k_shift(int d, const double *S, double tau, double *A) {
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < d * d; e += gridDim.x * blockDim.x)
    A[e] = S[e] + ((e % d) == (e / d) ? tau : 0.0);
}

// mean[i] = sum_k var rho(x*_i, x_k) alpha_k, FP64 entries and FP64 sums (alpha = K_tilde^-1 y
// carries magnitudes up to ~|y| / tau whose terms cancel).  One thread per new point; the
// points and alpha stream through shared memory in tiles.
constexpr int kPredThreads = 128;
constexpr int kPredTile = 256;
__global__ void __launch_bounds__(kPredThreads) k_predict_mean(int64_t n, int64_t n_new, int dim, int kind, double ell,
                                                               double var, const float *__restrict__ pts,
                                                               const float *__restrict__ alpha,
                                                               const float *__restrict__ xnew, double *mean) {
  __shared__ double sp[kPredTile * 3];
  __shared__ double sa[kPredTile];
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  double x[3] = {0.0, 0.0, 0.0};
  if (i < n_new)
    for (int t = 0; t < dim; ++t) x[t] = (double)xnew[i * dim + t];
  double acc = 0.0;
  for (int64_t k0 = 0; k0 < n; k0 += kPredTile) {
    const int cnt = (int)((n - k0) < kPredTile ? (n - k0) : kPredTile);
    __syncthreads();
    for (int e = threadIdx.x; e < cnt * dim; e += blockDim.x) sp[e] = (double)pts[k0 * dim + e];
    for (int e = threadIdx.x; e < cnt; e += blockDim.x) sa[e] = (double)alpha[k0 + e];
    __syncthreads();
    for (int k = 0; k < cnt; ++k) {
      double r2 = 0.0;
      for (int t = 0; t < dim; ++t) {
        const double df = x[t] - sp[k * dim + t];
        r2 = fma(df, df, r2);
      }
      acc = fma(rho_f64(kind, r2, ell), sa[k], acc);
    }
  }
  if (i < n_new) mean[i] = var * acc;
}

}  // namespace

Error two_pass_core(ckinv_ctx *ctx, ckinv_factor *f, int dim, const KernelParams &kp, const float *points,
                    double *colspace, cudaStream_t st) {
  const int64_t n = f->n;
  const int d = f->d;
  const int64_t kpad = ceil_div(n, 64) * 64;
  const int num_kb = (int)(kpad / 64);
  const int splits = (int)ceil_div(num_kb, kMaxBlocksPerSplit);
  const int64_t ldp = ceil_div(n, 128) * 128;
  __nv_bfloat16 *Bt = nullptr;
  float *part = nullptr, *W = nullptr;
  double *norm_part = nullptr, *norms = nullptr;
  const int sq_blocks = (int)ceil_div(n, kSqThreads);
  struct Release {
    std::vector<void *> p;
    cudaStream_t st;
    ~Release() {
      for (void *q : p)
        if (q) cudaFreeAsync(q, st);
    }
  } release{{}, st};
  CK_CUDA(dev_alloc(&Bt, sizeof(__nv_bfloat16) * 3 * d * kpad, st));
  release.p.push_back(Bt);
  CK_CUDA(dev_alloc(&part, sizeof(float) * (size_t)splits * ldp * d, st));
  release.p.push_back(part);
  CK_CUDA(dev_alloc(&W, sizeof(float) * (size_t)n * d, st));
  release.p.push_back(W);
  CK_CUDA(dev_alloc(&norm_part, sizeof(double) * sq_blocks, st));
  release.p.push_back(norm_part);
  CK_CUDA(dev_alloc(&norms, sizeof(double) * 2, st));
  release.p.push_back(norms);
  // Q_hat's columns as three BF16 terms
  note_launch();
  k_split_terms<<<dim3((unsigned)std::min<int64_t>(ceil_div(kpad, 256), 1024), d), 256, 0, st>>>(n, d, f->Q, n, kpad,
                                                                                                 Bt);
  CK_CUDA(cudaGetLastError());
  // W = var * K0 Q_hat: (3-term entries) x Bt_0 + (2-term) x Bt_1 + (1-term) x Bt_2
  for (int t = 0; t < 3; ++t)
    CK_TRY(sketch_tc_rhs(ctx, n, dim, d, 3 - t, kp, points, Bt + (size_t)t * d * kpad, kpad, splits, part, ldp, t > 0,
                         st));
  note_launch();
  k_fold_parts_f32<<<(unsigned)std::min<int64_t>(ceil_div(n * d, 256), 4096), 256, 0, st>>>(n, d, splits, part, ldp,
                                                                                            kp.var, W, n);
  CK_CUDA(cudaGetLastError());
  // S = Q_hat^T W (FP64 d x d), then the two-pass core: LU of S + tau I
  if (!f->S2) {
    CK_CUDA(dev_alloc(&f->S2, sizeof(double) * 2 * d * d, f->stream));
    CK_CUDA(dev_alloc(&f->pivS, sizeof(int32_t) * d, f->stream));
    CK_CUDA(dev_alloc(&f->logdet2, sizeof(double), f->stream));
  }
  double *S = f->S2, *luS = f->S2 + (size_t)d * d;
  CK_TRY(tsprod(ctx, n, d, d, f->Q, n, nullptr, nullptr, 0.0, W, n, S, st));
  note_launch();
  k_shift<<<64, 256, 0, st>>>(d, S, f->tau, luS);
  CK_CUDA(cudaGetLastError());
  CK_TRY(lu_factor_f64(ctx, d, luS, f->pivS, f->logdet2, st));
  f->two_pass = true;
  if (colspace) {
    // ||K0 - Q Q^T K0||_F^2 = ||K0||_F^2 - ||K0 Q||_F^2 (Q orthonormal); ||K0||_F^2 in FP64
    note_launch();
    k_kernel_sqnorm<<<sq_blocks, kSqThreads, 0, st>>>(n, dim, kp.kind, (float)kp.ell, points, norm_part);
    note_launch();
    k_finish_norms<<<1, 1024, 0, st>>>(sq_blocks, norm_part, n * d, W, norms);
    CK_CUDA(cudaGetLastError());
    double h[2] = {0.0, 0.0};
    CK_CUDA(cudaMemcpyAsync(h, norms, sizeof(h), cudaMemcpyDeviceToHost, st));
    CK_CUDA(cudaStreamSynchronize(st));
    const double k2 = kp.var * kp.var * h[0];
    *colspace = std::sqrt(std::max(0.0, k2 - h[1]) / k2);
  }
  return ok();
}

// W (n x d) = var * K0 M for a dense right factor M (n x d FP32, ld ldm), FP32-accurate up to the
// tensor cores' accumulation over 4096-point ranges: M and the kernel entries in three BF16
// terms each.
static Error kernel_times_dense(ckinv_ctx *ctx, int64_t n, int dim, int d, const KernelParams &kp,
                                const float *points, const float *M, int64_t ldm, float *W, int64_t ldw,
                                cudaStream_t st) {
  const int64_t kpad = ceil_div(n, 64) * 64;
  const int num_kb = (int)(kpad / 64);
  const int splits = (int)ceil_div(num_kb, kMaxBlocksPerSplit);
  const int64_t ldp = ceil_div(n, 128) * 128;
  __nv_bfloat16 *Bt = nullptr;
  float *part = nullptr;
  CK_CUDA(dev_alloc(&Bt, sizeof(__nv_bfloat16) * 3 * d * kpad, st));
  if (dev_alloc(&part, sizeof(float) * (size_t)splits * ldp * d, st) != cudaSuccess) {
    cudaFreeAsync(Bt, st);
    return fail(CKINV_ENOMEM, "dense-Omega sketch workspace");
  }
  Error e = ok();
  note_launch();
  k_split_terms<<<dim3((unsigned)std::min<int64_t>(ceil_div(kpad, 256), 1024), d), 256, 0, st>>>(n, d, M, ldm, kpad,
                                                                                                 Bt);
  cudaError_t ce = cudaGetLastError();
  if (ce != cudaSuccess) e = fail(CKINV_ECUDA, cudaGetErrorString(ce));
  // the six term products of order at most two (keeping the two of order three changed the
  // measured error by nothing: the tensor cores' accumulation sets it)
  const int terms_of_entry[3] = {3, 2, 1};
  for (int t = 0; t < 3 && !e.st; ++t)
    e = sketch_tc_rhs(ctx, n, dim, d, terms_of_entry[t], kp, points, Bt + (size_t)t * d * kpad, kpad, splits, part, ldp,
                      t > 0, st);
  if (!e.st) {
    note_launch();
    k_fold_parts_f32<<<(unsigned)std::min<int64_t>(ceil_div(n * d, 256), 4096), 256, 0, st>>>(n, d, splits, part, ldp,
                                                                                              kp.var, W, ldw);
    ce = cudaGetLastError();
    if (ce != cudaSuccess) e = fail(CKINV_ECUDA, cudaGetErrorString(ce));
  }
  cudaFreeAsync(Bt, st);
  cudaFreeAsync(part, st);
  return e;
}

Error sketch_dense_omega(ckinv_ctx *ctx, int64_t n, int dim, int d, const KernelParams &kp, const float *points,
                         const float *Om, float *Y, int64_t ldy, cudaStream_t st) {
  return kernel_times_dense(ctx, n, dim, d, kp, points, Om, n, Y, ldy, st);
}

Error predict_mean(ckinv_ctx *ctx, int64_t n, int dim, const KernelParams &kp, const float *points, const float *alpha,
                   const float *xnew, int64_t n_new, double *mean, cudaStream_t st) {
  note_launch();
  k_predict_mean<<<(unsigned)ceil_div(n_new, kPredThreads), kPredThreads, 0, st>>>(n, n_new, dim, kp.kind, kp.ell,
                                                                                    kp.var, points, alpha, xnew, mean);
  CK_CUDA(cudaGetLastError());
  return ok();
}

}  // namespace ckinv
