// Strided-batched GEMM on the CUDA cores (FP32 or FP64), column-major:
//   C_b = alpha * op(A_b) * B_b + beta * C_b,   op(A) = A or A^T,   b = 0 .. batch-1,
// with a two-level batch b = b1 + nb1 * b2 (operand offset b1 * s + b2 * s2) for blocks that
// repeat inside each of several matrices.
// Used by the blocked Householder QR (trailing updates, compact-WY assembly and the
// application of Q to a coefficient block).
//
// CTA tile BM x BN, thread tile TM x TN (two TM/2 x TN/2 quadrants, so that the shared
// memory reads of a warp are conflict-free 16-byte vectors), BK = 8 deep (64 FP32 or 32 FP64
// rows for the narrow 32 x 32 tile, whose loop would otherwise wait out one global round trip
// per 8 rows),
// double-buffered through registers: the next k-slab is fetched from global memory while the
// current one is multiplied.  Split-K over gridDim.z writes one partial product per split to a
// workspace, and a second kernel adds them in split order (so results do not depend on
// the order in which blocks finish).
#include "internal.cuh"

namespace ckinv {
namespace {

template <typename T, int BM, int BN, int TM, int TN_, bool TRANSA, int BK>
__global__ void __launch_bounds__((BM / TM) * (BN / TN_), (TM * TN_ >= 64) ? 2 : 3)
    k_gemm(int M, int N, int K, T alpha, const T *__restrict__ A, int64_t lda, int64_t sA,
           const T *__restrict__ B, int64_t ldb, int64_t sB, T beta, T *__restrict__ C, int64_t ldc, int64_t sC,
           int ksplit, T *__restrict__ part, int nb1, int64_t sA2, int64_t sB2, int64_t sC2) {
  constexpr int NTX = BN / TN_, NTY = BM / TM;
  constexpr int NT = NTX * NTY;
  constexpr int LA = BM * BK / NT;   // A elements loaded per thread per slab
  constexpr int LB = BN * BK / NT;
  static_assert(LA >= 1 && LB >= 1, "tile too small for the thread count");
  __shared__ __align__(16) T As[2][BK][BM + 4];   // +4: conflict-free transposing stores
  __shared__ __align__(16) T Bs[2][BK][BN + 4];
  const int batch = blockIdx.z / ksplit, split = blockIdx.z % ksplit;
  const int b1 = batch % nb1, b2 = batch / nb1;
  A += (int64_t)b1 * sA + (int64_t)b2 * sA2;
  B += (int64_t)b1 * sB + (int64_t)b2 * sB2;
  if (ksplit > 1) {   // partial (split, batch) of the workspace: M x N, ld M
    C = part + ((int64_t)split * (gridDim.z / ksplit) + batch) * M * N;
    ldc = M;
  } else {
    C += (int64_t)b1 * sC + (int64_t)b2 * sC2;
  }
  const int m0 = blockIdx.x * BM, n0 = blockIdx.y * BN;
  const int kchunk = ((K + ksplit - 1) / ksplit + BK - 1) / BK * BK;
  const int kb = split * kchunk, ke = min(K, kb + kchunk);
  const int tid = threadIdx.x;
  const int tx = tid % NTX, ty = tid / NTX;

  T ra[LA], rb[LB];
  auto fetch = [&](int k0) {
#pragma unroll
    for (int q = 0; q < LA; ++q) {
      int e = tid + q * NT;
      int mm, kk;
      if (TRANSA) { kk = e % BK; mm = e / BK; }
      else { mm = e % BM; kk = e / BM; }
      int m = m0 + mm, k = k0 + kk;
      ra[q] = (m < M && k < ke) ? (TRANSA ? A[k + (int64_t)m * lda] : A[m + (int64_t)k * lda]) : T(0);
    }
#pragma unroll
    for (int q = 0; q < LB; ++q) {
      int e = tid + q * NT;
      int kk = e % BK, nn = e / BK;
      int n = n0 + nn, k = k0 + kk;
      rb[q] = (n < N && k < ke) ? B[k + (int64_t)n * ldb] : T(0);
    }
  };
  auto stash = [&](int buf) {
#pragma unroll
    for (int q = 0; q < LA; ++q) {
      int e = tid + q * NT;
      int mm, kk;
      if (TRANSA) { kk = e % BK; mm = e / BK; }
      else { mm = e % BM; kk = e / BM; }
      As[buf][kk][mm] = ra[q];
    }
#pragma unroll
    for (int q = 0; q < LB; ++q) {
      int e = tid + q * NT;
      int kk = e % BK, nn = e / BK;
      Bs[buf][kk][nn] = rb[q];
    }
  };

  T acc[TM][TN_];
#pragma unroll
  for (int i = 0; i < TM; ++i)
#pragma unroll
    for (int j = 0; j < TN_; ++j) acc[i][j] = T(0);

  // Thread (tx, ty) owns rows {ty*TM/2 .. +TM/2} and {BM/2 + ty*TM/2 ..}, columns likewise.
  constexpr int HM = TM / 2, HN = TN_ / 2;
  int buf = 0;
  if (kb < ke) {
    fetch(kb);
    stash(0);
  }
  __syncthreads();
  for (int k0 = kb; k0 < ke; k0 += BK) {
    const bool more = (k0 + BK < ke);
    if (more) fetch(k0 + BK);
#pragma unroll
    for (int kk = 0; kk < BK; ++kk) {
      T a[TM], b[TN_];
#pragma unroll
      for (int i = 0; i < HM; ++i) {
        a[i] = As[buf][kk][ty * HM + i];
        a[HM + i] = As[buf][kk][BM / 2 + ty * HM + i];
      }
#pragma unroll
      for (int j = 0; j < HN; ++j) {
        b[j] = Bs[buf][kk][tx * HN + j];
        b[HN + j] = Bs[buf][kk][BN / 2 + tx * HN + j];
      }
#pragma unroll
      for (int i = 0; i < TM; ++i)
#pragma unroll
        for (int j = 0; j < TN_; ++j) acc[i][j] = fma(a[i], b[j], acc[i][j]);
    }
    if (more) {
      stash(buf ^ 1);
      __syncthreads();
      buf ^= 1;
    }
  }
#pragma unroll
  for (int i = 0; i < TM; ++i) {
    int m = m0 + (i < HM ? ty * HM + i : BM / 2 + ty * HM + (i - HM));
    if (m >= M) continue;
#pragma unroll
    for (int j = 0; j < TN_; ++j) {
      int n = n0 + (j < HN ? tx * HN + j : BN / 2 + tx * HN + (j - HN));
      if (n >= N) continue;
      T *c = C + m + (int64_t)n * ldc;
      if (ksplit > 1) *c = alpha * acc[i][j];
      else *c = alpha * acc[i][j] + (beta == T(0) ? T(0) : beta * *c);
    }
  }
}

// C_b = beta C_b + sum over s (in order) of part[s][b]
template <typename T>
__global__ void k_splitk_reduce(int M, int N, int batch, int ksplit, const T *part, T beta, T *C, int64_t ldc,
                                int64_t sC, int nb1, int64_t sC2) {
  const int64_t per = (int64_t)M * N;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < per * batch;
       e += (int64_t)gridDim.x * blockDim.x) {
    int64_t b = e / per, w = e % per;
    T acc = T(0);
    for (int s = 0; s < ksplit; ++s) acc += part[((int64_t)s * batch + b) * per + w];
    T *c = C + (b % nb1) * sC + (b / nb1) * sC2 + (w % M) + (w / M) * ldc;
    *c = acc + (beta == T(0) ? T(0) : beta * *c);
  }
}

template <typename T, int BM, int BN, int TM, int TN_, int BK = 8>
void launch_shape(bool transA, int M, int N, int K, T alpha, const T *A, int64_t lda, int64_t sA, const T *B,
                  int64_t ldb, int64_t sB, T beta, T *C, int64_t ldc, int64_t sC, int batch, int ksplit,
                  T *part, int nb1, int64_t sA2, int64_t sB2, int64_t sC2, cudaStream_t st) {
  dim3 grid((unsigned)ceil_div(M, BM), (unsigned)ceil_div(N, BN), (unsigned)(batch * ksplit));
  constexpr int NT = (BM / TM) * (BN / TN_);
  note_launch();
  if (transA)
    k_gemm<T, BM, BN, TM, TN_, true, BK><<<grid, NT, 0, st>>>(M, N, K, alpha, A, lda, sA, B, ldb, sB, beta, C, ldc,
                                                              sC, ksplit, part, nb1, sA2, sB2, sC2);
  else
    k_gemm<T, BM, BN, TM, TN_, false, BK><<<grid, NT, 0, st>>>(M, N, K, alpha, A, lda, sA, B, ldb, sB, beta, C, ldc,
                                                               sC, ksplit, part, nb1, sA2, sB2, sC2);
}

}  // namespace

template <typename T>
Error gemm_simt(const ckinv_ctx *ctx, bool transA, int M, int N, int K, T alpha, const T *A, int64_t lda, int64_t sA,
                const T *B, int64_t ldb, int64_t sB, T beta, T *C, int64_t ldc, int64_t sC, int nb1, int64_t sA2,
                int64_t sB2, int64_t sC2, int nb2, cudaStream_t st) {
  const int batch = nb1 * nb2;
  // tile choice: 128 x 128 (8 x 8 per thread) for large FP32 outputs, 32 x 32 (2 x 2) for
  // outputs of at most 32 x 32 (the inner products of narrow Householder blocks, where a
  // 64 x 64 tile would compute 4 to 16 times the output), else 64 x 64 (4 x 4)
  const bool big = (sizeof(T) == 4) && M >= 256 && N >= 128;
  const bool small = M <= 32 && N <= 32;
  const int bm = big ? 128 : small ? 32 : 64, bn = bm;
  const int64_t tiles = ceil_div(M, bm) * ceil_div(N, bn) * (int64_t)batch;
  int ksplit = 1;
  // split K while the output tiles alone would leave SMs idle: up to four CTAs per SM for FP32
  // (these products are short of parallelism, not of arithmetic), two for FP64
  const int64_t target = (sizeof(T) == 4 ? 4LL : 2LL) * ctx->sm_count;
  if (tiles < target && K >= 256) {
    ksplit = (int)std::min<int64_t>(std::max<int64_t>(1, target / tiles), K / 128);
    ksplit = std::max(ksplit, 1);
  }
  T *part = nullptr;
  if (ksplit > 1) CK_CUDA(dev_alloc((void **)&part, sizeof(T) * (size_t)M * N * batch * ksplit, st));
  if (big)
    launch_shape<T, 128, 128, 8, 8>(transA, M, N, K, alpha, A, lda, sA, B, ldb, sB, beta, C, ldc, sC, batch, ksplit,
                                    part, nb1, sA2, sB2, sC2, st);
  else if (small)   // deep k-slabs (36 KB of static shared memory): a narrow tile's loop is bound by round trips
    launch_shape<T, 32, 32, 2, 2, sizeof(T) == 4 ? 64 : 32>(transA, M, N, K, alpha, A, lda, sA, B, ldb, sB, beta, C,
                                                            ldc, sC, batch, ksplit, part, nb1, sA2, sB2, sC2, st);
  else
    launch_shape<T, 64, 64, 4, 4>(transA, M, N, K, alpha, A, lda, sA, B, ldb, sB, beta, C, ldc, sC, batch, ksplit,
                                  part, nb1, sA2, sB2, sC2, st);
  if (ksplit > 1) {
    unsigned g = (unsigned)std::min<int64_t>(ceil_div((int64_t)M * N * batch, 256), 4096);
    note_launch();
    k_splitk_reduce<T><<<g, 256, 0, st>>>(M, N, batch, ksplit, part, beta, C, ldc, sC, nb1, sC2);
    cudaFreeAsync(part, st);
  }
  CK_CUDA(cudaGetLastError());
  return ok();
}

template <typename T>
Error gemm_batched(const ckinv_ctx *ctx, bool transA, int M, int N, int K, T alpha, const T *A, int64_t lda,
                   int64_t sA, const T *B, int64_t ldb, int64_t sB, T beta, T *C, int64_t ldc, int64_t sC,
                   int batch, cudaStream_t st) {
  if (M <= 0 || N <= 0 || batch <= 0) return ok();
  if (K <= 0) {
    if (beta == T(1)) return ok();
    return fail(CKINV_EINVAL, "gemm_batched: K = 0 with beta != 1");
  }
  // FP32 products big enough to fill 128 x 128 tensor-core tiles over at least four K blocks
  // go to the tensor cores (with fewer, a tile's fixed costs - TMEM allocation, pipeline fill,
  // the epilogue's read-modify-write - outweigh its MMAs)
  if (sizeof(T) == 4 && ctx->gemm_tc && M >= 64 && N >= 64 && K >= 256 &&
      (double)M * N * (double)K * batch >= 3.0e7)
    return gemm_tc_f32(ctx, transA, M, N, K, (float)alpha, (const float *)A, lda, sA, (const float *)B, ldb, sB,
                       (float)beta, (float *)C, ldc, sC, batch, st);
  return gemm_simt<T>(ctx, transA, M, N, K, alpha, A, lda, sA, B, ldb, sB, beta, C, ldc, sC, batch, 0, 0, 0, 1, st);
}

template <typename T>
Error gemm_batched2(const ckinv_ctx *ctx, bool transA, int M, int N, int K, T alpha, const T *A, int64_t lda,
                    int64_t sA, int64_t sA2, const T *B, int64_t ldb, int64_t sB, int64_t sB2, T beta, T *C,
                    int64_t ldc, int64_t sC, int64_t sC2, int nb1, int nb2, cudaStream_t st) {
  if (M <= 0 || N <= 0 || nb1 <= 0 || nb2 <= 0) return ok();
  if (K <= 0) {
    if (beta == T(1)) return ok();
    return fail(CKINV_EINVAL, "gemm_batched2: K = 0 with beta != 1");
  }
  return gemm_simt<T>(ctx, transA, M, N, K, alpha, A, lda, sA, B, ldb, sB, beta, C, ldc, sC, nb1, sA2, sB2, sC2, nb2,
                      st);
}

template Error gemm_batched2<float>(const ckinv_ctx *, bool, int, int, int, float, const float *, int64_t, int64_t,
                                    int64_t, const float *, int64_t, int64_t, int64_t, float, float *, int64_t,
                                    int64_t, int64_t, int, int, cudaStream_t);
template Error gemm_batched<float>(const ckinv_ctx *, bool, int, int, int, float, const float *, int64_t, int64_t,
                                   const float *, int64_t, int64_t, float, float *, int64_t, int64_t, int,
                                   cudaStream_t);
template Error gemm_batched<double>(const ckinv_ctx *, bool, int, int, int, double, const double *, int64_t,
                                    int64_t, const double *, int64_t, int64_t, double, double *, int64_t, int64_t,
                                    int, cudaStream_t);

}  // namespace ckinv
