// Low-rank core and solve (Sec. 1: K^-1 A = R^-1 Q^T A; proof of Theorem 3:
// P_Khat K = R^-1 Q^T K), completed with a nugget in Woodbury form:
//   B = Omega^T Q_hat,  C' = R^T + tau B,
//   K_tilde^-1 A = tau^-1 (A - Q_hat C'^-1 R^T Q_hat^T A),
//   K_tilde X = tau X + Q_hat B^-1 R^T Q_hat^T X    (refinement residual, FP64).
// Long contractions over the n rows run on the CUDA cores in FP32 with FP64 accumulation
// across 256-row chunks; every d x d operation (LU, triangular solves) is FP64.
#include "internal.cuh"

namespace ckinv {
namespace {

// ---------------------------------------------------------------- G = L^T M over n rows
// Tile TM x TN of G per CTA (64 x 64, or 128 x 32 for a narrow right factor), rows split
// over gridDim.z chunks; FP32 FMA inside 256-row sub-chunks, FP64 accumulation across them;
// chunk z writes its partial product to G + z d1 d2, and the partials are folded in chunk
// order afterwards (deterministic).
template <bool OMEGA, int TM, int TN>
__global__ void __launch_bounds__(256) k_tsprod(int64_t n, int d1, int d2, const float *__restrict__ L,
                                                int64_t ldl, const uint32_t *__restrict__ bits,
                                                const int32_t *__restrict__ cols, double oscale,
                                                const float *__restrict__ M, int64_t ldm, double *G,
                                                int64_t rows_per_split, int64_t orow0) {
  static_assert((TM / 4) * (TN / 4) == 256, "4 x 4 outputs per thread");
  __shared__ float Ls[32][TM + 4];
  __shared__ float Ms[32][TN + 4];
  __shared__ uint32_t pc[TM];
  const int tid = threadIdx.x, tx = tid % (TN / 4), ty = tid / (TN / 4);
  const int i0 = blockIdx.x * TM, j0 = blockIdx.y * TN;
  const int64_t rb = (int64_t)blockIdx.z * rows_per_split;
  const int64_t re = min(n, rb + rows_per_split);
  if (OMEGA)
    for (int c = tid; c < TM; c += 256) pc[c] = (i0 + c < d1) ? (uint32_t)cols[i0 + c] : 0u;
  float acc[4][4];
  double accd[4][4];
#pragma unroll
  for (int a = 0; a < 4; ++a)
#pragma unroll
    for (int b = 0; b < 4; ++b) { acc[a][b] = 0.f; accd[a][b] = 0.0; }
  __syncthreads();
  // the next 32 rows are fetched into registers while the current ones are multiplied
  float lr[TM / 8], mr[TN / 8];
  auto fetch = [&](int64_t k0) {
#pragma unroll
    for (int q = 0; q < TM / 8; ++q) {
      int e = tid + 256 * q;
      int kk = e % 32, c = e / 32;
      int64_t k = k0 + kk;
      float lv = 0.f;
      if (k < re && i0 + c < d1) {
        if (OMEGA) {
          const int64_t kg = orow0 + k;           // row of Omega (a row shard starts at orow0)
          uint32_t s = (bits[kg >> 5] >> (kg & 31)) & 1u;
          s ^= (uint32_t)(__popcll((unsigned long long)kg & (unsigned long long)pc[c]) & 1);
          lv = s ? -1.0f : 1.0f;
        } else {
          lv = L[k + (int64_t)(i0 + c) * ldl];
        }
      }
      lr[q] = lv;
    }
#pragma unroll
    for (int q = 0; q < TN / 8; ++q) {
      int e = tid + 256 * q;
      int kk = e % 32, c = e / 32;
      int64_t k = k0 + kk;
      mr[q] = (k < re && j0 + c < d2) ? M[k + (int64_t)(j0 + c) * ldm] : 0.f;
    }
  };
  if (rb < re) fetch(rb);
  int step = 0;
  for (int64_t k0 = rb; k0 < re; k0 += 32) {
#pragma unroll
    for (int q = 0; q < TM / 8; ++q) {
      int e = tid + 256 * q;
      Ls[e % 32][e / 32] = lr[q];
    }
#pragma unroll
    for (int q = 0; q < TN / 8; ++q) {
      int e = tid + 256 * q;
      Ms[e % 32][e / 32] = mr[q];
    }
    __syncthreads();
    if (k0 + 32 < re) fetch(k0 + 32);
#pragma unroll 8
    for (int kk = 0; kk < 32; ++kk) {
      float a[4], b[4];
#pragma unroll
      for (int t = 0; t < 4; ++t) { a[t] = Ls[kk][ty * 4 + t]; b[t] = Ms[kk][tx * 4 + t]; }
#pragma unroll
      for (int x = 0; x < 4; ++x)
#pragma unroll
        for (int y = 0; y < 4; ++y) acc[x][y] = fmaf(a[x], b[y], acc[x][y]);
    }
    __syncthreads();
    if (++step == 8) {
      step = 0;
#pragma unroll
      for (int x = 0; x < 4; ++x)
#pragma unroll
        for (int y = 0; y < 4; ++y) { accd[x][y] += (double)acc[x][y]; acc[x][y] = 0.f; }
    }
  }
#pragma unroll
  for (int x = 0; x < 4; ++x)
#pragma unroll
    for (int y = 0; y < 4; ++y) {
      int i = i0 + ty * 4 + x, j = j0 + tx * 4 + y;
      if (i < d1 && j < d2)
        G[(int64_t)blockIdx.z * d1 * d2 + i + (int64_t)j * d1] = (OMEGA ? oscale : 1.0) * (accd[x][y] + (double)acc[x][y]);
    }
}

// ---------------------------------------------------------------- residual-grade sums
// Products of two FP32 numbers are split exactly into p + e (p = fl(ab), e = fma(a, b, -p));
// the p's are summed with TwoSum compensation and the e's plainly (they are 2^-24 smaller),
// and each 256-row chunk is folded into FP64.  This gives sums accurate to about 2^-48 at
// FP32 throughput, for the residual of the FP64 refinement step.
__device__ __forceinline__ void two_sum(float a, float b, float &s, float &err) {
  s = a + b;
  float bb = s - a;
  err = (a - (s - bb)) + (b - bb);
}

// Partial z of G (d1 x d2, FP64, ld d1) = L^T M over rows [rb, re) (L, M FP32), compensated.
__global__ void __launch_bounds__(256) k_tsprod_dd(int64_t n, int d1, int d2, const float *__restrict__ L,
                                                   int64_t ldl, const float *__restrict__ M, int64_t ldm,
                                                   double *G, int64_t rows_per_split) {
  __shared__ float Ls[32][64 + 4];
  __shared__ float Ms[32][32 + 4];
  const int tid = threadIdx.x, tx = tid % 16, ty = tid / 16;   // 64 x 32 tile: 4 x 2 per thread
  const int i0 = blockIdx.x * 64, j0 = blockIdx.y * 32;
  const int64_t rb = (int64_t)blockIdx.z * rows_per_split;
  const int64_t re = min(n, rb + rows_per_split);
  float hs[4][2], lc[4][2];
  double acc[4][2];
#pragma unroll
  for (int a = 0; a < 4; ++a)
#pragma unroll
    for (int b = 0; b < 2; ++b) { hs[a][b] = 0.f; lc[a][b] = 0.f; acc[a][b] = 0.0; }
  // the next 32 rows are fetched into registers while the current ones are multiplied
  float lr[8], mr[4];
  auto fetch = [&](int64_t k0) {
#pragma unroll
    for (int q = 0; q < 8; ++q) {
      int e = tid + 256 * q;
      int kk = e % 32, c = e / 32;
      int64_t k = k0 + kk;
      lr[q] = (k < re && i0 + c < d1) ? L[k + (int64_t)(i0 + c) * ldl] : 0.f;
    }
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      int e = tid + 256 * q;
      int kk = e % 32, c = e / 32;
      int64_t k = k0 + kk;
      mr[q] = (k < re && j0 + c < d2) ? M[k + (int64_t)(j0 + c) * ldm] : 0.f;
    }
  };
  if (rb < re) fetch(rb);
  int step = 0;
  for (int64_t k0 = rb; k0 < re; k0 += 32) {
#pragma unroll
    for (int q = 0; q < 8; ++q) {
      int e = tid + 256 * q;
      Ls[e % 32][e / 32] = lr[q];
    }
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      int e = tid + 256 * q;
      Ms[e % 32][e / 32] = mr[q];
    }
    __syncthreads();
    if (k0 + 32 < re) fetch(k0 + 32);
#pragma unroll 4
    for (int kk = 0; kk < 32; ++kk) {
      float b0 = Ms[kk][tx * 2], b1 = Ms[kk][tx * 2 + 1];
#pragma unroll
      for (int x = 0; x < 4; ++x) {
        float a = Ls[kk][ty * 4 + x];
        float p0 = a * b0, e0 = fmaf(a, b0, -p0);
        float p1 = a * b1, e1 = fmaf(a, b1, -p1);
        float s0, r0, s1, r1;
        two_sum(hs[x][0], p0, s0, r0);
        two_sum(hs[x][1], p1, s1, r1);
        hs[x][0] = s0; lc[x][0] += r0 + e0;
        hs[x][1] = s1; lc[x][1] += r1 + e1;
      }
    }
    __syncthreads();
    if (++step == 8) {
      step = 0;
#pragma unroll
      for (int x = 0; x < 4; ++x)
#pragma unroll
        for (int y = 0; y < 2; ++y) {
          acc[x][y] += (double)hs[x][y] + (double)lc[x][y];
          hs[x][y] = 0.f;
          lc[x][y] = 0.f;
        }
    }
  }
#pragma unroll
  for (int x = 0; x < 4; ++x)
#pragma unroll
    for (int y = 0; y < 2; ++y) {
      int i = i0 + ty * 4 + x, j = j0 + tx * 2 + y;
      if (i < d1 && j < d2)
        G[(int64_t)blockIdx.z * d1 * d2 + i + (int64_t)j * d1] = acc[x][y] + (double)hs[x][y] + (double)lc[x][y];
    }
}

// r = A - tau X - Q S  (Q FP32 n x d, S FP64 d x m), compensated FP32 sums, FP64 combination.
__global__ void __launch_bounds__(256) k_residual_dd(int64_t n, int d, int m, const float *__restrict__ Q,
                                                     int64_t ldq, const double *__restrict__ S,
                                                     const float *__restrict__ A, int64_t lda,
                                                     const float *__restrict__ X, int64_t ldx, double tau, float *Rs,
                                                     int64_t ldr) {
  __shared__ __align__(16) float Sh[64][16], Sl[64][16];   // read as broadcast float4s
  const int tid = threadIdx.x;
  const int64_t i = (int64_t)blockIdx.x * 256 + tid;
  const int c0 = blockIdx.y * 16;
  const int mc = min(16, m - c0);
  float hs[16], lc[16];
#pragma unroll
  for (int c = 0; c < 16; ++c) { hs[c] = 0.f; lc[c] = 0.f; }
  for (int k0 = 0; k0 < d; k0 += 64) {
    __syncthreads();
    for (int e = tid; e < 64 * 16; e += 256) {
      int kk = e % 64, c = e / 64;
      double v = (k0 + kk < d && c < mc) ? S[(k0 + kk) + (int64_t)(c0 + c) * d] : 0.0;
      float hi = (float)v;
      Sh[kk][c] = hi;
      Sl[kk][c] = (float)(v - (double)hi);
    }
    __syncthreads();
    if (i < n) {
      const int kmax = min(64, d - k0);
      for (int kb = 0; kb < kmax; kb += 16) {     // sixteen loads of Q in flight per thread
        float qv[16];
#pragma unroll
        for (int u = 0; u < 16; ++u) qv[u] = (kb + u < kmax) ? Q[i + (int64_t)(k0 + kb + u) * ldq] : 0.f;
#pragma unroll
        for (int t = 0; t < 16; ++t) {
          const float q = qv[t];
          const int kk = kb + t;
#pragma unroll
          for (int c4 = 0; c4 < 4; ++c4) {
            const float4 h4 = *reinterpret_cast<const float4 *>(&Sh[kk][4 * c4]);
            const float4 l4 = *reinterpret_cast<const float4 *>(&Sl[kk][4 * c4]);
            const float hv[4] = {h4.x, h4.y, h4.z, h4.w}, lv[4] = {l4.x, l4.y, l4.z, l4.w};
#pragma unroll
            for (int u = 0; u < 4; ++u) {
              const int c = 4 * c4 + u;
              float p = q * hv[u], e = fmaf(q, hv[u], -p);
              float sum, r;
              two_sum(hs[c], p, sum, r);
              hs[c] = sum;
              lc[c] += r + fmaf(q, lv[u], e);
            }
          }
        }
      }
    }
  }
  if (i < n)
#pragma unroll
    for (int c = 0; c < 16; ++c) {       // a compile-time bound keeps hs, lc in registers
      if (c >= mc) break;
      double qs = (double)hs[c] + (double)lc[c];
      double a = (double)A[i + (int64_t)(c0 + c) * lda];
      double x = (double)X[i + (int64_t)(c0 + c) * ldx];
      Rs[i + (int64_t)(c0 + c) * ldr] = (float)(a - tau * x - qs);
    }
}

// ---------------------------------------------------------------- LU (FP64, blocked)
// Panel step of a right-looking blocked LU with partial pivoting on nmat strided d x d
// matrices (ld d): rows k0 .. d-1 of columns k0 .. k0+kb-1 of matrix blockIdx.x are
// loaded into shared memory and factored there (pivot search, interchange within the
// panel, scaling, rank-1 updates); piv[j] is the LAPACK interchange and logabs[m]
// accumulates log|U_jj|.  The interchanges are applied to the other columns afterwards
// (k_lu_laswp).  FP64 instructions are scarce on this part (an FP64 warp instruction
// holds a scheduler's FP64 unit for 64 cycles), so the pivot search compares |x| as
// integer keys (the bits of a non-negative double order like its value), one thread forms
// the pivot's reciprocal, and the logarithms of the panel's diagonal are taken together at
// the end.  Per column: one barrier after the warps post their candidates (every thread
// then picks the winner itself), one after the interchange, one after the update.
constexpr int kLuPanelThreads = 512;
__global__ void __launch_bounds__(kLuPanelThreads) k_lu_panel(int d, int k0, int kb, double *A0, int32_t *piv0,
                                                              double *logabs, int *err) {
  extern __shared__ double P[];          // (d - k0) x kb, ld R
  __shared__ unsigned long long wkey[kLuPanelThreads / 32];
  __shared__ double wsgn[kLuPanelThreads / 32];
  __shared__ int widx[kLuPanelThreads / 32];
  __shared__ double s_inv;
  const int m = blockIdx.x;
  double *A = A0 + (int64_t)m * d * d;
  int32_t *piv = piv0 + (int64_t)m * d;
  const int R = d - k0;
  const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
  const int nw = (int)(blockDim.x >> 5);
  for (int c0 = 0; c0 < kb; c0 += 8) {   // eight loads in flight per thread
    for (int i = tid; i < R; i += blockDim.x) {
      double t[8];
#pragma unroll
      for (int u = 0; u < 8; ++u) t[u] = (c0 + u < kb) ? A[(k0 + i) + (int64_t)(k0 + c0 + u) * d] : 0.0;
#pragma unroll
      for (int u = 0; u < 8; ++u)
        if (c0 + u < kb) P[i + (c0 + u) * R] = t[u];
    }
  }
  __syncthreads();
  for (int j = 0; j < kb; ++j) {
    // pivot: largest |P[i, j]| over i >= j, ties to the smaller row
    unsigned long long best = 0ull;
    double bsg = 0.0;
    int bi = j;
    for (int i = j + tid; i < R; i += blockDim.x) {
      const double x = P[i + j * R];
      const unsigned long long k = (unsigned long long)__double_as_longlong(x) & 0x7fffffffffffffffull;
      if (k > best) { best = k; bsg = x; bi = i; }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      const unsigned long long ok = __shfl_down_sync(0xffffffffu, best, o);
      const double os = __shfl_down_sync(0xffffffffu, bsg, o);
      const int oi = __shfl_down_sync(0xffffffffu, bi, o);
      if (ok > best || (ok == best && oi < bi)) { best = ok; bsg = os; bi = oi; }
    }
    if (lane == 0) { wkey[wid] = best; wsgn[wid] = bsg; widx[wid] = bi; }
    __syncthreads();
    unsigned long long bk = wkey[0];
    int p = widx[0], pw = 0;
    for (int w = 1; w < nw; ++w) {
      const unsigned long long k = wkey[w];
      const int xi = widx[w];
      if (k > bk || (k == bk && xi < p)) { bk = k; p = xi; pw = w; }
    }
    if (p != j && tid < kb) {
      const double t = P[j + tid * R];
      P[j + tid * R] = P[p + tid * R];
      P[p + tid * R] = t;
    }
    if (tid == 0) {
      piv[k0 + j] = k0 + p;
      if (bk == 0ull || bk >= 0x7ff0000000000000ull) {   // a zero, infinite or NaN pivot
        atomicOr(err, DERR_SINGULAR);
        s_inv = 0.0;
      } else {
        s_inv = 1.0 / wsgn[pw];
      }
    }
    __syncthreads();
    const double inv = s_inv;
    for (int i = j + 1 + tid; i < R; i += blockDim.x) {   // scale, then rank-1 update of the row
      const double l = P[i + j * R] * inv;
      P[i + j * R] = l;
      for (int c = j + 1; c < kb; ++c) P[i + c * R] = fma(-l, P[j + c * R], P[i + c * R]);
    }
    __syncthreads();
  }
  for (int c = 0; c < kb; ++c)
    for (int i = tid; i < R; i += blockDim.x) A[(k0 + i) + (int64_t)(k0 + c) * d] = P[i + c * R];
  if (wid == 0) {                        // sum of log|U_jj| over the panel, fixed order
    double la = 0.0;
    for (int j = lane; j < kb; j += 32) {
      const double u = P[j + j * R];
      if (u != 0.0) la += log(fabs(u));
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) la += __shfl_xor_sync(0xffffffffu, la, o);
    if (lane == 0) logabs[m] += la;
  }
}

// The panel's interchanges (rows k0 .. k0+kb-1) applied to every column outside the panel.
__global__ void k_lu_laswp(int d, int k0, int kb, double *A0, const int32_t *piv0) {
  double *A = A0 + (int64_t)blockIdx.y * d * d;
  const int32_t *piv = piv0 + (int64_t)blockIdx.y * d;
  int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= d - kb) return;
  if (c >= k0) c += kb;                  // skip the panel's own columns
  double *col = A + (int64_t)c * d;
  for (int j = k0; j < k0 + kb; ++j) {
    int p = piv[j];
    if (p != j) { double t = col[j]; col[j] = col[p]; col[p] = t; }
  }
}

// A[k0:k0+kb, k0+kb:d] <- L11^-1 A[k0:k0+kb, k0+kb:d]  (L11 unit lower, kb <= 32), one
// thread per column: the column's kb entries in registers, L11 staged in shared memory
// and read as broadcasts, substitution by columns of L11 (independent FMAs per step).
constexpr int kLuTrsmThreads = 32;
__global__ void __launch_bounds__(kLuTrsmThreads) k_lu_trsm(int d, int k0, int kb, double *A0) {
  __shared__ double L[32 * 32];
  double *A = A0 + (int64_t)blockIdx.y * d * d;
  for (int e = threadIdx.x; e < kb * kb; e += blockDim.x) {
    const int i = e % kb, j = e / kb;
    L[i + 32 * j] = A[(k0 + i) + (int64_t)(k0 + j) * d];
  }
  __syncthreads();
  const int c = k0 + kb + blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= d) return;
  double *col = A + (int64_t)c * d + k0;
  double v[32];
#pragma unroll
  for (int i = 0; i < 32; ++i) v[i] = (i < kb) ? col[i] : 0.0;
#pragma unroll
  for (int j = 0; j < 31; ++j) {
#pragma unroll
    for (int i = j + 1; i < 32; ++i)
      if (i < kb) v[i] = fma(-L[i + 32 * j], v[j], v[i]);
  }
#pragma unroll
  for (int i = 0; i < 32; ++i)
    if (i < kb) col[i] = v[i];
}

// ---------------------------------------------------------------- triangular solves
// X (d x m, ld d) <- op(A)^-1 X with A = P L U packed (LAPACK interchanges), d <= 512.
// One block of four warps per right-hand side; row i of the vector lives in a register of
// thread i % 128 (slot i / 128), so the FP64 FMAs use all four schedulers of the SM.  The
// two triangular passes go by chunks of kSolveChunk unknowns: the warp that owns the
// chunk's rows solves its diagonal block by substitution (a shuffle and an FMA per
// unknown), then every thread applies the chunk to its rows still to be solved.  The
// factor streams through two shared-memory buffers, the next chunk copied by cp.async
// while the current one is applied: a column block of L or U for A, a row block (stride
// kSolveChunk + 1, against bank conflicts) for A^T.  The diagonal of U enters as
// reciprocals formed once per launch, so no divide lies on the substitution chain.
constexpr int kSolveThreads = 128;
constexpr int kSolveSlots = 4;                 // rows per thread: i = s * 128 + threadIdx.x
constexpr int kSolveChunk = 16;
constexpr int kSolveLdT = kSolveChunk + 1;
__device__ __forceinline__ double slot_get(const double (&v)[kSolveSlots], int s) {
  double r = 0.0;
#pragma unroll
  for (int t = 0; t < kSolveSlots; ++t) r = (t == s) ? v[t] : r;
  return r;
}
__device__ __forceinline__ void slot_set(double (&v)[kSolveSlots], int s, double x) {
#pragma unroll
  for (int t = 0; t < kSolveSlots; ++t) v[t] = (t == s) ? x : v[t];
}
template <int R>
__device__ __forceinline__ double slot_get_r(const double (&v)[kSolveSlots][R], int s, int r) {
  double x = 0.0;
#pragma unroll
  for (int t = 0; t < kSolveSlots; ++t) x = (t == s) ? v[t][r] : x;
  return x;
}
template <int R>
__device__ __forceinline__ void slot_set_r(double (&v)[kSolveSlots][R], int s, int r, double x) {
#pragma unroll
  for (int t = 0; t < kSolveSlots; ++t) v[t][r] = (t == s) ? x : v[t][r];
}
__device__ __forceinline__ void cp_async8(double *dst, const double *src) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"((unsigned)__cvta_generic_to_shared(dst)),
               "l"(src)
               : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() {
  asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory");
}

template <int R>
__global__ void __launch_bounds__(kSolveThreads) k_lu_solve(int d, int m, const double *__restrict__ LU,
                                                            const int32_t *__restrict__ piv, double *X, int trans) {
  extern __shared__ __align__(16) double sm[];
  const int bufsz = kSolveLdT * d;
  double *xs = sm + 2 * (size_t)bufsz;                 // R vectors, for the interchanges
  double *xc = xs + (size_t)R * d;                     // two chunks of solved unknowns per vector
  int32_t *ps = reinterpret_cast<int32_t *>(xc + 2 * R * kSolveChunk);
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int c0 = blockIdx.x * R;                       // this block's first right-hand side
  const int nr = min(R, m - c0);
  const int nchunk = (d + kSolveChunk - 1) / kSolveChunk;
  // chunk-steps 0 .. 2 nchunk - 1: the first pass ascends (forward), the second descends
  auto chunk_of = [&](int k) { return k < nchunk ? k : 2 * nchunk - 1 - k; };
  auto issue = [&](int k) {
    const int j0 = chunk_of(k) * kSolveChunk;
    const int w = min(kSolveChunk, d - j0);
    const bool fwd = k < nchunk;
    double *dst = sm + (size_t)(k & 1) * bufsz;
    if (!trans) {      // columns j0 .. j0+w of L (rows j0..d) or U (rows 0..j0+w)
      const int lo = fwd ? j0 : 0, hi = fwd ? d : j0 + w;
      for (int jj = 0; jj < w; ++jj)
        for (int r = lo + tid; r < hi; r += kSolveThreads)
          cp_async8(dst + (size_t)jj * d + r, LU + (int64_t)(j0 + jj) * d + r);
    } else {           // rows j0 .. j0+w of U (columns j0..d) or L (columns 0..j0+w)
      const int lo = fwd ? j0 : 0, hi = fwd ? d : j0 + w;
      for (int e = tid; e < (hi - lo) * kSolveChunk; e += kSolveThreads) {
        const int i = lo + (e >> 4), jj = e & (kSolveChunk - 1);
        if (jj < w) cp_async8(dst + (size_t)i * kSolveLdT + jj, LU + (int64_t)i * d + j0 + jj);
      }
    }
    cp_async_commit();
  };
  issue(0);
  for (int i = tid; i < d; i += kSolveThreads) ps[i] = piv[i];
  for (int r = 0; r < R; ++r)
    for (int i = tid; i < d; i += kSolveThreads) xs[(size_t)r * d + i] = r < nr ? X[(int64_t)(c0 + r) * d + i] : 0.0;
  __syncthreads();
  if (!trans && tid < R) {
    double *xr = xs + (size_t)tid * d;
    for (int j = 0; j < d; ++j) {
      const int p = ps[j];
      if (p != j) { double t = xr[j]; xr[j] = xr[p]; xr[p] = t; }
    }
  }
  __syncthreads();
  double v[kSolveSlots][R], rd[kSolveSlots];
#pragma unroll
  for (int s = 0; s < kSolveSlots; ++s) {
    const int i = s * kSolveThreads + tid;
#pragma unroll
    for (int r = 0; r < R; ++r) v[s][r] = i < d ? xs[(size_t)r * d + i] : 0.0;
    rd[s] = i < d ? 1.0 / LU[(int64_t)i * d + i] : 0.0;
  }
  for (int k = 0; k < 2 * nchunk; ++k) {
    if (k + 1 < 2 * nchunk) {
      issue(k + 1);
      cp_async_wait<1>();
    } else {
      cp_async_wait<0>();
    }
    __syncthreads();
    const double *cb = sm + (size_t)(k & 1) * bufsz;
    // op(A)(i, j0 + jj) from the staged block
    auto opA = [&](int i, int jj) -> double {
      return trans ? cb[(size_t)i * kSolveLdT + jj] : cb[(size_t)jj * d + i];
    };
    const bool fwd = k < nchunk;
    const bool unit = trans ? !fwd : fwd;      // L and L^T have a unit diagonal
    const int j0 = chunk_of(k) * kSolveChunk;
    const int w = min(kSolveChunk, d - j0);
    double *xck = xc + (k & 1) * R * kSolveChunk;
    // 1. diagonal block, by the warp that owns rows j0 .. j0+w (all in one slot); the
    // vectors' substitutions are independent chains, interleaved
    if (warp == ((j0 % kSolveThreads) >> 5)) {
      const int q0 = j0 / kSolveThreads;
      const int i = q0 * kSolveThreads + tid;
      double vq[R];
#pragma unroll
      for (int r = 0; r < R; ++r) vq[r] = slot_get_r<R>(v, q0, r);
      const double rq = slot_get(rd, q0);
      const bool mine = i >= j0 && i < j0 + w;
      for (int t = 0; t < w; ++t) {
        const int jj = fwd ? t : w - 1 - t;
        const int j = j0 + jj;
        const double a = (mine && (fwd ? i > j : i < j)) ? opA(i, jj) : 0.0;
#pragma unroll
        for (int r = 0; r < R; ++r) {
          if (!unit && i == j) vq[r] *= rq;
          const double xj = __shfl_sync(0xffffffffu, vq[r], j & 31);
          if (mine && (fwd ? i > j : i < j)) vq[r] = fma(-a, xj, vq[r]);
        }
      }
#pragma unroll
      for (int r = 0; r < R; ++r) {
        slot_set_r<R>(v, q0, r, vq[r]);
        if (mine) xck[r * kSolveChunk + (i - j0)] = vq[r];
      }
    }
    __syncthreads();
    // 2. the chunk applied to the rows still to be solved
#pragma unroll
    for (int s = 0; s < kSolveSlots; ++s) {
      const int i = s * kSolveThreads + tid;
      if (fwd ? (i >= j0 + w && i < d) : (i < j0)) {
#pragma unroll
        for (int r = 0; r < R; ++r) {
          double a = v[s][r];
          const double *xr = xck + r * kSolveChunk;
          if (w == kSolveChunk) {
#pragma unroll
            for (int t = 0; t < kSolveChunk; ++t) {
              const int jj = fwd ? t : kSolveChunk - 1 - t;
              a = fma(-opA(i, jj), xr[jj], a);
            }
          } else {
            for (int t = 0; t < w; ++t) {
              const int jj = fwd ? t : w - 1 - t;
              a = fma(-opA(i, jj), xr[jj], a);
            }
          }
          v[s][r] = a;
        }
      }
    }
    __syncthreads();                                   // buffer k & 1 is refilled at step k + 2
  }
  if (!trans) {
#pragma unroll
    for (int s = 0; s < kSolveSlots; ++s) {
      const int i = s * kSolveThreads + tid;
#pragma unroll
      for (int r = 0; r < R; ++r)
        if (i < d && r < nr) X[(int64_t)(c0 + r) * d + i] = v[s][r];
    }
  } else {
#pragma unroll
    for (int s = 0; s < kSolveSlots; ++s) {
      const int i = s * kSolveThreads + tid;
#pragma unroll
      for (int r = 0; r < R; ++r)
        if (i < d) xs[(size_t)r * d + i] = v[s][r];
    }
    __syncthreads();
    if (tid < R) {
      double *xr = xs + (size_t)tid * d;
      for (int j = d - 1; j >= 0; --j) {
        const int p = ps[j];
        if (p != j) { double t = xr[j]; xr[j] = xr[p]; xr[p] = t; }
      }
    }
    __syncthreads();
    for (int r = 0; r < nr; ++r)
      for (int i = tid; i < d; i += kSolveThreads) X[(int64_t)(c0 + r) * d + i] = xs[(size_t)r * d + i];
  }
}

static size_t lu_solve_smem(int d, int R) {
  return sizeof(double) * ((size_t)2 * kSolveLdT * d + (size_t)R * d + 2 * (size_t)R * kSolveChunk) +
         sizeof(int32_t) * (size_t)d;
}

// C (d x m) = op(A) (d x d) * Bm (d x m), FP64, ld = d.  transA: C = A^T B.
__global__ void k_gemm_small(int d, int m, const double *A, const double *Bm, double *C, int transA,
                             double alpha) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  int c = blockIdx.y;
  if (i >= d) return;
  double s = 0.0;
  for (int k = 0; k < d; ++k) {
    double a = transA ? A[k + (int64_t)i * d] : A[i + (int64_t)k * d];
    s = fma(a, Bm[k + (int64_t)c * d], s);
  }
  C[i + (int64_t)c * d] = alpha * s;
}

// C' = R^T + tau B  (and copies for the LUs)
__global__ void k_make_core(int d, const double *R, const double *B, double tau, double *Cp, double *luB,
                            double *luC) {
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < d * d; e += gridDim.x * blockDim.x) {
    int i = e % d, j = e / d;
    double c = R[j + (int64_t)i * d] + tau * B[e];
    Cp[e] = c;
    luC[e] = c;
    luB[e] = B[e];
  }
}

// X = (A - Q V) * inv_tau  (FP32 GEMM n x d x m; V is FP64 d x m, converted per tile).
__global__ void __launch_bounds__(256) k_apply_x(int64_t n, int d, int m, const float *__restrict__ Q,
                                                 int64_t ldq, const double *__restrict__ V,
                                                 const float *__restrict__ A, int64_t lda, float *X,
                                                 int64_t ldx, float inv_tau) {
  __shared__ __align__(16) float Vs[64][32];   // read as broadcast float4s
  const int tid = threadIdx.x;
  const int64_t i = (int64_t)blockIdx.x * 256 + tid;
  const int c0 = blockIdx.y * 32;
  const int mc = min(32, m - c0);
  float acc[32];
#pragma unroll
  for (int c = 0; c < 32; ++c) acc[c] = 0.f;
  for (int k0 = 0; k0 < d; k0 += 64) {
    __syncthreads();
    for (int e = tid; e < 64 * 32; e += 256) {
      int kk = e % 64, c = e / 64;
      Vs[kk][c] = (k0 + kk < d && c < mc) ? (float)V[(k0 + kk) + (int64_t)(c0 + c) * d] : 0.f;
    }
    __syncthreads();
    if (i < n) {
      const int kmax = min(64, d - k0);
      for (int kb = 0; kb < kmax; kb += 16) {     // sixteen loads of Q in flight per thread
        float q[16];
#pragma unroll
        for (int u = 0; u < 16; ++u) q[u] = (kb + u < kmax) ? Q[i + (int64_t)(k0 + kb + u) * ldq] : 0.f;
#pragma unroll
        for (int u = 0; u < 16; ++u) {
#pragma unroll
          for (int c4 = 0; c4 < 8; ++c4) {
            const float4 v = *reinterpret_cast<const float4 *>(&Vs[kb + u][4 * c4]);
            acc[4 * c4 + 0] = fmaf(q[u], v.x, acc[4 * c4 + 0]);
            acc[4 * c4 + 1] = fmaf(q[u], v.y, acc[4 * c4 + 1]);
            acc[4 * c4 + 2] = fmaf(q[u], v.z, acc[4 * c4 + 2]);
            acc[4 * c4 + 3] = fmaf(q[u], v.w, acc[4 * c4 + 3]);
          }
        }
      }
    }
  }
  if (i < n)
#pragma unroll
    for (int c = 0; c < 32; ++c)          // a compile-time bound keeps acc in registers
      if (c < mc) X[i + (int64_t)(c0 + c) * ldx] = (A[i + (int64_t)(c0 + c) * lda] - acc[c]) * inv_tau;
}

__global__ void k_add_inplace(int64_t n, int m, float *X, int64_t ldx, const float *D, int64_t ldd) {
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < n * m;
       e += (int64_t)gridDim.x * blockDim.x) {
    int64_t i = e % n, c = e / n;
    X[i + c * ldx] += D[i + c * ldd];
  }
}

int splits_for(const ckinv_ctx *ctx, int64_t n, int tiles) {
  int want = std::max(1, (ctx->sm_count * 3) / std::max(1, tiles));
  int64_t max_split = ceil_div(n, 256);
  return (int)std::max<int64_t>(1, std::min<int64_t>(want, max_split));
}

}  // namespace

// G = sum over s (in order) of part[s]: the row splits of a product folded deterministically.
__global__ void k_fold_splits(int64_t count, int splits, const double *part, double *G) {
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < count; e += (int64_t)gridDim.x * blockDim.x) {
    double acc = 0.0;
    for (int s = 0; s < splits; ++s) acc += part[(int64_t)s * count + e];
    G[e] = acc;
  }
}

static Error fold_splits(int64_t count, int splits, double *part, double *G, cudaStream_t st) {
  ::ckinv::note_launch(), k_fold_splits<<<(unsigned)std::min<int64_t>(ceil_div(count, 256), 2048), 256, 0, st>>>(
                              count, splits, part, G);
  CK_CUDA(cudaGetLastError());
  cudaFreeAsync(part, st);
  return ok();
}

Error tsprod(ckinv_ctx *ctx, int64_t n, int d1, int d2, const float *L, int64_t ldl, const uint32_t *bits,
             const int32_t *cols, double oscale, const float *M, int64_t ldm, double *G, cudaStream_t st,
             int64_t orow0) {
  const bool narrow = d2 <= 32;                 // 128 x 32 tiles: no lanes wasted on a thin M
  const int TMv = narrow ? 128 : 64, TNv = narrow ? 32 : 64;
  int tx = (int)ceil_div(d1, TMv), ty = (int)ceil_div(d2, TNv);
  int sp = splits_for(ctx, n, tx * ty);
  int64_t rps = ceil_div(ceil_div(n, sp), 256) * 256;
  sp = (int)ceil_div(n, rps);
  double *part = nullptr;
  CK_CUDA(dev_alloc((void **)&part, sizeof(double) * (size_t)sp * d1 * d2, st));
  dim3 grid(tx, ty, sp);
  ::ckinv::note_launch();
  if (narrow) {
    if (L) k_tsprod<false, 128, 32><<<grid, 256, 0, st>>>(n, d1, d2, L, ldl, bits, cols, oscale, M, ldm, part, rps, orow0);
    else k_tsprod<true, 128, 32><<<grid, 256, 0, st>>>(n, d1, d2, L, ldl, bits, cols, oscale, M, ldm, part, rps, orow0);
  } else {
    if (L) k_tsprod<false, 64, 64><<<grid, 256, 0, st>>>(n, d1, d2, L, ldl, bits, cols, oscale, M, ldm, part, rps, orow0);
    else k_tsprod<true, 64, 64><<<grid, 256, 0, st>>>(n, d1, d2, L, ldl, bits, cols, oscale, M, ldm, part, rps, orow0);
  }
  CK_CUDA(cudaGetLastError());
  return fold_splits((int64_t)d1 * d2, sp, part, G, st);
}

static Error tsprod_dd(ckinv_ctx *ctx, int64_t n, int d1, int d2, const float *L, int64_t ldl, const float *M,
                       int64_t ldm, double *G, cudaStream_t st) {
  int tx = (int)ceil_div(d1, 64), ty = (int)ceil_div(d2, 32);
  int sp = splits_for(ctx, n, tx * ty);
  int64_t rps = ceil_div(ceil_div(n, sp), 256) * 256;
  sp = (int)ceil_div(n, rps);
  double *part = nullptr;
  CK_CUDA(dev_alloc((void **)&part, sizeof(double) * (size_t)sp * d1 * d2, st));
  dim3 grid(tx, ty, sp);
  ::ckinv::note_launch(), k_tsprod_dd<<<grid, 256, 0, st>>>(n, d1, d2, L, ldl, M, ldm, part, rps);
  CK_CUDA(cudaGetLastError());
  return fold_splits((int64_t)d1 * d2, sp, part, G, st);
}

// Blocked LU of nmat strided d x d matrices: panel (one CTA per matrix), TRSM, GEMM update.
static Error lu_blocked(ckinv_ctx *ctx, int nmat, int d, double *A, int32_t *piv, double *logabs, cudaStream_t st) {
  constexpr int NBL = 32;
  CK_CUDA(cudaMemsetAsync(logabs, 0, sizeof(double) * nmat, st));
  const int64_t sA = (int64_t)d * d;
  const size_t smem_max = sizeof(double) * (size_t)d * NBL;
  CK_CUDA(cudaFuncSetAttribute(k_lu_panel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_max));
  for (int k0 = 0; k0 < d; k0 += NBL) {
    const int kb = std::min(NBL, d - k0);
    note_launch();
    k_lu_panel<<<nmat, kLuPanelThreads, sizeof(double) * (size_t)(d - k0) * kb, st>>>(d, k0, kb, A, piv, logabs,
                                                                                      ctx->d_err);
    CK_CUDA(cudaGetLastError());
    if (d > kb) {
      note_launch();
      k_lu_laswp<<<dim3((unsigned)ceil_div(d - kb, 128), nmat), 128, 0, st>>>(d, k0, kb, A, piv);
      CK_CUDA(cudaGetLastError());
    }
    const int rest = d - k0 - kb;
    if (rest <= 0) continue;
    note_launch();
    k_lu_trsm<<<dim3((unsigned)ceil_div(rest, kLuTrsmThreads), nmat), kLuTrsmThreads, 0, st>>>(d, k0, kb, A);
    CK_CUDA(cudaGetLastError());
    double *L21 = A + (k0 + kb) + (int64_t)k0 * d;
    double *U12 = A + k0 + (int64_t)(k0 + kb) * d;
    double *A22 = A + (k0 + kb) + (int64_t)(k0 + kb) * d;
    CK_TRY(gemm_batched<double>(ctx, false, rest, rest, kb, -1.0, L21, d, sA, U12, d, sA, 1.0, A22, d, sA, nmat, st));
  }
  return ok();
}

Error lu_factor_f64(ckinv_ctx *ctx, int n, double *A, int32_t *piv, double *logabsdet, cudaStream_t st) {
  return lu_blocked(ctx, 1, n, A, piv, logabsdet, st);
}

// Right-hand sides per block: one for a vector or a few columns (the latency of the
// substitution chain sets the time); four for a matrix of many columns, where one column per
// block would fill every SM with blocks that each stage the whole factor and keep the FP64
// units a quarter busy.  A column's operations are the same whatever the grouping.
static Error lu_solve(int d, int m, const double *LU, const int32_t *piv, double *X, int trans, cudaStream_t st) {
  if (d > kSolveThreads * kSolveSlots) return fail(CKINV_EUNSUPPORTED, "triangular solve: d above 512");
  if (m <= 0 || d <= 0) return ok();
  const int R = m >= 64 ? 4 : 1;
  const size_t smem = lu_solve_smem(d, R);
  if (R == 4) {
    CK_CUDA(cudaFuncSetAttribute(k_lu_solve<4>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)lu_solve_smem(kSolveThreads * kSolveSlots, 4)));
    ::ckinv::note_launch(),
        k_lu_solve<4><<<(unsigned)ceil_div(m, 4), kSolveThreads, smem, st>>>(d, m, LU, piv, X, trans);
  } else {
    CK_CUDA(cudaFuncSetAttribute(k_lu_solve<1>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)lu_solve_smem(kSolveThreads * kSolveSlots, 1)));
    ::ckinv::note_launch(), k_lu_solve<1><<<(unsigned)m, kSolveThreads, smem, st>>>(d, m, LU, piv, X, trans);
  }
  CK_CUDA(cudaGetLastError());
  return ok();
}

Error lu_solve_dev(int d, int m, const double *LU, const int32_t *piv, double *X, int trans, cudaStream_t st) {
  return lu_solve(d, m, LU, piv, X, trans, st);
}

Error gemm_small_dev(int d, int m, const double *A, const double *Bm, double *C, int transA, cudaStream_t st) {
  dim3 g((unsigned)ceil_div(d, 128), (unsigned)m);
  ::ckinv::note_launch(), k_gemm_small<<<g, 128, 0, st>>>(d, m, A, Bm, C, transA, 1.0);
  CK_CUDA(cudaGetLastError());
  return ok();
}

Error lowrank_core(ckinv_ctx *ctx, ckinv_factor *f, cudaStream_t st) {
  const int d = f->d;
  // B = Omega^T Q_hat  (B^T = Q_hat^T Omega: rows of A are the columns of Q_hat).  The BF16
  // and fast-transform forms apply the Walsh-Hadamard Omega as the fast transform over
  // Q_hat's d columns in FP32 (~6e-7 relative; for the BF16 form that replaces a three-term
  // tensor-core product at ~1e-5).  The FP32-level reference forms keep the compensated
  // contraction with Omega from its bits (FP64 across 256-row chunks): their FP64-leaf
  // likelihood is pinned tighter than FP32 sums of B allow.  A dense Omega: FP32 contraction.
  if (f->omega_dense)        // a dense Omega (Gaussian, Hartley, cosine): B = Omega^T Q_hat in FP32
    CK_TRY(tsprod(ctx, f->n, d, d, f->omega_dense, f->n, nullptr, nullptr, 0.0, f->Q, f->n, f->B, st));
  else if (omega_by_transform(f->prec, f->n, d))
    CK_TRY(omega_t_times_wht(ctx, f->n, d, f->Q, f->n, f->bits, f->cols, f->omega_scale, f->B, st));
  else if (f->n % 4 == 0 && f->prec == CKINV_BF16)
    CK_TRY(dense_tc(ctx, d, f->n, d, 3, f->Q, f->n, f->omega_scale, nullptr, 0, f->B, d, 1, st));
  else
    CK_TRY(tsprod(ctx, f->n, d, d, nullptr, 0, f->bits, f->cols, f->omega_scale, f->Q, f->n, f->B, st));
  return core_from_b(ctx, f, st);
}

Error core_from_b(ckinv_ctx *ctx, ckinv_factor *f, cudaStream_t st) {
  const int d = f->d;
  ::ckinv::note_launch(), k_make_core<<<64, 256, 0, st>>>(d, f->R, f->B, f->tau, f->Cp, f->luB, f->luC);
  CK_CUDA(cudaGetLastError());
  // luB and luC (and pivB, pivC) are adjacent: one strided batch of two LUs
  CK_TRY(lu_blocked(ctx, 2, d, f->luB, f->pivB, f->logdet_parts, st));
  return ok();
}

Error solve_from_z(ckinv_ctx *ctx, const ckinv_factor *f, const double *Z, const float *A, int64_t lda, int m,
                   float *X, int64_t ldx, cudaStream_t st) {
  (void)ctx;
  const int d = f->d;
  const int64_t n = f->n;
  double *W = nullptr;
  CK_CUDA(dev_alloc((void **)&W, sizeof(double) * d * m, st));
  struct Release {
    double *w;
    cudaStream_t st;
    ~Release() { cudaFreeAsync(w, st); }
  } release{W, st};
  dim3 g((unsigned)ceil_div(d, 128), (unsigned)m);
  if (f->two_pass) {
    ::ckinv::note_launch(), k_gemm_small<<<g, 128, 0, st>>>(d, m, f->S2, Z, W, 0, 1.0);
    CK_CUDA(cudaGetLastError());
    CK_TRY(lu_solve(d, m, f->S2 + (size_t)d * d, f->pivS, W, 0, st));
  } else {
    ::ckinv::note_launch(), k_gemm_small<<<g, 128, 0, st>>>(d, m, f->R, Z, W, 1, 1.0);
    CK_CUDA(cudaGetLastError());
    CK_TRY(lu_solve(d, m, f->luC, f->pivC, W, 0, st));
  }
  dim3 gx((unsigned)ceil_div(n, 256), (unsigned)ceil_div(m, 32));
  ::ckinv::note_launch(), k_apply_x<<<gx, 256, 0, st>>>(n, d, m, f->Q, n, W, A, lda, X, ldx, (float)(1.0 / f->tau));
  CK_CUDA(cudaGetLastError());
  return ok();
}

// X = K_tilde^-1 A, then refine_steps steps of refinement.
Error lowrank_solve(ckinv_ctx *ctx, const ckinv_factor *f, const float *A, int64_t lda, int m, float *X,
                    int64_t ldx, int refine_steps, cudaStream_t st) {
  const int d = f->d;
  const int64_t n = f->n;
  double *Z = nullptr, *W = nullptr;
  float *Acopy = nullptr, *Rs = nullptr, *Dx = nullptr;
  // the workspaces go back to the pool on every path out of this function, errors included
  struct Release {
    std::vector<void *> p;
    cudaStream_t st;
    ~Release() {
      for (void *q : p)
        if (q) cudaFreeAsync(q, st);
    }
  } release{{}, st};
  auto keep = [&](void *q) { release.p.push_back(q); };
  CK_CUDA(dev_alloc((void **)&Z, sizeof(double) * d * m, st));
  keep(Z);
  CK_CUDA(dev_alloc((void **)&W, sizeof(double) * d * m, st));
  keep(W);
  const float *Ain = A;
  if (refine_steps > 0 || X == A) {
    // keep A: X may alias it and the refinement needs it
    CK_CUDA(dev_alloc((void **)&Acopy, sizeof(float) * n * m, st));
    keep(Acopy);
    CK_CUDA(cudaMemcpy2DAsync(Acopy, sizeof(float) * n, A, sizeof(float) * lda, sizeof(float) * n, m,
                              cudaMemcpyDeviceToDevice, st));
    Ain = Acopy;
    lda = n;
  }
  // single-pass core: K_tilde = tau I + Q_hat B^-1 R^T Q_hat^T, solved through C' = R^T + tau B;
  // two-pass core: K_tilde = tau I + Q_hat S Q_hat^T, solved through S + tau I
  const double *S2 = f->two_pass ? f->S2 : nullptr;
  const double *luS = f->two_pass ? f->S2 + (size_t)d * d : nullptr;
  auto solve_into = [&](const float *rhs, int64_t ldr, float *out, int64_t ldo) -> Error {
    CK_TRY(tsprod(ctx, n, d, m, f->Q, n, nullptr, nullptr, 0.0, rhs, ldr, Z, st));     // Z = Q^T rhs
    dim3 g((unsigned)ceil_div(d, 128), (unsigned)m);
    if (S2) {
      ::ckinv::note_launch(), k_gemm_small<<<g, 128, 0, st>>>(d, m, S2, Z, W, 0, 1.0);                          // W = S Z
      CK_CUDA(cudaGetLastError());
      CK_TRY(lu_solve(d, m, luS, f->pivS, W, 0, st));                                   // W = (S + tau I)^-1 W
    } else {
      ::ckinv::note_launch(), k_gemm_small<<<g, 128, 0, st>>>(d, m, f->R, Z, W, 1, 1.0);                         // W = R^T Z
      CK_CUDA(cudaGetLastError());
      CK_TRY(lu_solve(d, m, f->luC, f->pivC, W, 0, st));                                 // W = C'^-1 W
    }
    dim3 gx((unsigned)ceil_div(n, 256), (unsigned)ceil_div(m, 32));
    ::ckinv::note_launch(), k_apply_x<<<gx, 256, 0, st>>>(n, d, m, f->Q, n, W, rhs, ldr, out, ldo, (float)(1.0 / f->tau));
    CK_CUDA(cudaGetLastError());
    return ok();
  };
  CK_TRY(solve_into(Ain, lda, X, ldx));
  if (refine_steps > 0) {
    CK_CUDA(dev_alloc((void **)&Rs, sizeof(float) * n * m, st));
    keep(Rs);
    CK_CUDA(dev_alloc((void **)&Dx, sizeof(float) * n * m, st));
    keep(Dx);
    for (int s = 0; s < refine_steps; ++s) {
      // W = B^-1 R^T Q^T X (single-pass) or S Q^T X (two-pass), FP64
      CK_TRY(tsprod_dd(ctx, n, d, m, f->Q, n, X, ldx, Z, st));
      dim3 g((unsigned)ceil_div(d, 128), (unsigned)m);
      if (S2) {
        ::ckinv::note_launch(), k_gemm_small<<<g, 128, 0, st>>>(d, m, S2, Z, W, 0, 1.0);
        CK_CUDA(cudaGetLastError());
      } else {
        ::ckinv::note_launch(), k_gemm_small<<<g, 128, 0, st>>>(d, m, f->R, Z, W, 1, 1.0);
        CK_CUDA(cudaGetLastError());
        CK_TRY(lu_solve(d, m, f->luB, f->pivB, W, 0, st));
      }
      dim3 gx((unsigned)ceil_div(n, 256), (unsigned)ceil_div(m, 16));
      ::ckinv::note_launch(), k_residual_dd<<<gx, 256, 0, st>>>(n, d, m, f->Q, n, W, Ain, lda, X, ldx, f->tau, Rs, n);
      CK_CUDA(cudaGetLastError());
      CK_TRY(solve_into(Rs, n, Dx, n));
      ::ckinv::note_launch(), k_add_inplace<<<(unsigned)std::min<int64_t>(ceil_div(n * m, 256), 65535), 256, 0, st>>>(n, m, X, ldx, Dx, n);
      CK_CUDA(cudaGetLastError());
    }
  }
  return ok();
}

}  // namespace ckinv
