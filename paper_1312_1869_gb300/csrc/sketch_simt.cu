// Sketch Y = K0 Omega (Sec. 3.1-3.3), FP32 form, on the CUDA cores.
//
// This form contracts the FP32-rounded kernel matrix exactly: every kernel entry is
// evaluated in FP64 from the FP32 points and rounded once to FP32 (so the contraction sees
// the correctly rounded K0), the +-1 Omega entries make every product exact, and the sums
// over the n points use compensated (Kahan) FP32 accumulation.  Y therefore carries about
// one FP32 rounding.  Kernel entries are materialised one block of rows at a time in a
// workspace, so each is evaluated once; a materialised K (CKINV_DENSE) is contracted
// directly.
#include "internal.cuh"

namespace ckinv {
namespace {

constexpr int BM = 64, BN = 64, BK = 32;

__device__ __forceinline__ double rho64(int kind, double r2, double ell, bool deriv) {
  if (kind == CKINV_SE) {
    double q = r2 / (ell * ell);
    double e = exp(-0.5 * q);
    return deriv ? e * q : e;
  }
  double u = 2.2360679774997896964 * sqrt(r2) / ell;
  double e = exp(-u);
  return deriv ? (u * u / 3.0) * (1.0 + u) * e : (1.0 + u + u * u / 3.0) * e;
}

// Kb[i + k * ldb] = fl32(var * rho(x_{r0+i}, x_k)) for i < rows, k < n.
template <bool DERIV>
__global__ void k_kmat_f64(int64_t rows, int64_t r0, int64_t n, int dim, int kind, double ell, double var,
                           const float *__restrict__ pts, float *__restrict__ Kb, int64_t ldb) {
  const int64_t total = rows * n;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total;
       e += (int64_t)gridDim.x * blockDim.x) {
    int64_t i = e % rows, k = e / rows;
    const float *xi = pts + (r0 + i) * dim;
    const float *xk = pts + k * dim;
    double r2 = 0.0;
    for (int t = 0; t < dim; ++t) {
      double df = (double)xi[t] - (double)xk[t];
      r2 = fma(df, df, r2);
    }
    Kb[i + k * ldb] = (float)(var * rho64(kind, r2, ell, DERIV));
  }
}

// Y[0:rows, 0:d] = scale * K[0:rows, 0:kn] Omega[0:kn, 0:d]; Kahan-compensated sums.
__global__ void __launch_bounds__(256) k_contract(int64_t rows, int64_t kn, int d, const float *__restrict__ K,
                                                  int64_t ldk, const uint32_t *__restrict__ bits,
                                                  const int32_t *__restrict__ cols, double scale,
                                                  float *__restrict__ Y, int64_t ldy) {
  __shared__ float As[BK][BM + 4];
  __shared__ float Bs[BK][BN + 4];
  __shared__ uint32_t pc[BN];
  const int tid = threadIdx.x;
  const int tx = tid % 16, ty = tid / 16;
  const int64_t i0 = (int64_t)blockIdx.x * BM;
  const int j0 = blockIdx.y * BN;
  for (int c = tid; c < BN; c += 256) pc[c] = (j0 + c < d) ? (uint32_t)cols[j0 + c] : 0u;
  float acc[4][4], cmp[4][4];
#pragma unroll
  for (int a = 0; a < 4; ++a)
#pragma unroll
    for (int b = 0; b < 4; ++b) { acc[a][b] = 0.0f; cmp[a][b] = 0.0f; }
  __syncthreads();
  for (int64_t k0 = 0; k0 < kn; k0 += BK) {
#pragma unroll
    for (int q = 0; q < (BK * BM) / 256; ++q) {
      int e = tid + 256 * q;
      int kk = e / BM, r = e % BM;
      int64_t k = k0 + kk, i = i0 + r;
      As[kk][r] = (k < kn && i < rows) ? K[i + k * ldk] : 0.0f;
    }
#pragma unroll
    for (int q = 0; q < (BK * BN) / 256; ++q) {
      int e = tid + 256 * q;
      int kk = e / BN, c = e % BN;
      int64_t k = k0 + kk;
      float v = 0.0f;
      if (k < kn && j0 + c < d) {
        uint32_t s = (bits[k >> 5] >> (k & 31)) & 1u;
        s ^= (uint32_t)(__popcll((unsigned long long)k & (unsigned long long)pc[c]) & 1);
        v = s ? -1.0f : 1.0f;
      }
      Bs[kk][c] = v;
    }
    __syncthreads();
#pragma unroll 4
    for (int kk = 0; kk < BK; ++kk) {
      float a[4], b[4];
#pragma unroll
      for (int t = 0; t < 4; ++t) {
        a[t] = As[kk][ty * 4 + t];
        b[t] = Bs[kk][tx * 4 + t];
      }
#pragma unroll
      for (int x = 0; x < 4; ++x)
#pragma unroll
        for (int y = 0; y < 4; ++y) {
          float term = a[x] * b[y] - cmp[x][y];   // a * (+-1) is exact
          float t = acc[x][y] + term;
          cmp[x][y] = (t - acc[x][y]) - term;
          acc[x][y] = t;
        }
    }
    __syncthreads();
  }
#pragma unroll
  for (int x = 0; x < 4; ++x) {
    int64_t i = i0 + ty * 4 + x;
    if (i >= rows) continue;
#pragma unroll
    for (int y = 0; y < 4; ++y) {
      int j = j0 + tx * 4 + y;
      if (j < d) Y[i + (int64_t)j * ldy] = (float)((double)acc[x][y] * scale);
    }
  }
}

}  // namespace

Error sketch_simt(ckinv_ctx *ctx, int64_t n, int dim, int d, const KernelParams &kp, const float *points,
                  const float *K, int64_t ldk, bool deriv, float *Y, int64_t ldy, cudaStream_t st, int64_t row0,
                  int64_t m) {
  const uint32_t *bits = ctx->om.bits;
  const int32_t *cols = ctx->om.cols;
  const double c = 1.0 / std::sqrt((double)padded_order(n));
  if (m < 0) m = n;
  if (K) {
    dim3 grid((unsigned)ceil_div(m, BM), (unsigned)ceil_div(d, BN));
    ::ckinv::note_launch(), k_contract<<<grid, 256, 0, st>>>(m, n, d, K + row0, ldk, bits, cols, c, Y, ldy);
    CK_CUDA(cudaGetLastError());
    return ok();
  }
  // row blocks of the kernel matrix, evaluated once each (about 2 GB of workspace at most)
  int64_t R = std::max<int64_t>(BM, ((int64_t)1 << 29) / std::max<int64_t>(n, 1));
  R = std::min<int64_t>(R, m);
  R = ceil_div(R, BM) * BM;
  float *Kb = nullptr;
  CK_CUDA(dev_alloc((void **)&Kb, sizeof(float) * R * n, st));
  const double ell = kp.ell, var = kp.var;
  for (int64_t r0 = row0; r0 < row0 + m; r0 += R) {
    int64_t rows = std::min<int64_t>(R, row0 + m - r0);
    unsigned g = (unsigned)std::min<int64_t>(ceil_div(rows * n, 256), (int64_t)ctx->sm_count * 32);
    if (deriv)
      ::ckinv::note_launch(), k_kmat_f64<true><<<g, 256, 0, st>>>(rows, r0, n, dim, kp.kind, ell, var, points, Kb, rows);
    else
      ::ckinv::note_launch(), k_kmat_f64<false><<<g, 256, 0, st>>>(rows, r0, n, dim, kp.kind, ell, var, points, Kb, rows);
    dim3 grid((unsigned)ceil_div(rows, BM), (unsigned)ceil_div(d, BN));
    ::ckinv::note_launch(), k_contract<<<grid, 256, 0, st>>>(rows, n, d, Kb, rows, bits, cols, c, Y + (r0 - row0), ldy);
    CK_CUDA(cudaGetLastError());
  }
  CK_CUDA(cudaFreeAsync(Kb, st));
  return ok();
}

Error kernel_matrix(ckinv_ctx *ctx, int64_t n, int dim, const KernelParams &kp, const float *points, float *K,
                    int64_t ldk, cudaStream_t st) {
  const unsigned g = (unsigned)std::min<int64_t>(ceil_div(n * n, 256), (int64_t)ctx->sm_count * 64);
  note_launch();
  k_kmat_f64<false><<<g, 256, 0, st>>>(n, 0, n, dim, kp.kind, kp.ell, kp.var, points, K, ldk);
  CK_CUDA(cudaGetLastError());
  return ok();
}

}  // namespace ckinv
