// Sketch Y = K0 Omega through the fast Walsh-Hadamard transform (Definition 1's T applied as
// a transform, the cost the paper claims for the structured Omega, Sec. 1 and 3.2), in FP32
// on the CUDA cores.
//
// With N = 2^L and B = 1024 = 2^10, an index splits as k = k_a B + k_b and a column as
// p = p_a B + p_b, and H_N[k, p] = (-1)^popcount(k_a & p_a) (-1)^popcount(k_b & p_b).  So for
// a row i of K0 R (the kernel row with the Rademacher signs folded in)
//   Y[i, j] = c sum_{k_a} (-1)^popcount(k_a & p_a(j)) U_{k_a}[i, p_b(j)],
//   U_{k_a}[i, .] = H_B (K0 R)[i, k_a B : k_a B + B],
// a length-B Walsh-Hadamard transform of each 1024-point chunk of the row, then a signed gather
// of the d outputs.  Work per kernel entry: its evaluation, log2 B = 10 additions of the
// transform and d / B gathered additions, all in FP32 with round-to-nearest (the transform's
// sums are pairwise), against 2d MMA FLOP for the dense product.
//
// One warp transforms one row's chunk: lane l holds the 32 entries k_b = l + 32 t (t < 32) in
// registers; the five stages over t run in registers, the chunk is transposed through shared
// memory (padded rows of 33), and the five stages over the lane bits run in registers again,
// leaving U[q] in lane q / 32, register q % 32; it goes back to shared memory for the gather.
// Lane l owns the outputs j = l + 32 u of its warp's rows and accumulates them in registers
// over the chunks.  A CTA of 8 warps owns 32 rows (4 per warp) and streams the points of every
// chunk through shared memory, the next chunk's fetched into registers while the current one
// is transformed.
#include "internal.cuh"

namespace ckinv {
namespace {

constexpr int kWB = 1024;             // transform length (chunk of points)
constexpr int kWWarps = 8;
constexpr int kWThreads = 32 * kWWarps;
constexpr int kWRowsPerWarp = 4;
constexpr int kWRows = kWWarps * kWRowsPerWarp;   // rows per CTA
constexpr int kWMaxU = 16;            // outputs per lane: d <= 512

// In-register Walsh-Hadamard transform of 32 values along the register index.
__device__ __forceinline__ void wht32(float (&v)[32]) {
#pragma unroll
  for (int h = 1; h < 32; h <<= 1) {
#pragma unroll
    for (int t = 0; t < 32; ++t) {
      if ((t & h) == 0) {
        const float a = v[t], b = v[t + h];
        v[t] = a + b;
        v[t + h] = a - b;
      }
    }
  }
}

// Shared memory of one CTA (about 61 KB: dynamic, above the 48 KB of static declarations).
struct WhtSmem {
  float sp[2][kWB * 3];              // the chunk's points (pre-scaled), two buffers
  uint32_t ssg[2][kWB / 32];         // the chunk's sign words
  float buf[kWWarps][32 * 33];       // per-warp transpose / gather buffer
  int sq[32 * kWMaxU];               // output j: address of U[p_b(j)] in buf
  int spa[32 * kWMaxU];              // output j: p_a(j) = p_j / B
};

template <bool DERIV, int KIND>
__global__ void __launch_bounds__(kWThreads, 1)
    k_sketch_wht(int64_t n, int64_t row0, int64_t m, int dim, int d, int nchunks, KernelParams kp,
                 const float *__restrict__ pts, const uint32_t *__restrict__ bits, const int32_t *__restrict__ cols,
                 float *__restrict__ Y, int64_t ldy) {
  extern __shared__ __align__(16) unsigned char wht_smem[];
  WhtSmem &S = *reinterpret_cast<WhtSmem *>(wht_smem);
  auto &sp = S.sp;
  auto &ssg = S.ssg;
  auto &buf = S.buf;
  int *sq = S.sq, *spa = S.spa;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const float cs = kp.coord_scale, inv_l = kp.inv_l;
  const int nu = (d + 31) / 32;
  // lane l owns the outputs j = l + 32 u: where U[p_b(j)] lies in the padded buffer, and p_a(j)
  for (int j = threadIdx.x; j < 32 * kWMaxU; j += kWThreads) {
    const int p = j < d ? cols[j] : 0;
    const int q = p & (kWB - 1);
    sq[j] = (q >> 5) * 33 + (q & 31);
    spa[j] = p >> 10;
  }
  // this warp's rows
  const int64_t rbase = (int64_t)blockIdx.x * kWRows + warp * kWRowsPerWarp;
  float xr[kWRowsPerWarp][3];
#pragma unroll
  for (int r = 0; r < kWRowsPerWarp; ++r) {
    const int64_t i = min(rbase + r, m - 1);
#pragma unroll
    for (int c = 0; c < 3; ++c) xr[r][c] = c < dim ? pts[(row0 + i) * dim + c] * cs : 0.f;
  }
  float acc[kWRowsPerWarp][kWMaxU];
#pragma unroll
  for (int r = 0; r < kWRowsPerWarp; ++r)
#pragma unroll
    for (int u = 0; u < kWMaxU; ++u) acc[r][u] = 0.f;

  // chunk staging: each thread fetches up to 12 coordinates and one sign word
  constexpr int kPerThread = (kWB * 3 + kWThreads - 1) / kWThreads;
  float pf[kPerThread];
  uint32_t sf = 0;
  auto fetch = [&](int ka) {
    const int64_t k0 = (int64_t)ka * kWB;
    const int64_t lim = (n - k0) * dim;                // coordinates of this chunk inside [0, n)
#pragma unroll
    for (int q = 0; q < kPerThread; ++q) {
      const int e = threadIdx.x + q * kWThreads;
      pf[q] = (e < kWB * dim && e < lim) ? pts[k0 * dim + e] * cs : 0.f;
    }
    const int64_t w = k0 / 32 + threadIdx.x;
    sf = (threadIdx.x < kWB / 32 && w * 32 < n) ? bits[w] : 0u;
  };
  auto stash = [&](int b) {
#pragma unroll
    for (int q = 0; q < kPerThread; ++q) {
      const int e = threadIdx.x + q * kWThreads;
      if (e < kWB * dim) sp[b][e] = pf[q];
    }
    if (threadIdx.x < kWB / 32) ssg[b][threadIdx.x] = sf;
  };
  fetch(0);
  stash(0);
  __syncthreads();
  float *wb = buf[warp];
  for (int ka = 0; ka < nchunks; ++ka) {
    const int b = ka & 1;
    if (ka + 1 < nchunks) fetch(ka + 1);
    const int64_t k0 = (int64_t)ka * kWB;
    // the signs of this lane's 32 entries (k_b = lane + 32 t) as one mask; entries at or past
    // n are zero (the padding of K0 to order N)
    uint32_t smask = 0, vmask = 0;
#pragma unroll
    for (int t = 0; t < 32; ++t) {
      smask |= ((ssg[b][t] >> lane) & 1u) << t;
      vmask |= (k0 + lane + 32 * t < n ? 1u : 0u) << t;
    }
    // the signs H_B-independent part: (-1)^popcount(k_a & p_a(j)) for this lane's outputs
    uint32_t gsg = 0;
#pragma unroll
    for (int u = 0; u < kWMaxU; ++u) gsg |= (uint32_t)(__popc(ka & spa[lane + 32 * u]) & 1) << u;
#pragma unroll
    for (int r = 0; r < kWRowsPerWarp; ++r) {
      float v[32];
      const float *P = sp[b];
#pragma unroll
      for (int t = 0; t < 32; ++t) {
        const int kb = lane + 32 * t;
        float r2;
        if (dim == 2) {
          const float2 q2 = reinterpret_cast<const float2 *>(P)[kb];     // conflict-free 8-byte reads
          const float dx = xr[r][0] - q2.x, dy = xr[r][1] - q2.y;
          r2 = fmaf(dy, dy, dx * dx);
        } else {
          const float dx = xr[r][0] - P[dim * kb];
          const float dy = dim > 1 ? xr[r][1] - P[dim * kb + 1] : 0.f;
          const float dz = dim > 2 ? xr[r][2] - P[dim * kb + 2] : 0.f;
          r2 = fmaf(dz, dz, fmaf(dy, dy, dx * dx));
        }
        float e = dev::kernel_value(KIND, r2, inv_l, DERIV);
        e = ((vmask >> t) & 1u) ? e : 0.f;
        v[t] = __uint_as_float(__float_as_uint(e) ^ (((smask >> t) & 1u) << 31));
      }
      wht32(v);                                       // bits 5..9 of k_b
      __syncwarp();
#pragma unroll
      for (int t = 0; t < 32; ++t) wb[t * 33 + lane] = v[t];
      __syncwarp();
#pragma unroll
      for (int t = 0; t < 32; ++t) v[t] = wb[lane * 33 + t];
      wht32(v);                                       // bits 0..4 of k_b
      __syncwarp();
#pragma unroll
      for (int t = 0; t < 32; ++t) wb[lane * 33 + t] = v[t];   // U[32 lane + t]
      __syncwarp();
#pragma unroll
      for (int u = 0; u < kWMaxU; ++u) {
        if (u < nu) {
          const float g = wb[sq[lane + 32 * u]];
          acc[r][u] += ((gsg >> u) & 1u) ? -g : g;
        }
      }
    }
    if (ka + 1 < nchunks) {
      stash(b ^ 1);
    }
    __syncthreads();
  }
  // Y = scale * acc (column-major): lane l writes its columns of the warp's rows
  const float scale = (float)kp.scale;
#pragma unroll
  for (int r = 0; r < kWRowsPerWarp; ++r) {
    const int64_t i = rbase + r;
    if (i >= m) continue;
#pragma unroll
    for (int u = 0; u < kWMaxU; ++u) {
      const int j = lane + 32 * u;
      if (u < nu && j < d) Y[i + (int64_t)j * ldy] = acc[r][u] * scale;
    }
  }
}

template <bool DERIV>
Error launch_wht(int kind, dim3 grid, int64_t n, int64_t row0, int64_t m, int dim, int d, int nchunks,
                 const KernelParams &kp, const float *pts, const uint32_t *bits, const int32_t *cols, float *Y,
                 int64_t ldy, cudaStream_t st) {
  auto kfn = kind == CKINV_SE ? k_sketch_wht<DERIV, CKINV_SE> : k_sketch_wht<DERIV, CKINV_MATERN52>;
  constexpr size_t smem = sizeof(WhtSmem);
  CK_CUDA(cudaFuncSetAttribute(kfn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  note_launch();
  kfn<<<grid, kWThreads, smem, st>>>(n, row0, m, dim, d, nchunks, kp, pts, bits, cols, Y, ldy);
  CK_CUDA(cudaGetLastError());
  return ok();
}

}  // namespace

bool sketch_wht_supported(int64_t n, int d) { return padded_order(n) >= kWB && d <= 32 * kWMaxU; }

Error sketch_wht(ckinv_ctx *ctx, int64_t n, int dim, int d, const KernelParams &kp, const float *points, bool deriv,
                 float *Y, int64_t ldy, cudaStream_t st, int64_t row0, int64_t m) {
  if (m < 0) m = n;
  if (!sketch_wht_supported(n, d)) return fail(CKINV_EUNSUPPORTED, "structured sketch: needs N >= 1024, d <= 512");
  const int nchunks = (int)(padded_order(n) / kWB);
  // chunks wholly past n hold only padding: their entries are zero
  const int live = (int)ceil_div(n, kWB);
  const dim3 grid((unsigned)ceil_div(m, kWRows));
  if (deriv)
    return launch_wht<true>(kp.kind, grid, n, row0, m, dim, d, std::min(nchunks, live), kp, points, ctx->om.bits,
                            ctx->om.cols, Y, ldy, st);
  return launch_wht<false>(kp.kind, grid, n, row0, m, dim, d, std::min(nchunks, live), kp, points, ctx->om.bits,
                           ctx->om.cols, Y, ldy, st);
}

}  // namespace ckinv
