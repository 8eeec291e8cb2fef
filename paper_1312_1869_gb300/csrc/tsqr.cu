// Blocked tall-skinny QR of Y (Sec. 3.3, Eqs. 1-4) and the explicit Q_hat.
//
// The TSQR is a sequence of stages, each a batch of independent dense QRs of the same
// shape H x d: the leaves (blocks of b rows of Y, Eq. 1) and then, level by level, the
// combines of stacked pairs of R factors [R_a; R_b] (2d x d, Eqs. 2-3).  Pairs are formed
// left to right at every level and an odd last node passes up unchanged.  A leaf QR is
// Householder QR in recursive blocked form (Elmroth & Gustavson): column ranges are split
// in two down to 16-column panels, which one CTA per problem factors in shared memory with
// warp-shuffle reductions; everything else - applying the left part's reflectors to the
// right part and assembling the compact-WY factor T (Q = I - V T V^T) - is batched GEMM.
// A combine exploits the stacked-triangle structure and runs panel by panel, one launch per
// panel for all combines of a level (k_sq_step, below).
// Leaves run in FP32 (or FP64 on request), the top `fp64_levels` tree levels in FP64; the
// R factors passed between levels are FP64 throughout.  Q_hat is formed top-down from the
// root's coefficient block D = sign(diag R): each stage maps its blocks X to
// Q [X; 0] = [X; 0] - V (T (V_top^T X)), three batched GEMMs, in the leaves' precision (FP64
// tree levels hand FP32 copies of their reflectors to an FP32 Q_hat: the combine is where
// FP64 buys accuracy, and an FP64 product on this part costs ~60x an FP32 one).
#include "internal.cuh"
#include "dfloat.cuh"

#include <type_traits>

namespace ckinv {
namespace {

constexpr int NB = 16;            // panel width of the recursion's base case
constexpr int PF_THREADS = 512;   // panel-factor CTA
constexpr size_t kPanelSmemMax = 220 * 1024;

template <typename T>
size_t panel_smem(int h) {
  int hp = h | 1;
  return sizeof(T) * ((size_t)NB * hp + (PF_THREADS / 32) * NB + NB + NB + NB * NB + 4);
}

// Threads of a panel CTA: short panels and FP64 panels use fewer warps, because the
// cross-warp reductions dominate there (an FP64 warp instruction is slow on this part).
template <typename T>
int panel_threads(int h) {
  if (sizeof(T) == 8) return h > 1024 ? 256 : 128;
  return h > 1024 ? 512 : (h > 256 ? 256 : 128);
}

// Reduce NV per-thread values over the whole CTA; result in out[0..NV).  Within a warp the
// NV values are reduced by recursive halving (NV - 1 + 32 / NV shuffles instead of 5 NV):
// at offset o every lane keeps half of its values, adds its partner's copy of that half, and
// after the halvings lane l holds the warp sum of value kept(l) (lanes that share a value
// finish with plain butterflies).
template <typename T, int NV, int NT>
__device__ __forceinline__ void block_sum(T (&vals)[NV], T *red, T *out) {
  static_assert(NV >= 1 && NV <= 32 && (NV & (NV - 1)) == 0, "NV must be a power of two <= 32");
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  int idx = 0;                                   // index of the value this lane ends with
#pragma unroll
  for (int o = 16, n = NV; n > 1; o >>= 1, n >>= 1) {
    const bool up = (lane & o) != 0;             // keep the upper half of the n values
#pragma unroll
    for (int j = 0; j < n / 2; ++j) {
      const T send = up ? vals[j] : vals[j + n / 2];
      const T keep = up ? vals[j + n / 2] : vals[j];
      vals[j] = keep + __shfl_xor_sync(0xffffffffu, send, o);
    }
    idx = 2 * idx + (up ? 1 : 0);
  }
  constexpr int kFirst = 32 / NV;                // lanes still sharing one value
  T x = vals[0];
#pragma unroll
  for (int o = kFirst / 2; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
  if ((lane & (kFirst - 1)) == 0) red[warp * NV + idx] = x;
  __syncthreads();
  if (threadIdx.x < NV) {
    T s = 0;
    for (int w = 0; w < NT / 32; ++w) s += red[w * NV + threadIdx.x];
    out[threadIdx.x] = s;
  }
  __syncthreads();
}

// Householder QR of the panel M[c0:H, c0:c0+NB] of problem blockIdx.x (M: H x d, ld H).
// Writes R and the reflectors into M, the explicit reflectors (unit diagonal, zeros above)
// into Vx[:, c0:c0+NB], and the panel's compact-WY block into Tm[c0:c0+NB, c0:c0+NB].
// Stacked mode (a combine, H = 2d, M = [R_a; R_b] with both upper triangular): the
// structurally nonzero rows of the panel are the top rows c0..c0+NB-1 and the bottom rows
// 0..c0+NB-1 (physical rows d..d+c0+NB-1); only those are loaded and factored.
template <typename T>
__device__ __forceinline__ int panel_row(bool stacked, int c0, int d, int r) {
  return stacked ? (r < NB ? c0 + r : d + r - NB) : c0 + r;
}

// Shared-memory staging of a column-major global tile, U loads in flight per thread (a
// load-store loop would wait out one memory latency per element):
//   dst[i * ldd + c * cstride] = c < cvalid ? src[i + c * lds] : 0,  i < rows, c < cols.
template <typename T, int U>
__device__ __forceinline__ void stage_tile(T *dst, int ldd, int cstride, const T *src, int64_t lds, int rows,
                                           int cols, int cvalid) {
  const int total = rows * cols;
  for (int base = 0; base < total; base += (int)blockDim.x * U) {
    T v[U];
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const int e = base + u * (int)blockDim.x + (int)threadIdx.x;
      const int i = e % rows, c = e / rows;
      v[u] = (e < total && c < cvalid) ? src[i + (int64_t)c * lds] : T(0);
    }
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const int e = base + u * (int)blockDim.x + (int)threadIdx.x;
      if (e < total) dst[(e % rows) * ldd + (e / rows) * cstride] = v[u];
    }
  }
}

template <typename T, int PT>
__global__ void __launch_bounds__(PT) k_panel(T *M, T *Vx, T *Tm, int H, int d, int c0, int stacked) {
  extern __shared__ __align__(16) uint8_t sm_raw[];
  const int64_t pslot = (int64_t)H * d;
  M += blockIdx.x * pslot;
  Vx += blockIdx.x * pslot;
  Tm += (int64_t)blockIdx.x * d * d;
  const int h = stacked ? c0 + 2 * NB : H - c0;
  const int hp = h | 1;
  T *Ps = reinterpret_cast<T *>(sm_raw);                  // NB x hp
  T *red = Ps + NB * hp;                                  // 16 warps x NB
  T *sums = red + (PT / 32) * NB;                 // NB
  T *wv = sums + NB;                                      // NB
  T *Ts = wv + NB;                                        // NB x NB
  T *scal = Ts + NB * NB;                                 // [tau, rdiag, head]
  const int tid = threadIdx.x;
  T *base = M + (int64_t)c0 * H;                          // column c0

  if (!stacked) {
    stage_tile<T, 8>(Ps, 1, hp, base + c0, H, h, NB, NB);
  } else {
    for (int c = 0; c < NB; ++c)
      for (int r = tid; r < h; r += PT)
        Ps[c * hp + r] = base[panel_row<T>(stacked, c0, d, r) + (int64_t)c * H];
  }
  for (int e = tid; e < NB * NB; e += PT) Ts[e] = 0;
  __syncthreads();

  for (int jj = 0; jj < NB; ++jj) {
    T *x = Ps + jj * hp;
    // one pass and one reduction per step: raw dots of x (rows below jj) with every panel
    // column, c == jj giving |x|^2; the reflector v = x / head is applied through them
    T dots[NB];
#pragma unroll
    for (int c = 0; c < NB; ++c) dots[c] = 0;
    for (int r = jj + 1 + tid; r < h; r += PT) {
      const T xr = x[r];
#pragma unroll
      for (int c = 0; c < NB; ++c) dots[c] += Ps[c * hp + r] * xr;
    }
    block_sum<T, NB, PT>(dots, red, sums);
    // every thread derives the reflector from the reduced norm (no broadcast round trip)
    // tau = 2 / (v^T v) from the same |x|^2 and 1 / head that form the stored reflector v,
    // so that tau and v agree to one rounding at the working precision
    const T alpha = x[jj];
    const T sig = sums[jj];
    const T normx = sqrt(alpha * alpha + sig);
    T tau = 0, rd = 0, inv_head = 0;
    if (normx > 0) {
      const T sg = alpha >= 0 ? T(1) : T(-1);
      const T head = alpha + sg * normx;
      inv_head = T(1) / head;
      tau = T(2) / (T(1) + sig * inv_head * inv_head);
      rd = -sg * normx;
    }
    for (int r = jj + 1 + tid; r < h; r += PT) x[r] *= inv_head;   // this thread's rows only
    if (tid < NB && tid != jj) wv[tid] = Ps[tid * hp + jj] + sums[tid] * inv_head;
    __syncthreads();
    if (tid == 0) x[jj] = rd;
    for (int c = jj + 1; c < NB; ++c) {
      T w = tau * wv[c];
      T *col = Ps + c * hp;
      for (int r = jj + 1 + tid; r < h; r += PT) col[r] -= w * x[r];
      if (tid == 0) col[jj] -= w;
    }
    if (tid < jj) {
      int i = tid;
      T acc = 0;
      for (int l = i; l < jj; ++l) acc += Ts[i * NB + l] * wv[l];
      Ts[i * NB + jj] = -tau * acc;
    }
    if (tid == 0) Ts[jj * NB + jj] = tau;
    __syncthreads();
  }
  for (int c = 0; c < NB; ++c) {
    T *vcol = Vx + (int64_t)(c0 + c) * H;
    for (int r = tid; r < H; r += PT) {
      int lr;                                   // logical panel row of physical row r, or -1
      if (stacked) lr = (r >= c0 && r < c0 + NB) ? r - c0 : ((r >= d && r < d + c0 + NB) ? r - d + NB : -1);
      else lr = r - c0;
      vcol[r] = (lr < 0 || lr < c) ? T(0) : (lr == c ? T(1) : Ps[c * hp + lr]);
    }
    for (int r = tid; r < h; r += PT) base[panel_row<T>(stacked, c0, d, r) + (int64_t)c * H] = Ps[c * hp + r];
  }
  for (int e = tid; e < NB * NB; e += PT) {
    int i = e / NB, j = e % NB;              // Ts is row-major [i][j]; Tm column-major
    Tm[(c0 + i) + (int64_t)(c0 + j) * d] = Ts[e];
  }
}

// Leaf blocks into the stage matrix (H x d per leaf), zero-padded: leaf p's rows start at
// src[p] (FP32, column-major, ld ld[p]; leaves of several problems may share a stage).
template <typename T>
__global__ void k_gather_leaves(const float *const *srcs, const int64_t *ld, const int *rows, int H, int d, T *M) {
  const int p = blockIdx.y;
  const float *Yp = srcs[p];
  const int64_t ldp = ld[p];
  const int h = rows[p];
  T *dst = M + (int64_t)p * H * d;
  for (int c = blockIdx.x; c < d; c += gridDim.x) {
    const float *src = Yp + (int64_t)c * ldp;
    T *out = dst + (int64_t)c * H;
    for (int r = threadIdx.x; r < H; r += blockDim.x) out[r] = (r < h) ? (T)src[r] : T(0);
  }
}

// Rslot[slot[p]] = upper triangle of M_p[0:d, 0:d] (FP64, zeros below).
template <typename T>
__global__ void k_extract_r(const T *M, int H, int d, const int *slot, double *Rslot) {
  const int p = blockIdx.y;
  const T *src = M + (int64_t)p * H * d;
  double *dst = Rslot + (int64_t)slot[p] * d * d;
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < d * d; e += gridDim.x * blockDim.x) {
    int r = e % d, c = e / d;
    dst[e] = (r <= c) ? (double)src[r + (int64_t)c * H] : 0.0;
  }
}

// S_p = [R_top; R_bot] (2d x d, ld 2d) from the FP64 slots.
template <typename T>
__global__ void k_build_stack(const double *Rslot, const int *top, const int *bot, int d, T *S) {
  const int p = blockIdx.y;
  const double *ra = Rslot + (int64_t)top[p] * d * d;
  const double *rb = Rslot + (int64_t)bot[p] * d * d;
  T *dst = S + (int64_t)p * 2 * d * d;
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < 2 * d * d; e += gridDim.x * blockDim.x) {
    int r = e % (2 * d), c = e / (2 * d);
    dst[e] = (T)((r < d) ? ra[r + (int64_t)c * d] : rb[(r - d) + (int64_t)c * d]);
  }
}

// R_out = D R_root, Xslot[0] = D, D = sign(diag R_root) (0 -> +1).
__global__ void k_finish_root(const double *Rroot, int d, double *Rout, double *Xroot) {
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < d * d; e += gridDim.x * blockDim.x) {
    int r = e % d, c = e / d;
    double s = (Rroot[r + (int64_t)r * d] < 0.0) ? -1.0 : 1.0;
    Rout[e] = (r <= c) ? s * Rroot[e] : 0.0;
    Xroot[e] = (r == c) ? s : 0.0;
  }
}

// Qs_p = [X_{top[p]}; 0] (H x d), X from the FP64 slots.
template <typename T>
__global__ void k_init_qs(const double *Xslot, const int *top, int H, int d, T *Qs) {
  const int p = blockIdx.y;
  const double *x = Xslot + (int64_t)top[p] * d * d;
  T *dst = Qs + (int64_t)p * H * d;
  for (int c = blockIdx.x; c < d; c += gridDim.x) {
    T *out = dst + (int64_t)c * H;
    for (int r = threadIdx.x; r < H; r += blockDim.x) out[r] = (r < d) ? (T)x[r + (int64_t)c * d] : T(0);
  }
}

// Xslot[top[p]] = Qs_p[0:d], Xslot[bot[p]] = Qs_p[d:2d]  (combine stages, H = 2d).
template <typename T>
__global__ void k_scatter_x(const T *Qs, const int *top, const int *bot, int d, double *Xslot) {
  const int p = blockIdx.y;
  const T *src = Qs + (int64_t)p * 2 * d * d;
  double *xa = Xslot + (int64_t)top[p] * d * d;
  double *xb = Xslot + (int64_t)bot[p] * d * d;
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < 2 * d * d; e += gridDim.x * blockDim.x) {
    int r = e % (2 * d), c = e / (2 * d);
    if (r < d) xa[r + (int64_t)c * d] = (double)src[e];
    else xb[(r - d) + (int64_t)c * d] = (double)src[e];
  }
}

// dst = (float) src, n elements.
template <typename T>
__global__ void k_narrow(const T *src, float *dst, int64_t n) {
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x)
    dst[e] = static_cast<float>(src[e]);
}

// Q_hat rows of leaf p = Qs_p[0:h_p], to dst[p] (FP32, column-major, ld ld[p]).
template <typename T>
__global__ void k_leaf_q(const T *Qs, int H, int d, float *const *dsts, const int64_t *ld, const int *rows) {
  const int p = blockIdx.y;
  const int h = rows[p];
  const T *src = Qs + (int64_t)p * H * d;
  for (int c = blockIdx.x; c < d; c += gridDim.x) {
    const T *in = src + (int64_t)c * H;
    float *out = dsts[p] + (int64_t)c * ld[p];
    for (int r = threadIdx.x; r < h; r += blockDim.x) out[r] = (float)in[r];
  }
}

// dst_b = alpha * src_b + beta * dst_b on an m x n block (column-major, strided batches).
template <typename T>
__global__ void k_axpby(int m, int n, T alpha, const T *src, int64_t lds, int64_t ss, T beta, T *dst, int64_t ldd,
                        int64_t sd, int batch) {
  const int64_t per = (int64_t)m * n;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < per * batch;
       e += (int64_t)gridDim.x * blockDim.x) {
    int64_t b = e / per, w = e % per;
    int64_t r = w % m, c = w / m;
    T *o = dst + b * sd + r + c * ldd;
    T v = alpha * src[b * ss + r + c * lds];
    *o = (beta == T(0)) ? v : v + beta * *o;
  }
}

template <typename T>
Error axpby(int m, int n, T alpha, const T *src, int64_t lds, int64_t ss, T beta, T *dst, int64_t ldd, int64_t sd,
            int batch, cudaStream_t st) {
  unsigned g = (unsigned)std::min<int64_t>(ceil_div((int64_t)m * n * batch, 256), 4096);
  note_launch();
  k_axpby<T><<<g, 256, 0, st>>>(m, n, alpha, src, lds, ss, beta, dst, ldd, sd, batch);
  CK_CUDA(cudaGetLastError());
  return ok();
}

// ---------------------------------------------------------------- tree combine panels
// Householder QR of stacked pairs S = [R_a; R_b] (2d x d, ld 2d, both blocks upper
// triangular) in panels of sq_nb(T) columns.  Reflector j is e_j on top and v_j (rows
// 0..j) below, so only the top row j and the bottom rows 0..j take part.  Per panel there
// is one launch over all combines of the level (k_sq_step), its CTAs in four roles:
//   panel:  apply the previous panel's block reflector to this panel's columns, then
//           factor the panel in shared memory (every dot product of a step in one pass,
//           one warp per column);
//   update: apply the previous panel's block reflector to the columns after this panel
//           (W = C_top + V^T C_bot, W2 = T_kk^T W, C_top -= W2, C_bot -= V W2);
//   S:      S = V_bot[:, 0:jp]^T V_jp for the previous panel jp;
//   T:      T[0:jq, panel jq] = -T[0:jq, 0:jq] S T_kk for the panel before that.
// The next panel thus waits on one launch only: it finishes its own columns' update from
// the panel before it (lookahead), while the rest of that update, the S products and the
// T blocks run beside it on other SMs.
// FP64 panels are narrower: every step of a panel takes a dot product with each of its
// columns, and FP64 products are what this part has least of.
template <typename T>
constexpr int sq_nb() { return sizeof(T) == 4 ? 32 : 8; }
constexpr int SQ_KC = 64;         // rows of S (and columns of T) per step of a T-block CTA

// Threads that share one of n_out dot products when there are fewer outputs than threads
// (FP64 tiles: otherwise half the schedulers' FP64 units would idle).
__host__ __device__ constexpr int sq_split(int n_out) { return n_out >= 512 ? 1 : 512 / n_out; }

// sum_{i < n} f(i) over a group of KS consecutive lanes (part = index in the group), four
// chains per thread; every lane of the group gets the total.  All 32 lanes must call it.
template <typename T, int KS, typename F>
__device__ __forceinline__ T group_dot(int n, int part, F f) {
  T a0 = 0, a1 = 0, a2 = 0, a3 = 0;
  int i = part;
  for (; i + 3 * KS < n; i += 4 * KS) {
    a0 += f(i);
    a1 += f(i + KS);
    a2 += f(i + 2 * KS);
    a3 += f(i + 3 * KS);
  }
  for (; i < n; i += KS) a0 += f(i);
  T acc = (a0 + a1) + (a2 + a3);
#pragma unroll
  for (int o = 1; o < KS; o <<= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
  return acc;
}
constexpr int SQ_THREADS = 512;

template <typename T>
size_t sq_step_smem(int d) {
  constexpr int NBS = sq_nb<T>(), LD = NBS + 1;
  const size_t pan = (size_t)NBS * d + (size_t)d * LD + 4 * NBS * LD + 2 * NBS * NBS + 3 * NBS + 4;
  const size_t upd = (size_t)2 * d * LD + 4 * NBS * LD;
  const size_t tbl = (size_t)NBS * (SQ_KC + 1) + (size_t)SQ_KC * LD + 2 * NBS * LD;
  return sizeof(T) * std::max(std::max(pan, upd), tbl);
}

// Panel [j0, j0 + nb): R rows into the top of S, V_bot columns into rows d..2d-1 of Vx
// (zeros below each reflector), the panel's T block into Tm's diagonal.  For j0 > 0 the
// previous panel's reflector is first applied to the panel's columns (its top rows are
// written back; the bottom rows stay in shared memory and are factored).
template <typename T>
__device__ void sq_panel_role(T *sm, T *M, T *Vx, T *Tm, int d, int j0) {
  constexpr int NBS = sq_nb<T>(), LD = NBS + 1;
  constexpr int NW = SQ_THREADS / 32;
  T *Vp = sm;                                     // NBS columns x d rows: the panel's bottom part
  T *Vq = Vp + (size_t)NBS * d;                   // d x LD: the previous panel's V_bot, row-major
  T *Ctp = Vq + (size_t)d * LD;                   // NBS x LD: previous panel's top rows of these columns
  T *Tkp = Ctp + NBS * LD;                        // NBS x LD: previous panel's T_kk
  T *W = Tkp + NBS * LD;
  T *W2 = W + NBS * LD;
  T *Ct = W2 + NBS * LD;                          // NBS x NBS top block, row-major
  T *Tk = Ct + NBS * NBS;                         // NBS x NBS panel T, row-major
  T *Dt = Tk + NBS * NBS;                         // NBS raw dots of the current step
  T *Ih = Dt + NBS;                               // 1 / head of each reflector (Vp keeps x unscaled)
  T *Tau = Ih + NBS;                              // tau of the current step
  const int H = 2 * d;
  const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
  const int nb = min(NBS, d - j0);
  const int rows = j0 + nb;                       // bottom rows the panel touches
  stage_tile<T, 8>(Vp, 1, d, M + d + (int64_t)j0 * H, H, rows, nb, nb);
  for (int e = tid; e < NBS * NBS; e += SQ_THREADS) {
    const int r = e / NBS, c = e % NBS;
    Ct[e] = (r < nb && c < nb) ? M[j0 + r + (int64_t)(j0 + c) * H] : T(0);
    Tk[e] = T(0);
  }
  if (j0 > 0) {
    const int jp = j0 - NBS;                      // full width; its reflectors use bottom rows 0..j0-1
    stage_tile<T, 8>(Vq, LD, 1, Vx + d + (int64_t)jp * H, H, j0, NBS, NBS);
    for (int e = tid; e < NBS * NBS; e += SQ_THREADS) {
      const int r = e % NBS, c = e / NBS;
      Ctp[r * LD + c] = (c < nb) ? M[jp + r + (int64_t)(j0 + c) * H] : T(0);
      Tkp[r * LD + c] = Tm[(jp + r) + (int64_t)(jp + c) * d];
    }
    __syncthreads();
    // W = C_top + V^T C_bot  (r: previous reflector, c: this panel's column)
    constexpr int KS = sq_split(NBS * NBS);
    for (int e = tid; e < NBS * NBS * KS; e += SQ_THREADS) {
      const int o = e / KS, part = e % KS;
      const int r = o % NBS, c = o / NBS;
      const T *y = Vp + (size_t)c * d;
      const T acc = group_dot<T, KS>(c < nb ? j0 : 0, part, [&](int i) { return Vq[i * LD + r] * y[i]; });
      if (part == 0) W[r * LD + c] = (c < nb) ? Ctp[r * LD + c] + acc : T(0);
    }
    __syncthreads();
    // W2 = T_kk^T W ; C_top -= W2
    for (int e = tid; e < NBS * NBS; e += SQ_THREADS) {
      const int c = e % NBS, r = e / NBS;
      T acc = 0;
      for (int k = 0; k <= r; ++k) acc += Tkp[k * LD + r] * W[k * LD + c];
      W2[r * LD + c] = acc;
      if (c < nb) M[jp + r + (int64_t)(j0 + c) * H] = Ctp[r * LD + c] - acc;
    }
    __syncthreads();
    // C_bot -= V W2 on bottom rows 0..j0-1
    for (int e = tid; e < j0 * nb; e += SQ_THREADS) {
      const int i = e % j0, c = e / j0;
      T acc = 0;
#pragma unroll 8
      for (int r = 0; r < NBS; ++r) acc += Vq[i * LD + r] * W2[r * LD + c];
      Vp[(size_t)c * d + i] -= acc;
    }
  }
  __syncthreads();
  for (int jj = 0; jj < nb; ++jj) {
    const int j = j0 + jj;                        // bottom rows 0..j are active
    const T *x = Vp + jj * d;                     // unscaled: the reflector is x / head
    // raw dots of x with every panel column (c == jj gives |x|^2), one warp per column
    for (int c = wid; c < nb; c += NW) {
      const T *y = Vp + c * d;
      T a0 = 0, a1 = 0;
      int i = lane;
      for (; i + 32 <= j; i += 64) {
        a0 += x[i] * y[i];
        a1 += x[i + 32] * y[i + 32];
      }
      if (i <= j) a0 += x[i] * y[i];
      T acc = a0 + a1;
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
      if (lane == 0) {
        Dt[c] = acc;
        if (c == jj) {                            // this step's reflector, formed once
          // normx = |(alpha, x)|, rd = -sign(alpha) normx, head = alpha - rd and
          // tau = (rd - alpha) / rd = 1 + |alpha| / normx: two independent reciprocals
          const T alpha = Ct[jj * NBS + jj];
          const T sig = acc;
          const T normx = sqrt(alpha * alpha + sig);
          T tau = 0, rd = alpha, inv_head = 0;
          if (normx > T(0) && sig > T(0)) {
            const bool neg = alpha < T(0);
            const T aa = neg ? -alpha : alpha;
            const T inv_n = T(1) / normx;
            const T ih = T(1) / (aa + normx);
            tau = T(1) + aa * inv_n;
            inv_head = neg ? -ih : ih;
            rd = neg ? normx : -normx;
          }
          Ct[jj * NBS + jj] = rd;                 // read by no other thread this step
          Tk[jj * NBS + jj] = tau;
          Ih[jj] = inv_head;
          Tau[0] = tau;
        }
      }
    }
    __syncthreads();
    const T tau = Tau[0], inv_head = Ih[jj];
    // the rest of the panel: w_c = Ct[jj][c] + (x . col_c) / head, then the reflection
    for (int c = jj + 1 + wid; c < nb; c += NW) {
      const T w = tau * (Ct[jj * NBS + c] + Dt[c] * inv_head);
      const T g = w * inv_head;
      T *col = Vp + c * d;
      for (int i = lane; i <= j; i += 32) col[i] -= g * x[i];
      if (lane == 0) Ct[jj * NBS + c] -= w;
    }
    // T within the panel: T[r][jj] = -tau sum_{l=r}^{jj-1} T[r][l] (v_l . v_jj), one warp
    // per row r, with v_l . v_jj = Dt[l] Ih[l] inv_head
    for (int r = wid; r < jj; r += NW) {
      T t = 0;
      for (int l = r + lane; l < jj; l += 32) t += Tk[r * NBS + l] * (Dt[l] * Ih[l]);
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
      if (lane == 0) Tk[r * NBS + jj] = -tau * inv_head * t;
    }
    __syncthreads();
  }
  for (int e = tid; e < nb * nb; e += SQ_THREADS) {
    const int r = e / nb, c = e % nb;
    M[j0 + r + (int64_t)(j0 + c) * H] = (r <= c) ? Ct[r * NBS + c] : T(0);
    Tm[(j0 + r) + (int64_t)(j0 + c) * d] = Tk[r * NBS + c];
  }
  for (int c = 0; c < nb; ++c)
    for (int i = tid; i < d; i += SQ_THREADS)
      Vx[d + i + (int64_t)(j0 + c) * H] = (i <= j0 + c) ? Vp[c * d + i] * Ih[c] : T(0);
}

// Panel jp's block reflector applied to nt tiles of NBS columns from cb0 (V_panel and C_bot
// use bottom rows 0..jp+nb-1); V_panel and T_kk are staged once for all of them.
template <typename T>
__device__ void sq_update_role(T *sm, T *M, const T *Vx, const T *Tm, int d, int jp, int cb0, int nt) {
  constexpr int NBS = sq_nb<T>(), LD = NBS + 1;
  T *Vs = sm;                                     // rows x NBS: the panel's V_bot
  T *Cs = Vs + (size_t)d * LD;                    // rows x NBS: C_bot tile
  T *Ctp = Cs + (size_t)d * LD;                   // NBS x NBS: C_top tile
  T *Tk = Ctp + NBS * LD;                         // NBS x NBS: T_kk
  T *W = Tk + NBS * LD;
  T *W2 = W + NBS * LD;
  const int H = 2 * d;
  const int nb = min(NBS, d - jp), rows = jp + nb;
  const int tid = threadIdx.x;
  stage_tile<T, 8>(Vs, LD, 1, Vx + d + (int64_t)jp * H, H, rows, NBS, nb);
  for (int e = tid; e < NBS * NBS; e += blockDim.x) {
    const int r = e % NBS, cc = e / NBS;
    Tk[r * LD + cc] = (r < nb && cc < nb) ? Tm[(jp + r) + (int64_t)(jp + cc) * d] : T(0);
  }
  for (int t = 0; t < nt; ++t) {
    const int cb = cb0 + t * NBS;
    if (cb >= d) break;
    const int nc = min(NBS, d - cb);
    if (t > 0) __syncthreads();                   // the previous tile's reads of Cs, W2 are done
    stage_tile<T, 8>(Cs, LD, 1, M + d + (int64_t)cb * H, H, rows, NBS, nc);
    for (int e = tid; e < NBS * NBS; e += blockDim.x) {
      const int r = e % NBS, cc = e / NBS;
      Ctp[r * LD + cc] = (r < nb && cc < nc) ? M[jp + r + (int64_t)(cb + cc) * H] : T(0);
    }
    __syncthreads();
    // W = C_top + V^T C_bot
    constexpr int KS = sq_split(NBS * NBS);
    for (int e = tid; e < NBS * NBS * KS; e += blockDim.x) {
      const int o = e / KS, part = e % KS;
      const int cc = o % NBS, r = o / NBS;
      const T acc = group_dot<T, KS>(rows, part, [&](int i) { return Vs[i * LD + r] * Cs[i * LD + cc]; });
      if (part == 0) W[r * LD + cc] = Ctp[r * LD + cc] + acc;
    }
    __syncthreads();
    // W2 = T_kk^T W ; C_top -= W2
    for (int e = tid; e < NBS * NBS; e += blockDim.x) {
      const int cc = e % NBS, r = e / NBS;
      T acc = 0;
      for (int k = 0; k <= r; ++k) acc += Tk[k * LD + r] * W[k * LD + cc];
      W2[r * LD + cc] = acc;
      if (r < nb && cc < nc) M[jp + r + (int64_t)(cb + cc) * H] = Ctp[r * LD + cc] - acc;
    }
    __syncthreads();
    // C_bot -= V W2
    for (int e = tid; e < rows * NBS; e += blockDim.x) {
      const int cc = e % NBS, i = e / NBS;
      if (cc >= nc) continue;
      T acc = 0;
#pragma unroll 8
      for (int r = 0; r < NBS; ++r) acc += Vs[i * LD + r] * W2[r * LD + cc];
      M[d + i + (int64_t)(cb + cc) * H] = Cs[i * LD + cc] - acc;
    }
  }
}

// NBS rows from l0 of S = V_bot[:, 0:jp]^T V_panel for panel jp (S: jp x nb, ld d).
template <typename T>
__device__ void sq_s_role(T *sm, const T *Vx, T *S, int d, int jp, int l0) {
  constexpr int NBS = sq_nb<T>(), LD = NBS + 1;
  T *Vs = sm;
  T *Cs = Vs + (size_t)d * LD;
  const int H = 2 * d;
  const int nb = min(NBS, d - jp), rows = jp + nb;
  const int nl = min(NBS, jp - l0);
  const int tid = threadIdx.x;
  stage_tile<T, 8>(Vs, LD, 1, Vx + d + (int64_t)jp * H, H, rows, NBS, nb);
  stage_tile<T, 8>(Cs, LD, 1, Vx + d + (int64_t)l0 * H, H, rows, NBS, nl);
  __syncthreads();
  // S[l0 + ll][c] = V_bot[:, l0 + ll] . V_panel[:, c]  (rows 0..l0+ll carry V_bot)
  constexpr int KS = sq_split(NBS * NBS);
  for (int e = tid; e < NBS * NBS * KS; e += blockDim.x) {
    const int o = e / KS, part = e % KS;
    const int c = o % NBS, ll = o / NBS;
    const bool valid = ll < nl && c < nb;
    const int imax = valid ? min(rows, l0 + ll + 1) : 0;
    const T acc = group_dot<T, KS>(imax, part, [&](int i) { return Cs[i * LD + ll] * Vs[i * LD + c]; });
    if (valid && part == 0) S[(l0 + ll) + (int64_t)c * d] = acc;
  }
}

// T[r][panel jq] = -(sum_{l >= r} T[r][l] S[l][.]) T_kk for NBS rows from r0 (< jq); S and
// T stream through shared memory SQ_KC rows / columns at a time.
template <typename T>
__device__ void sq_tblock_role(T *sm, T *Tm, const T *S, int d, int jq, int r0) {
  constexpr int NBS = sq_nb<T>(), LD = NBS + 1, LK = SQ_KC + 1;
  T *Tt = sm;                                     // NBS x LK: T[r0 + a][l0 + b]
  T *Sb = Tt + NBS * LK;                          // SQ_KC x LD: S[l0 + a][b]   (row-major, ld LD)
  T *U = Sb + SQ_KC * LD;                         // NBS x LD
  T *Tk = U + NBS * LD;                           // NBS x LD
  const int nb = min(NBS, d - jq);
  const int nr = min(NBS, jq - r0);
  const int tid = threadIdx.x;
  for (int e = tid; e < NBS * NBS; e += blockDim.x) {
    const int a = e % NBS, b = e / NBS;
    U[a * LD + b] = 0;
    Tk[a * LD + b] = (a < nb && b < nb) ? Tm[(jq + a) + (int64_t)(jq + b) * d] : T(0);
  }
  for (int l0 = r0; l0 < jq; l0 += SQ_KC) {
    const int nl = min(SQ_KC, jq - l0);
    __syncthreads();
    for (int e = tid; e < NBS * SQ_KC; e += blockDim.x) {
      const int a = e % NBS, b = e / NBS;         // T column-major: consecutive a are consecutive rows
      Tt[a * LK + b] = (a < nr && b < nl) ? Tm[(r0 + a) + (int64_t)(l0 + b) * d] : T(0);
    }
    for (int e = tid; e < SQ_KC * NBS; e += blockDim.x) {
      const int a = e % SQ_KC, b = e / SQ_KC;
      Sb[a * LD + b] = (a < nl && b < nb) ? S[(l0 + a) + (int64_t)b * d] : T(0);
    }
    __syncthreads();
    constexpr int KS = sq_split(NBS * NBS);
    for (int e = tid; e < NBS * NBS * KS; e += blockDim.x) {
      const int o = e / KS, part = e % KS;
      const int c = o % NBS, a = o / NBS;
      const T acc = group_dot<T, KS>(nl, part, [&](int l) { return Tt[a * LK + l] * Sb[l * LD + c]; });
      if (part == 0) U[a * LD + c] += acc;
    }
  }
  __syncthreads();
  for (int e = tid; e < NBS * NBS; e += blockDim.x) {
    const int c = e % NBS, a = e / NBS;
    if (a >= nr || c >= nb) continue;
    T acc = 0;
    for (int k = 0; k < NBS; ++k) acc += U[a * LD + k] * Tk[k * LD + c];
    Tm[(r0 + a) + (int64_t)(jq + c) * d] = -acc;
  }
}

// Step q of a level (j0 = q NBS), combine blockIdx.y: CTAs [0, nP) factor panel q, the
// next nU apply panel q-1 to the columns after panel q, the next nS form S for panel q-1
// (into buffer (q-1) & 1), the rest form T's blocks for panel q-2 (from buffer q & 1).
// CTAs of k_sq_step resident per SM: FP64 tiles are short of FP64 units, not registers;
// double-FP32 ones need twice the registers of FP64 for the same values.
template <typename T>
constexpr int sq_min_blocks() {
  return std::is_same<T, double>::value ? 3 : std::is_same<T, dfloat>::value ? 2 : 1;
}

template <typename T>
__global__ void __launch_bounds__(SQ_THREADS, sq_min_blocks<T>()) k_sq_step(T *M0, T *Vx0, T *Tm0, T *S0, int d, int q, int nP, int nU,
                                                        int nS, int uw) {
  constexpr int NBS = sq_nb<T>();
  // launched as a programmatic dependent of the previous step: wait for that grid to complete
  // (and its writes to be visible), then let the next step's grid be scheduled, so that its
  // CTAs are resident when this one ends (both are no-ops in an ordinary launch)
  asm volatile("griddepcontrol.wait;" ::: "memory");
  asm volatile("griddepcontrol.launch_dependents;");
  extern __shared__ __align__(16) uint8_t sm_raw[];
  T *sm = reinterpret_cast<T *>(sm_raw);
  const int H = 2 * d;
  const int y = blockIdx.y;
  T *M = M0 + (int64_t)y * H * d;
  T *Vx = Vx0 + (int64_t)y * H * d;
  T *Tm = Tm0 + (int64_t)y * d * d;
  const int64_t sS = (int64_t)gridDim.y * d * NBS;
  const int j0 = q * NBS;
  int b = blockIdx.x;
  if (b < nP) {
    sq_panel_role<T>(sm, M, Vx, Tm, d, j0);
    return;
  }
  b -= nP;
  if (b < nU) {
    sq_update_role<T>(sm, M, Vx, Tm, d, j0 - NBS, j0 + NBS + b * uw * NBS, uw);
    return;
  }
  b -= nU;
  if (b < nS) {
    sq_s_role<T>(sm, Vx, S0 + ((q - 1) & 1) * sS + (int64_t)y * d * NBS, d, j0 - NBS, b * NBS);
    return;
  }
  b -= nS;
  sq_tblock_role<T>(sm, Tm, S0 + (q & 1) * sS + (int64_t)y * d * NBS, d, j0 - 2 * NBS, b * NBS);
}

// One stage: P independent QRs of H x d matrices (strided, ld H).
template <typename T>
struct Stage {
  int P = 0, H = 0;
  bool stacked = false;                 // a combine stage: M = [R_a; R_b], H = 2d
  T *M = nullptr, *Vx = nullptr, *Tm = nullptr;
  int *top = nullptr, *bot = nullptr;   // device slot indices (combines); top = slot for leaves
};

template <typename T>
Error run_panel(const Stage<T> &s, int d, int c0, cudaStream_t st) {
  const int h = s.stacked ? c0 + 2 * NB : s.H - c0;
  size_t smem = panel_smem<T>(h);
  const int pt = panel_threads<T>(h);
  note_launch();
  if (pt == 512) {
    CK_CUDA(cudaFuncSetAttribute(k_panel<T, 512>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    k_panel<T, 512><<<s.P, 512, smem, st>>>(s.M, s.Vx, s.Tm, s.H, d, c0, s.stacked ? 1 : 0);
  } else if (pt == 256) {
    CK_CUDA(cudaFuncSetAttribute(k_panel<T, 256>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    k_panel<T, 256><<<s.P, 256, smem, st>>>(s.M, s.Vx, s.Tm, s.H, d, c0, s.stacked ? 1 : 0);
  } else {
    CK_CUDA(cudaFuncSetAttribute(k_panel<T, 128>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    k_panel<T, 128><<<s.P, 128, smem, st>>>(s.M, s.Vx, s.Tm, s.H, d, c0, s.stacked ? 1 : 0);
  }
  CK_CUDA(cudaGetLastError());
  return ok();
}

// Recursive blocked Householder QR of columns [c0, c0 + w) (rows c0..H-1); w % 16 == 0.
// W, W2 are scratch of P * d * d / 4 elements each (enough for every wl x wr block).
template <typename T>
Error rqr(const ckinv_ctx *ctx, const Stage<T> &s, int d, int c0, int w, T *W, T *W2, cudaStream_t st) {
  if (w == NB) return run_panel<T>(s, d, c0, st);
  const int wl = ((w / NB + 1) / 2) * NB, wr = w - wl;
  const int H = s.H, P = s.P;
  const int64_t sM = (int64_t)H * d, sT = (int64_t)d * d, sW = (int64_t)wl * wr;
  CK_TRY(rqr<T>(ctx, s, d, c0, wl, W, W2, st));
  if (s.stacked) {
    // Stacked triangles: V1 = [I (top rows c0..c0+wl); V1_bot (bottom rows 0..c0+wl)],
    // C2's active rows are top c0..c0+w and bottom 0..c0+w.
    const int Kb = c0 + wl;
    T *V1b = s.Vx + d + (int64_t)c0 * H;
    T *C2t = s.M + c0 + (int64_t)(c0 + wl) * H;
    T *C2b = s.M + d + (int64_t)(c0 + wl) * H;
    T *T11 = s.Tm + c0 + (int64_t)c0 * d;
    // W = C2_top[0:wl] + V1_bot^T C2_bot ; W2 = T11^T W
    CK_TRY(axpby<T>(wl, wr, T(1), C2t, H, sM, T(0), W, wl, sW, P, st));
    CK_TRY(gemm_batched<T>(ctx, true, wl, wr, Kb, T(1), V1b, H, sM, C2b, H, sM, T(1), W, wl, sW, P, st));
    CK_TRY(gemm_batched<T>(ctx, true, wl, wr, wl, T(1), T11, d, sT, W, wl, sW, T(0), W2, wl, sW, P, st));
    // C2_top[0:wl] -= W2 ; C2_bot -= V1_bot W2
    CK_TRY(axpby<T>(wl, wr, T(-1), W2, wl, sW, T(1), C2t, H, sM, P, st));
    CK_TRY(gemm_batched<T>(ctx, false, Kb, wr, wl, T(-1), V1b, H, sM, W2, wl, sW, T(1), C2b, H, sM, P, st));
    CK_TRY(rqr<T>(ctx, s, d, c0 + wl, wr, W, W2, st));
    // T12 = -T11 (V1_bot^T V2_bot) T22   (the identity parts of V1 and V2 do not overlap)
    T *V2b = s.Vx + d + (int64_t)(c0 + wl) * H;
    T *T22 = s.Tm + (c0 + wl) + (int64_t)(c0 + wl) * d;
    T *T12 = s.Tm + c0 + (int64_t)(c0 + wl) * d;
    CK_TRY(gemm_batched<T>(ctx, true, wl, wr, Kb, T(1), V1b, H, sM, V2b, H, sM, T(0), W, wl, sW, P, st));
    CK_TRY(gemm_batched<T>(ctx, false, wl, wr, wl, T(1), T11, d, sT, W, wl, sW, T(0), W2, wl, sW, P, st));
    CK_TRY(gemm_batched<T>(ctx, false, wl, wr, wr, T(-1), W2, wl, sW, T22, d, sT, T(0), T12, d, sT, P, st));
    return ok();
  }
  const int K = H - c0;
  T *V1 = s.Vx + c0 + (int64_t)c0 * H;              // rows c0.., columns c0 .. c0+wl
  T *C2 = s.M + c0 + (int64_t)(c0 + wl) * H;        // rows c0.., columns c0+wl .. c0+w
  T *T11 = s.Tm + c0 + (int64_t)c0 * d;
  // W = V1^T C2 ; W2 = T11^T W ; C2 -= V1 W2
  CK_TRY(gemm_batched<T>(ctx, true, wl, wr, K, T(1), V1, H, sM, C2, H, sM, T(0), W, wl, sW, P, st));
  CK_TRY(gemm_batched<T>(ctx, true, wl, wr, wl, T(1), T11, d, sT, W, wl, sW, T(0), W2, wl, sW, P, st));
  CK_TRY(gemm_batched<T>(ctx, false, K, wr, wl, T(-1), V1, H, sM, W2, wl, sW, T(1), C2, H, sM, P, st));
  CK_TRY(rqr<T>(ctx, s, d, c0 + wl, wr, W, W2, st));
  // T12 = -T11 (V1^T V2) T22
  T *V2 = s.Vx + c0 + (int64_t)(c0 + wl) * H;
  T *T22 = s.Tm + (c0 + wl) + (int64_t)(c0 + wl) * d;
  T *T12 = s.Tm + c0 + (int64_t)(c0 + wl) * d;
  CK_TRY(gemm_batched<T>(ctx, true, wl, wr, K, T(1), V1, H, sM, V2, H, sM, T(0), W, wl, sW, P, st));
  CK_TRY(gemm_batched<T>(ctx, false, wl, wr, wl, T(1), T11, d, sT, W, wl, sW, T(0), W2, wl, sW, P, st));
  CK_TRY(gemm_batched<T>(ctx, false, wl, wr, wr, T(-1), W2, wl, sW, T22, d, sT, T(0), T12, d, sT, P, st));
  return ok();
}

// Qs = [X; 0] - V (T (V_top^T X)) for every problem of the stage.
template <typename T>
Error apply_q(const ckinv_ctx *ctx, const Stage<T> &s, int d, const double *Xslot, T *Qs, T *Z1, T *Z2,
              cudaStream_t st) {
  const int H = s.H, P = s.P;
  const int64_t sM = (int64_t)H * d, sD = (int64_t)d * d;
  dim3 g((unsigned)std::min(d, 128), P);
  note_launch();
  k_init_qs<T><<<g, 256, 0, st>>>(Xslot, s.top, H, d, Qs);
  CK_CUDA(cudaGetLastError());
  if (s.stacked) {
    // V = [I; V_bot]:  Z2 = T X ;  top = X - Z2 ;  bottom = -V_bot Z2
    CK_TRY(gemm_batched<T>(ctx, false, d, d, d, T(1), s.Tm, d, sD, Qs, H, sM, T(0), Z2, d, sD, P, st));
    CK_TRY(axpby<T>(d, d, T(-1), Z2, d, sD, T(1), Qs, H, sM, P, st));
    CK_TRY(gemm_batched<T>(ctx, false, d, d, d, T(-1), s.Vx + d, H, sM, Z2, d, sD, T(0), Qs + d, H, sM, P, st));
    return ok();
  }
  // V^T [X; 0] = V[0:d]^T X: the zero rows of [X; 0] contribute nothing
  CK_TRY(gemm_batched<T>(ctx, true, d, d, d, T(1), s.Vx, H, sM, Qs, H, sM, T(0), Z1, d, sD, P, st));
  CK_TRY(gemm_batched<T>(ctx, false, d, d, d, T(1), s.Tm, d, sD, Z1, d, sD, T(0), Z2, d, sD, P, st));
  CK_TRY(gemm_batched<T>(ctx, false, H, d, d, T(-1), s.Vx, H, sM, Z2, d, sD, T(1), Qs, H, sM, P, st));
  return ok();
}

// Leaves of one height whose Q_hat rows follow each other at a fixed stride in one output.
struct LeafRun {
  int first, count, h;
  float *dst;          // Q_hat rows of leaf `first`
  int64_t ldq, stride; // leading dimension, rows between consecutive leaves
};

// The leaf stage of the top-down pass for FP32 leaves, written straight into Q_hat: leaf p's
// rows are Q_p [X_p; 0] = [X_p; 0] - V_p (T_p (V_p[0:d]^T X_p)); the product goes to Q_hat's
// rows as -V Z2, and X is then added to each leaf's first d rows (the sum the GEMM's epilogue
// would form, in the same FP32 operation), so no staging array is filled with [X; 0] and none
// is copied out.
Error apply_q_leaves(const ckinv_ctx *ctx, const Stage<float> &s, int d, const double *Xslot, float *X0, float *Z1,
                     float *Z2, const std::vector<LeafRun> &runs, cudaStream_t st) {
  const int H = s.H, P = s.P;
  const int64_t sM = (int64_t)H * d, sD = (int64_t)d * d;
  dim3 g((unsigned)std::min(d, 128), P);
  note_launch();
  k_init_qs<float><<<g, 256, 0, st>>>(Xslot, s.top, d, d, X0);   // each leaf's X, d x d
  CK_CUDA(cudaGetLastError());
  CK_TRY(gemm_batched<float>(ctx, true, d, d, d, 1.f, s.Vx, H, sM, X0, d, sD, 0.f, Z1, d, sD, P, st));
  CK_TRY(gemm_batched<float>(ctx, false, d, d, d, 1.f, s.Tm, d, sD, Z1, d, sD, 0.f, Z2, d, sD, P, st));
  for (const LeafRun &r : runs) {
    CK_TRY(gemm_batched<float>(ctx, false, r.h, d, d, -1.f, s.Vx + r.first * sM, H, sM, Z2 + r.first * sD, d, sD,
                               0.f, r.dst, r.ldq, r.stride, r.count, st));
    CK_TRY(axpby<float>(d, d, 1.f, X0 + r.first * sD, d, sD, 1.f, r.dst, r.ldq, r.stride, r.count, st));
  }
  return ok();
}

struct Level {
  std::vector<int> top, bot;   // combines (top slot, bottom slot)
  bool fp64 = false;
};

template <typename T>
Error alloc_stage(Stage<T> &s, int P, int H, int d, const std::vector<int> &top, const std::vector<int> &bot,
                  ckinv_ctx *ctx, std::vector<void *> &owned, cudaStream_t st) {
  s.P = P;
  s.H = H;
  CK_CUDA(dev_alloc((void **)&s.M, sizeof(T) * (size_t)P * H * d, st));
  owned.push_back(s.M);
  CK_CUDA(dev_alloc((void **)&s.Vx, sizeof(T) * (size_t)P * H * d, st));
  owned.push_back(s.Vx);
  CK_CUDA(dev_alloc((void **)&s.Tm, sizeof(T) * (size_t)P * d * d, st));
  owned.push_back(s.Tm);
  CK_CUDA(cudaMemsetAsync(s.Tm, 0, sizeof(T) * (size_t)P * d * d, st));
  CK_CUDA(dev_alloc((void **)&s.top, sizeof(int) * P, st));
  owned.push_back(s.top);
  CK_TRY(stage_upload(ctx, top.data(), sizeof(int) * P, s.top, st));
  if (!bot.empty()) {
    CK_CUDA(dev_alloc((void **)&s.bot, sizeof(int) * P, st));
    owned.push_back(s.bot);
    CK_TRY(stage_upload(ctx, bot.data(), sizeof(int) * P, s.bot, st));
  }
  return ok();
}

// Panel by panel over all combines of a level, one k_sq_step launch per panel plus two
// that finish the last panels' S products and T blocks.
template <typename T>
Error sq_factor(const ckinv_ctx *ctx, const Stage<T> &s, int d, bool with_t, cudaStream_t st) {
  (void)ctx;
  constexpr int NBS = sq_nb<T>();
  const int P = s.P;
  const int npan = (d + NBS - 1) / NBS;
  const size_t smem = sq_step_smem<T>(d);
  CK_CUDA(cudaFuncSetAttribute(k_sq_step<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  T *S = nullptr;
  CK_CUDA(dev_alloc((void **)&S, sizeof(T) * 2 * (size_t)P * d * NBS, st));
  // update tiles per CTA: with many combines the level is FP64-throughput bound, and a CTA
  // that stages the panel's reflectors once for several tiles wastes less; with few it is
  // latency bound, and one tile per CTA keeps each CTA short
  const int uw = (sizeof(T) == 8 && P >= 16) ? 4 : 1;
  // steps after the first start as programmatic dependents (the launch latency between
  // steps overlaps the previous step); in stream capture, ordinary launches
  cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
  CK_CUDA(cudaStreamIsCapturing(st, &cap));
  cudaLaunchAttribute pdl[1];
  pdl[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  pdl[0].val.programmaticStreamSerializationAllowed = 1;
  bool first = true;
  Error e = ok();
  for (int q = 0; q <= npan + 1 && !e.st; ++q) {
    const int j0 = q * NBS, jp = j0 - NBS, jq = j0 - 2 * NBS;
    const int nP = q < npan ? 1 : 0;
    const int ntile = (q >= 1 && q < npan) ? (std::max(0, d - j0 - NBS) + NBS - 1) / NBS : 0;
    const int nU = (ntile + uw - 1) / uw;
    const int nS = (with_t && q >= 1 && q - 1 < npan && jp > 0) ? (jp + NBS - 1) / NBS : 0;
    const int nT = (with_t && q >= 2 && q - 2 < npan && jq > 0) ? (jq + NBS - 1) / NBS : 0;
    const int nx = nP + nU + nS + nT;
    if (nx == 0) continue;
    note_launch();
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)nx, (unsigned)P);
    cfg.blockDim = dim3(SQ_THREADS);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    cfg.attrs = pdl;
    cfg.numAttrs = (!first && cap == cudaStreamCaptureStatusNone) ? 1 : 0;
    first = false;
    cudaError_t ce = cudaLaunchKernelEx(&cfg, k_sq_step<T>, s.M, s.Vx, s.Tm, S, d, q, nP, nU, nS, uw);
    if (ce == cudaSuccess) ce = cudaGetLastError();
    if (ce != cudaSuccess) e = fail(CKINV_ECUDA, cudaGetErrorString(ce));
  }
  cudaFreeAsync(S, st);
  return e;
}

// Off-diagonal blocks of the compact-WY factor T of every combine of a stage, from its
// diagonal blocks (width nb0, the combine's panels) and G = V_bot^T V_bot (the identity parts
// of different reflectors do not overlap, so V^T V = V_bot^T V_bot off the diagonal):
// T12 = -T11 G12 T22 for adjacent blocks of width w, w = nb0, 2 nb0, ..., a ragged last
// block pairing with its full neighbour when their count is even.  Full pairs of a width
// are one two-level batched GEMM (pairs x combines).
template <typename T>
Error assemble_t(const ckinv_ctx *ctx, const Stage<T> &s, int d, int nb0, cudaStream_t st) {
  const int P = s.P, H = s.H;
  const int64_t sM = (int64_t)H * d, sD = (int64_t)d * d;
  T *G = nullptr, *W = nullptr;
  CK_CUDA(dev_alloc((void **)&G, sizeof(T) * (size_t)P * d * d, st));
  CK_CUDA(dev_alloc((void **)&W, sizeof(T) * (size_t)P * ((size_t)d * d / 4 + 1), st));
  Error e = gemm_batched<T>(ctx, true, d, d, d, T(1), s.Vx + d, H, sM, s.Vx + d, H, sM, T(0), G, d, sD, P, st);
  for (int w = nb0; w < d && !e.st; w *= 2) {
    const int nfull = d / w, rem = d - nfull * w, np = nfull / 2;
    const int64_t sp = 2LL * w * (d + 1);        // between pairs along the diagonal
    if (np > 0) {
      const int64_t sW = (int64_t)w * w, sW2 = (int64_t)np * w * w;
      // W = G12 T22 ; T12 = -T11 W
      if ((e = gemm_batched2<T>(ctx, false, w, w, w, T(1), G + (int64_t)w * d, d, sp, sD, s.Tm + w + (int64_t)w * d,
                                d, sp, sD, T(0), W, w, sW, sW2, np, P, st)).st)
        break;
      if ((e = gemm_batched2<T>(ctx, false, w, w, w, T(-1), s.Tm, d, sp, sD, W, w, sW, sW2, T(0),
                                s.Tm + (int64_t)w * d, d, sp, sD, np, P, st)).st)
        break;
    }
    if ((nfull & 1) && rem > 0) {                // block nfull-1 (full) with the ragged block
      const int c0 = (nfull - 1) * w;
      const int64_t o12 = c0 + (int64_t)(c0 + w) * d, o22 = (c0 + w) + (int64_t)(c0 + w) * d;
      const int64_t o11 = c0 + (int64_t)c0 * d;
      if ((e = gemm_batched<T>(ctx, false, w, rem, rem, T(1), G + o12, d, sD, s.Tm + o22, d, sD, T(0), W, w,
                               (int64_t)w * rem, P, st)).st)
        break;
      if ((e = gemm_batched<T>(ctx, false, w, rem, w, T(-1), s.Tm + o11, d, sD, W, w, (int64_t)w * rem, T(0),
                               s.Tm + o12, d, sD, P, st)).st)
        break;
    }
  }
  cudaFreeAsync(G, st);
  cudaFreeAsync(W, st);
  return e;
}

// A combine stage: the panel-by-panel factorization, then its R factors into the slots.
template <typename T>
Error factor_stacked(const ckinv_ctx *ctx, const Stage<T> &s, int d, double *Rslot, cudaStream_t st, bool with_t) {
  CK_TRY(sq_factor<T>(ctx, s, d, with_t, st));
  dim3 g((unsigned)std::min<int64_t>(ceil_div((int64_t)d * d, 256), 64), s.P);
  note_launch();
  k_extract_r<T><<<g, 256, 0, st>>>(s.M, s.H, d, s.top, Rslot);
  CK_CUDA(cudaGetLastError());
  return ok();
}

template <typename T>
Error factor_stage(const ckinv_ctx *ctx, const Stage<T> &s, int d, double *Rslot, cudaStream_t st,
                   bool with_t = true) {
  if (s.stacked) return factor_stacked<T>(ctx, s, d, Rslot, st, with_t);
  T *W = nullptr, *W2 = nullptr;
  const size_t sw = (size_t)s.P * ((d / 2 + NB) * (d / 2 + NB));
  CK_CUDA(dev_alloc((void **)&W, sizeof(T) * sw, st));
  CK_CUDA(dev_alloc((void **)&W2, sizeof(T) * sw, st));
  Error e = rqr<T>(ctx, s, d, 0, d, W, W2, st);
  cudaFreeAsync(W, st);
  cudaFreeAsync(W2, st);
  CK_TRY(e);
  dim3 g((unsigned)std::min<int64_t>(ceil_div((int64_t)d * d, 256), 64), s.P);
  note_launch();
  k_extract_r<T><<<g, 256, 0, st>>>(s.M, s.H, d, s.top, Rslot);
  CK_CUDA(cudaGetLastError());
  return ok();
}

// Several independent problems of the same width d factor together: their leaves form one
// leaf stage, and level l of every problem's tree (counted from its leaves) one combine stage,
// so each launch covers all problems.  A problem's arithmetic does not depend on the others:
// every leaf and combine is its own QR (the GEMMs' split of the K dimension may differ with
// the batch size, which changes rounding only).
template <typename TL>
Error tsqr_impl(ckinv_ctx *ctx, const std::vector<TsqrProblem> &probs, int d, int b, int fp64_levels,
                cudaStream_t st) {
  constexpr bool LEAF64 = sizeof(TL) == 8;
  // ---- leaves (Eq. 1), problem by problem
  std::vector<const float *> lsrc;
  std::vector<float *> ldst;
  std::vector<int64_t> lld, lldq;
  std::vector<int> rows;
  std::vector<int> first(probs.size() + 1, 0);
  for (size_t q = 0; q < probs.size(); ++q) {
    const TsqrProblem &pr = probs[q];
    first[q] = (int)rows.size();
    std::vector<int64_t> r0;
    std::vector<int> h;
    for (int64_t s0 = 0; s0 < pr.n; s0 += b) {
      r0.push_back(s0);
      h.push_back((int)std::min<int64_t>(b, pr.n - s0));
    }
    if (h.size() > 1 && h.back() < d) {
      int last = h.back();
      h.pop_back();
      r0.pop_back();
      h.back() += last;
    }
    for (size_t i = 0; i < h.size(); ++i) {
      lsrc.push_back(pr.Y + r0[i]);
      lld.push_back(pr.ldy);
      ldst.push_back(pr.Q + r0[i]);
      lldq.push_back(pr.ldq);
      rows.push_back(h[i]);
    }
  }
  first[probs.size()] = (int)rows.size();
  const int L = (int)rows.size();
  int Hl = 0;
  for (int m : rows) Hl = std::max(Hl, m);
  Hl = (int)ceil_div(Hl, 16) * 16;
  if (panel_smem<TL>(Hl) > kPanelSmemMax)
    return fail(CKINV_EUNSUPPORTED, "tsqr: leaf height too large for the shared-memory panel");
  // ---- tree levels (Eqs. 2-3): each problem's binary tree over its own leaves; level l of
  // all problems is one stage.  The top fp64_levels of a problem's tree are FP64-class.
  std::vector<Level> levels;
  std::vector<int> root(probs.size());
  for (size_t q = 0; q < probs.size(); ++q) {
    std::vector<int> active;
    for (int i = first[q]; i < first[q + 1]; ++i) active.push_back(i);
    std::vector<Level> own;
    while (active.size() > 1) {
      Level lv;
      std::vector<int> nxt;
      for (size_t i = 0; i + 1 < active.size(); i += 2) {
        lv.top.push_back(active[i]);
        lv.bot.push_back(active[i + 1]);
        nxt.push_back(active[i]);
      }
      if (active.size() % 2) nxt.push_back(active.back());
      active = nxt;
      own.push_back(lv);
    }
    root[q] = active[0];
    const int Hq = (int)own.size();
    int nf64 = (fp64_levels < 0) ? Hq : std::min(fp64_levels, Hq);
    if (LEAF64) nf64 = Hq;   // an FP64 leaf stage feeds an all-FP64 tree
    if (levels.size() < own.size()) levels.resize(own.size());
    for (int l = 0; l < Hq; ++l) {
      const bool f64 = l >= Hq - nf64;
      if (!levels[l].top.empty() && levels[l].fp64 != f64)
        return fail(CKINV_EINVAL, "tsqr: problems of one factorization need the same FP64-class levels");
      levels[l].fp64 = f64;
      levels[l].top.insert(levels[l].top.end(), own[l].top.begin(), own[l].top.end());
      levels[l].bot.insert(levels[l].bot.end(), own[l].bot.begin(), own[l].bot.end());
    }
  }
  const int Hn = (int)levels.size();

  std::vector<void *> owned;
  double *Rslot = nullptr, *Xslot = nullptr;
  const float **d_src = nullptr;
  float **d_dst = nullptr;
  int64_t *d_ld = nullptr, *d_ldq = nullptr;
  int *d_rows = nullptr;
  Error e = ok();
  do {
    if (dev_alloc((void **)&Rslot, sizeof(double) * (size_t)L * d * d, st) != cudaSuccess ||
        dev_alloc((void **)&Xslot, sizeof(double) * (size_t)L * d * d, st) != cudaSuccess ||
        dev_alloc((void **)&d_src, sizeof(float *) * L, st) != cudaSuccess ||
        dev_alloc((void **)&d_dst, sizeof(float *) * L, st) != cudaSuccess ||
        dev_alloc((void **)&d_ld, sizeof(int64_t) * L, st) != cudaSuccess ||
        dev_alloc((void **)&d_ldq, sizeof(int64_t) * L, st) != cudaSuccess ||
        dev_alloc((void **)&d_rows, sizeof(int) * L, st) != cudaSuccess) {
      e = fail(CKINV_ENOMEM, "tsqr workspace");
      break;
    }
    owned.insert(owned.end(), {(void *)Rslot, (void *)Xslot, (void *)d_src, (void *)d_dst, (void *)d_ld,
                               (void *)d_ldq, (void *)d_rows});
    if ((e = stage_upload(ctx, lsrc.data(), sizeof(float *) * L, d_src, st)).st) break;
    if ((e = stage_upload(ctx, ldst.data(), sizeof(float *) * L, d_dst, st)).st) break;
    if ((e = stage_upload(ctx, lld.data(), sizeof(int64_t) * L, d_ld, st)).st) break;
    if ((e = stage_upload(ctx, lldq.data(), sizeof(int64_t) * L, d_ldq, st)).st) break;
    if ((e = stage_upload(ctx, rows.data(), sizeof(int) * L, d_rows, st)).st) break;
    // ---- leaf stage
    Stage<TL> leaf;
    std::vector<int> ident(L);
    for (int i = 0; i < L; ++i) ident[i] = i;
    if ((e = alloc_stage<TL>(leaf, L, Hl, d, ident, {}, ctx, owned, st)).st) break;
    {
      dim3 g((unsigned)std::min(d, 128), L);
      note_launch();
      k_gather_leaves<TL><<<g, 256, 0, st>>>(d_src, d_ld, d_rows, Hl, d, leaf.M);
    }
    if ((e = factor_stage<TL>(ctx, leaf, d, Rslot, st)).st) break;
    // ---- tree stages, bottom-up
    std::vector<Stage<float>> sf(Hn);
    std::vector<Stage<double>> sd(Hn);
    std::vector<Stage<dfloat>> sx(Hn);
    for (int l = 0; l < Hn && !e.st; ++l) {
      const Level &lv = levels[l];
      const int P = (int)lv.top.size();
      dim3 g((unsigned)std::min<int64_t>(ceil_div(2LL * d * d, 256), 256), P);
      if (lv.fp64 && LEAF64) {
        // FP64 leaves: an FP64 tree, whose reflectors and T factors form an FP64 Q_hat
        if ((e = alloc_stage<double>(sd[l], P, 2 * d, d, lv.top, lv.bot, ctx, owned, st)).st) break;
        sd[l].stacked = true;
        note_launch();
        k_build_stack<double><<<g, 256, 0, st>>>(Rslot, sd[l].top, sd[l].bot, d, sd[l].M);
        if ((e = factor_stacked<double>(ctx, sd[l], d, Rslot, st, true)).st) break;
      } else if (lv.fp64) {
        // FP32 leaves: the combine in double-FP32 arithmetic (R in and out as FP64); Q_hat
        // is applied in FP32, so keep FP32 copies of the level's reflectors and T factors
        if ((e = alloc_stage<dfloat>(sx[l], P, 2 * d, d, lv.top, lv.bot, ctx, owned, st)).st) break;
        sx[l].stacked = true;
        note_launch();
        k_build_stack<dfloat><<<g, 256, 0, st>>>(Rslot, sx[l].top, sx[l].bot, d, sx[l].M);
        if ((e = factor_stacked<dfloat>(ctx, sx[l], d, Rslot, st, false)).st) break;
        Stage<float> &q = sf[l];
        q.P = P;
        q.H = 2 * d;
        q.stacked = true;
        q.top = sx[l].top;
        q.bot = sx[l].bot;
        const int64_t nv = (int64_t)P * 2 * d * d, nt = (int64_t)P * d * d;
        if (dev_alloc((void **)&q.Vx, sizeof(float) * nv, st) != cudaSuccess ||
            dev_alloc((void **)&q.Tm, sizeof(float) * nt, st) != cudaSuccess) {
          e = fail(CKINV_ENOMEM, "tsqr FP32 reflector copies");
          break;
        }
        owned.insert(owned.end(), {(void *)q.Vx, (void *)q.Tm});
        note_launch();
        k_narrow<dfloat><<<(unsigned)std::min<int64_t>(ceil_div(nv, 256), 4096), 256, 0, st>>>(sx[l].Vx, q.Vx, nv);
        note_launch();
        k_narrow<dfloat><<<(unsigned)std::min<int64_t>(ceil_div(nt, 256), 4096), 256, 0, st>>>(sx[l].Tm, q.Tm, nt);
        // the combine formed T's diagonal blocks only; the rest in FP32 for Q_hat
        if ((e = assemble_t<float>(ctx, q, d, sq_nb<dfloat>(), st)).st) break;
      } else {
        if ((e = alloc_stage<float>(sf[l], P, 2 * d, d, lv.top, lv.bot, ctx, owned, st)).st) break;
        sf[l].stacked = true;
        note_launch();
        k_build_stack<float><<<g, 256, 0, st>>>(Rslot, sf[l].top, sf[l].bot, d, sf[l].M);
        e = factor_stage<float>(ctx, sf[l], d, Rslot, st);
      }
    }
    if (e.st) break;
    // ---- each problem's root (Eq. 4): R = D R_root, X_root = D
    for (size_t q = 0; q < probs.size(); ++q) {
      const int64_t o = (int64_t)root[q] * d * d;
      note_launch();
      k_finish_root<<<(unsigned)std::min<int64_t>(ceil_div((int64_t)d * d, 256), 256), 256, 0, st>>>(
          Rslot + o, d, probs[q].R, Xslot + o);
    }
    // ---- Q_hat, top-down
    const size_t qmax = std::max((size_t)L * Hl * d, (size_t)L * 2 * d * d);
    const size_t zmax = (size_t)L * d * d;
    const size_t esz = LEAF64 ? sizeof(double) : sizeof(float);
    void *Qs = nullptr, *Z1 = nullptr, *Z2 = nullptr;
    if (dev_alloc(&Qs, esz * qmax, st) != cudaSuccess || dev_alloc(&Z1, esz * zmax, st) != cudaSuccess ||
        dev_alloc(&Z2, esz * zmax, st) != cudaSuccess) {
      e = fail(CKINV_ENOMEM, "tsqr Q workspace");
      break;
    }
    owned.insert(owned.end(), {Qs, Z1, Z2});
    for (int l = Hn - 1; l >= 0 && !e.st; --l) {
      const int P = (int)levels[l].top.size();
      dim3 g((unsigned)std::min<int64_t>(ceil_div(2LL * d * d, 256), 256), P);
      if (LEAF64) {
        if ((e = apply_q<double>(ctx, sd[l], d, Xslot, (double *)Qs, (double *)Z1, (double *)Z2, st)).st) break;
        note_launch();
        k_scatter_x<double><<<g, 256, 0, st>>>((double *)Qs, sd[l].top, sd[l].bot, d, Xslot);
      } else {
        if ((e = apply_q<float>(ctx, sf[l], d, Xslot, (float *)Qs, (float *)Z1, (float *)Z2, st)).st) break;
        note_launch();
        k_scatter_x<float><<<g, 256, 0, st>>>((float *)Qs, sf[l].top, sf[l].bot, d, Xslot);
      }
    }
    if (e.st) break;
    if constexpr (LEAF64) {
      if ((e = apply_q<TL>(ctx, leaf, d, Xslot, (TL *)Qs, (TL *)Z1, (TL *)Z2, st)).st) break;
      dim3 g((unsigned)std::min(d, 128), L);
      note_launch();
      k_leaf_q<TL><<<g, 256, 0, st>>>((TL *)Qs, Hl, d, d_dst, d_ldq, d_rows);
    } else {
      // runs of equal-height leaves of one problem, consecutive in its Q_hat
      std::vector<LeafRun> runs;
      for (int i = 0; i < L; ++i) {
        if (!runs.empty()) {
          LeafRun &r = runs.back();
          const int last = r.first + r.count - 1;
          if (rows[i] == r.h && lldq[i] == r.ldq && ldst[i] == ldst[last] + r.h && (r.count == 1 || r.stride == r.h)) {
            r.stride = r.h;
            ++r.count;
            continue;
          }
        }
        runs.push_back(LeafRun{i, 1, rows[i], ldst[i], lldq[i], rows[i]});
      }
      if ((e = apply_q_leaves(ctx, leaf, d, Xslot, (float *)Qs, (float *)Z1, (float *)Z2, runs, st)).st) break;
    }
    cudaError_t ce = cudaGetLastError();
    if (ce != cudaSuccess) e = fail(CKINV_ECUDA, cudaGetErrorString(ce));
  } while (0);
  for (void *p : owned)
    if (p) cudaFreeAsync(p, st);
  return e;
}

// Tallest leaf whose NB-column panel fits in shared memory; a leaf may hold up to
// b + d - 1 rows after the short tail is merged, so b is capped at that minus d.
int max_block_rows(int d, bool leaf_fp64) {
  int h = 16;
  while ((leaf_fp64 ? panel_smem<double>(h + 16) : panel_smem<float>(h + 16)) <= kPanelSmemMax) h += 16;
  int b = h - d;
  return std::max(b, 0) / 16 * 16;
}

}  // namespace

int max_leaf_rows(int d, bool leaf_fp64) { return max_block_rows(d, leaf_fp64); }

int auto_block_rows(int64_t n, int d, int sm_count) {
  (void)sm_count;
  int64_t b = 2048;
  if (n < 2 * b) b = std::max<int64_t>(d, (n + 1) / 2);
  if (b < d) b = d;
  return (int)b;
}

Error tsqr_factor_multi(ckinv_ctx *ctx, const std::vector<TsqrProblem> &probs, int d, int b, int fp64_levels,
                        bool leaf_fp64, bool tc_gemm, cudaStream_t st) {
  // the FP32 GEMMs of this factorization on the tensor cores or on the CUDA cores
  struct Restore {
    ckinv_ctx *c;
    bool v;
    ~Restore() { c->gemm_tc = v; }
  } restore{ctx, ctx->gemm_tc};
  ctx->gemm_tc = tc_gemm;
  if (probs.empty()) return ok();
  if (d % NB != 0) return fail(CKINV_EINVAL, "tsqr: d must be a multiple of 16");
  for (const TsqrProblem &pr : probs)
    if (pr.n < d || !pr.Y || !pr.Q || !pr.R || pr.ldy < pr.n || pr.ldq < pr.n)
      return fail(CKINV_EINVAL, "tsqr: each problem needs n >= d, ld >= n and its buffers");
  const int bmax = max_block_rows(d, leaf_fp64);
  if (bmax < d) return fail(CKINV_EUNSUPPORTED, "tsqr: d too large for a shared-memory panel");
  if (b > bmax) b = bmax;   // R and Q_hat do not depend on the leaf height
  if (leaf_fp64) return tsqr_impl<double>(ctx, probs, d, b, fp64_levels, st);
  return tsqr_impl<float>(ctx, probs, d, b, fp64_levels, st);
}

Error tsqr_factor(ckinv_ctx *ctx, int64_t n, int d, int b, int fp64_levels, bool leaf_fp64, bool tc_gemm,
                  const float *Y, int64_t ldy, float *Qout, double *Rout, cudaStream_t st) {
  const TsqrProblem pr{n, Y, ldy, Qout, n, Rout};
  return tsqr_factor_multi(ctx, std::vector<TsqrProblem>{pr}, d, b, fp64_levels, leaf_fp64, tc_gemm, st);
}

// The top of a TSQR whose leaves were factored elsewhere (row shards, one per GPU): the
// binary tree of FP64 combines over the G given R factors (Rin, G strided d x d blocks,
// column-major), the root normalised to diag(R) >= 0 (Rout), and every leaf's d x d block of
// the combined Q factor (Xout, G strided blocks): the stacked R's equal Qtop Rout, so a
// shard's final Q_hat rows are its own Q_hat times its block.  Pairs are formed left to
// right and an odd node passes up, as in the single-GPU tree.
Error tsqr_combine_r(ckinv_ctx *ctx, int G, int d, const double *Rin, double *Rout, double *Xout, cudaStream_t st) {
  if (G < 1 || d % NB != 0) return fail(CKINV_EINVAL, "tsqr_combine_r: need G >= 1 and d % 16 == 0");
  std::vector<Level> levels;
  {
    std::vector<int> active(G);
    for (int i = 0; i < G; ++i) active[i] = i;
    while (active.size() > 1) {
      Level lv;
      std::vector<int> nxt;
      for (size_t i = 0; i + 1 < active.size(); i += 2) {
        lv.top.push_back(active[i]);
        lv.bot.push_back(active[i + 1]);
        nxt.push_back(active[i]);
      }
      if (active.size() % 2) nxt.push_back(active.back());
      active = nxt;
      levels.push_back(lv);
    }
  }
  const int Hn = (int)levels.size();
  const size_t dd = (size_t)d * d;
  std::vector<void *> owned;
  double *Rslot = nullptr, *Xslot = nullptr;
  Error e = ok();
  do {
    if (dev_alloc((void **)&Rslot, sizeof(double) * G * dd, st) != cudaSuccess ||
        dev_alloc((void **)&Xslot, sizeof(double) * G * dd, st) != cudaSuccess) {
      e = fail(CKINV_ENOMEM, "tsqr_combine_r workspace");
      break;
    }
    owned.insert(owned.end(), {(void *)Rslot, (void *)Xslot});
    if (cudaMemcpyAsync(Rslot, Rin, sizeof(double) * G * dd, cudaMemcpyDeviceToDevice, st) != cudaSuccess) {
      e = fail(CKINV_ECUDA, "tsqr_combine_r: copy of the R factors");
      break;
    }
    std::vector<Stage<double>> sd(Hn);
    for (int l = 0; l < Hn && !e.st; ++l) {
      const Level &lv = levels[l];
      const int P = (int)lv.top.size();
      dim3 g((unsigned)std::min<int64_t>(ceil_div(2LL * d * d, 256), 256), P);
      if ((e = alloc_stage<double>(sd[l], P, 2 * d, d, lv.top, lv.bot, ctx, owned, st)).st) break;
      sd[l].stacked = true;
      note_launch();
      k_build_stack<double><<<g, 256, 0, st>>>(Rslot, sd[l].top, sd[l].bot, d, sd[l].M);
      e = factor_stage<double>(ctx, sd[l], d, Rslot, st, true);
    }
    if (e.st) break;
    note_launch();
    k_finish_root<<<(unsigned)std::min<int64_t>(ceil_div((int64_t)d * d, 256), 256), 256, 0, st>>>(Rslot, d, Rout,
                                                                                                   Xslot);
    double *Qs = nullptr, *Z1 = nullptr, *Z2 = nullptr;
    const size_t qmax = std::max<size_t>(1, (size_t)G * 2 * dd);
    if (dev_alloc((void **)&Qs, sizeof(double) * qmax, st) != cudaSuccess ||
        dev_alloc((void **)&Z1, sizeof(double) * G * dd, st) != cudaSuccess ||
        dev_alloc((void **)&Z2, sizeof(double) * G * dd, st) != cudaSuccess) {
      e = fail(CKINV_ENOMEM, "tsqr_combine_r Q workspace");
      break;
    }
    owned.insert(owned.end(), {(void *)Qs, (void *)Z1, (void *)Z2});
    for (int l = Hn - 1; l >= 0 && !e.st; --l) {
      const int P = (int)levels[l].top.size();
      dim3 g((unsigned)std::min<int64_t>(ceil_div(2LL * d * d, 256), 256), P);
      if ((e = apply_q<double>(ctx, sd[l], d, Xslot, Qs, Z1, Z2, st)).st) break;
      note_launch();
      k_scatter_x<double><<<g, 256, 0, st>>>(Qs, sd[l].top, sd[l].bot, d, Xslot);
    }
    if (e.st) break;
    if (cudaMemcpyAsync(Xout, Xslot, sizeof(double) * G * dd, cudaMemcpyDeviceToDevice, st) != cudaSuccess)
      e = fail(CKINV_ECUDA, "tsqr_combine_r: copy of the Q blocks");
    cudaError_t ce = cudaGetLastError();
    if (e.st == CKINV_OK && ce != cudaSuccess) e = fail(CKINV_ECUDA, cudaGetErrorString(ce));
  } while (0);
  for (void *p : owned)
    if (p) cudaFreeAsync(p, st);
  return e;
}

}  // namespace ckinv
