// Blocked tall-skinny QR of Y (Sec. 3.3, Eqs. 1-4) and the explicit Q_hat.
//
// Leaves: each block of b rows is factored by blocked Householder QR (compact WY,
// panels of NB = 16 columns): one CTA per leaf factors the panel in shared memory with
// warp-shuffle reductions, then (leaf x column-tile) CTAs apply the panel's block
// reflector to the trailing columns.  Tree: pairs of d x d upper-triangular R factors are
// combined by the same two kernels working on the stacked matrix [R_a; R_b] restricted to
// its structurally nonzero rows (top rows c0..c0+NB-1 of R_a, bottom rows 0..c0+NB-1 of
// R_b for the panel at column c0), so a combine costs ~2/3 d^3 flops instead of ~3.3 d^3.
// The top `fp64_levels` tree levels run in FP64, the rest in FP32.  Pairs are formed left
// to right at every level; an odd last node passes up unchanged.  Finally Q_hat is formed
// top-down: the root's coefficient block D = sign(diag R) is pushed through the tree's
// reflectors into one d x d block per leaf, then through each leaf's reflectors.
#include "internal.cuh"

namespace ckinv {
namespace {

constexpr int NB = 16;            // panel width
constexpr int PF_THREADS = 512;   // panel-factor CTA
constexpr int BR_THREADS = 256;   // block-reflector CTA
constexpr int TW = 32;            // columns per block-reflector CTA
constexpr int CH = 64;            // rows per staged chunk in the block-reflector CTA
constexpr size_t kPanelSmemMax = 220 * 1024;

// A matrix whose logical rows are two segments, derived per panel start column c0.
//   kind 0 (leaf):     rows c0..m-1 of `a` (m = a_rows0);       segment b empty.
//   kind 1 (combine):  rows c0..c0+NB-1 of `a` (the top R);     then rows 0..c0+NB-1 of `b`.
template <typename T>
struct Prob {
  T *a;
  T *b;
  int64_t lda, ldb;
  int a_rows0;     // leaf height m (kind 0)
  int kind;
  int slot;        // index into tau / T arrays
};

template <typename T>
struct SegView {
  T *a, *b;
  int64_t lda, ldb;
  int na, nb_rows;
  __device__ __forceinline__ int rows() const { return na + nb_rows; }
  __device__ __forceinline__ T &at(int r, int c) const {
    return (r < na) ? a[r + (int64_t)c * lda] : b[(r - na) + (int64_t)c * ldb];
  }
};

template <typename T>
__device__ __forceinline__ SegView<T> view(const Prob<T> &p, int c0) {
  SegView<T> v;
  v.lda = p.lda;
  v.ldb = p.ldb;
  if (p.kind == 0) {
    v.a = p.a + c0;
    v.na = p.a_rows0 - c0;
    v.b = p.b;
    v.nb_rows = 0;
  } else {
    v.a = p.a + c0;
    v.na = NB;
    v.b = p.b;
    v.nb_rows = c0 + NB;
  }
  return v;
}

// Reduce NV per-thread values over the whole CTA; result in out[0..NV).
template <typename T, int NV, int NT>
__device__ __forceinline__ void block_sum(T (&vals)[NV], T *red, T *out) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int v = 0; v < NV; ++v) {
    T x = vals[v];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
    vals[v] = x;
  }
  if (lane == 0) {
#pragma unroll
    for (int v = 0; v < NV; ++v) red[warp * NV + v] = vals[v];
  }
  __syncthreads();
  if (threadIdx.x < NV) {
    T s = 0;
    for (int w = 0; w < NT / 32; ++w) s += red[w * NV + threadIdx.x];
    out[threadIdx.x] = s;
  }
  __syncthreads();
}

// --------------------------------------------------------------------------- panel
// Householder QR of the h x NB panel at columns c0..c0+NB-1 (one CTA per problem).
// Writes R (upper part) and V (below the diagonal, unit diagonal implicit) in place,
// tau[slot][c0..c0+NB-1] and the compact-WY factor Tm[slot][panel] (NB x NB, upper).
template <typename T>
__global__ void __launch_bounds__(PF_THREADS) k_panel(const Prob<T> *probs, int c0, int d,
                                                      T *tau_all, T *T_all, int npanels) {
  extern __shared__ __align__(16) uint8_t sm_raw[];
  const Prob<T> pr = probs[blockIdx.x];
  const SegView<T> M = view(pr, c0);
  const int h = M.rows();
  const int hp = h | 1;   // odd pitch: fewer bank conflicts
  T *Ps = reinterpret_cast<T *>(sm_raw);                  // NB x hp
  T *red = Ps + NB * hp;                                  // 16 warps x NB
  T *sums = red + (PF_THREADS / 32) * NB;                 // NB
  T *wv = sums + NB;                                      // NB
  T *Ts = wv + NB;                                        // NB x NB
  T *scal = Ts + NB * NB;                                 // [tau, rdiag, head]
  const int tid = threadIdx.x;

  for (int c = 0; c < NB; ++c)
    for (int r = tid; r < h; r += PF_THREADS) Ps[c * hp + r] = M.at(r, c0 + c);
  for (int e = tid; e < NB * NB; e += PF_THREADS) Ts[e] = 0;
  __syncthreads();

  for (int jj = 0; jj < NB; ++jj) {
    T *x = Ps + jj * hp;
    // 1. norm of the part below the diagonal
    T part[1] = {0};
    for (int r = jj + 1 + tid; r < h; r += PF_THREADS) part[0] += x[r] * x[r];
    block_sum<T, 1, PF_THREADS>(part, red, sums);
    if (tid == 0) {
      T alpha = x[jj];
      T sig = sums[0];
      T normx = sqrt(alpha * alpha + sig);
      T tau = 0, rd = 0, head = 1;
      if (normx > 0) {
        T s = alpha >= 0 ? T(1) : T(-1);
        head = alpha + s * normx;
        tau = T(2) / (T(1) + sig / (head * head));
        rd = -s * normx;
      }
      scal[0] = tau;
      scal[1] = rd;
      scal[2] = head;
    }
    __syncthreads();
    const T tau = scal[0], head = scal[2];
    for (int r = jj + 1 + tid; r < h; r += PF_THREADS) x[r] = x[r] / head;
    __syncthreads();
    if (tid == 0) x[jj] = scal[1];
    // 2. dots of v with every other panel column (rows > jj)
    T dots[NB];
#pragma unroll
    for (int c = 0; c < NB; ++c) dots[c] = 0;
    for (int r = jj + 1 + tid; r < h; r += PF_THREADS) {
      T vr = x[r];
#pragma unroll
      for (int c = 0; c < NB; ++c) dots[c] += (c == jj) ? T(0) : Ps[c * hp + r] * vr;
    }
    block_sum<T, NB, PF_THREADS>(dots, red, sums);
    // 3. w_c = row-jj entry + dot (c > jj);  g_i (i < jj) for the T column
    if (tid < NB) {
      int c = tid;
      if (c != jj) wv[c] = Ps[c * hp + jj] + sums[c];
    }
    __syncthreads();
    // 4. apply the reflector to the trailing panel columns
    for (int c = jj + 1; c < NB; ++c) {
      T w = tau * wv[c];
      T *col = Ps + c * hp;
      for (int r = jj + 1 + tid; r < h; r += PF_THREADS) col[r] -= w * x[r];
      if (tid == 0) col[jj] -= w;
    }
    // 5. T column jj: T[jj][jj] = tau, T[0:jj, jj] = -tau T[0:jj,0:jj] g
    if (tid < jj) {
      int i = tid;
      T acc = 0;
      for (int l = i; l < jj; ++l) acc += Ts[i * NB + l] * wv[l];
      Ts[i * NB + jj] = -tau * acc;
    }
    if (tid == 0) Ts[jj * NB + jj] = tau;
    if (tid == 0) tau_all[(int64_t)pr.slot * d + c0 + jj] = tau;
    __syncthreads();
  }
  for (int c = 0; c < NB; ++c)
    for (int r = tid; r < h; r += PF_THREADS) M.at(r, c0 + c) = Ps[c * hp + r];
  T *Tout = T_all + ((int64_t)pr.slot * npanels + c0 / NB) * NB * NB;
  for (int e = tid; e < NB * NB; e += PF_THREADS) Tout[e] = Ts[e];
}

// --------------------------------------------------------------------------- reflector
// C <- (I - V T V^T) C  (trans = 0)  or  (I - V T^T V^T) C  (trans = 1) on columns
// [cbeg + TW*blockIdx.y, ...) < cend of problem blockIdx.x.  V is the panel at c0 of
// vprobs (unit diagonal implicit, zeros above), C has the same logical rows in cprobs.
template <typename T>
__global__ void __launch_bounds__(BR_THREADS) k_reflect(const Prob<T> *vprobs, const Prob<T> *cprobs,
                                                        int c0, int cbeg, int cend, int d,
                                                        const T *T_all, int npanels, int trans) {
  extern __shared__ __align__(16) uint8_t br_raw[];
  T (*Vs)[NB + 1] = reinterpret_cast<T (*)[NB + 1]>(br_raw);
  T (*Cs)[CH + 1] = reinterpret_cast<T (*)[CH + 1]>(br_raw + sizeof(T) * CH * (NB + 1));
  T (*Wp)[NB][TW] = reinterpret_cast<T (*)[NB][TW]>(br_raw + sizeof(T) * (CH * (NB + 1) + TW * (CH + 1)));
  T (*Wf)[TW] = reinterpret_cast<T (*)[TW]>(br_raw + sizeof(T) * (CH * (NB + 1) + TW * (CH + 1) + 8 * NB * TW));
  T (*Tm)[NB] = reinterpret_cast<T (*)[NB]>(br_raw + sizeof(T) * (CH * (NB + 1) + TW * (CH + 1) + 9 * NB * TW));
  const int col0 = cbeg + TW * blockIdx.y;
  if (col0 >= cend) return;
  const int ncols = min(TW, cend - col0);
  const Prob<T> pv = vprobs[blockIdx.x];
  const SegView<T> V = view(pv, c0);
  const SegView<T> C = view(cprobs[blockIdx.x], c0);
  const int h = V.rows();
  const int tid = threadIdx.x;
  const T *Tsrc = T_all + ((int64_t)pv.slot * npanels + c0 / NB) * NB * NB;
  for (int e = tid; e < NB * NB; e += BR_THREADS) Tm[e / NB][e % NB] = Tsrc[e];

  // ---- W = V^T C
  const int jj = tid & 31, rg = tid >> 5;
  T acc[NB];
#pragma unroll
  for (int i = 0; i < NB; ++i) acc[i] = 0;
  for (int r0 = 0; r0 < h; r0 += CH) {
    __syncthreads();
    for (int e = tid; e < CH * NB; e += BR_THREADS) {
      int i = e / CH, rl = e % CH, r = r0 + rl;
      T v = 0;
      if (r < h) v = (r == i) ? T(1) : (r > i ? V.at(r, c0 + i) : T(0));
      Vs[rl][i] = v;
    }
    for (int e = tid; e < CH * TW; e += BR_THREADS) {
      int c = e / CH, rl = e % CH, r = r0 + rl;
      Cs[c][rl] = (r < h && c < ncols) ? C.at(r, col0 + c) : T(0);
    }
    __syncthreads();
    for (int rl = rg; rl < CH; rl += 8) {
      T cv = Cs[jj][rl];
#pragma unroll
      for (int i = 0; i < NB; ++i) acc[i] += Vs[rl][i] * cv;
    }
  }
#pragma unroll
  for (int i = 0; i < NB; ++i) Wp[rg][i][jj] = acc[i];
  __syncthreads();
  for (int e = tid; e < NB * TW; e += BR_THREADS) {
    int i = e / TW, c = e % TW;
    T s = 0;
#pragma unroll
    for (int g = 0; g < 8; ++g) s += Wp[g][i][c];
    Wf[i][c] = s;
  }
  __syncthreads();
  // ---- W' = T W  or  T^T W   (into Wp[0])
  for (int e = tid; e < NB * TW; e += BR_THREADS) {
    int i = e / TW, c = e % TW;
    T s = 0;
    if (!trans) {
      for (int l = i; l < NB; ++l) s += Tm[i][l] * Wf[l][c];
    } else {
      for (int l = 0; l <= i; ++l) s += Tm[l][i] * Wf[l][c];
    }
    Wp[0][i][c] = s;
  }
  __syncthreads();
  // ---- C -= V W'
  const int rl_t = tid & 63, cgp = tid >> 6;   // 4 groups of 8 columns
  for (int r0 = 0; r0 < h; r0 += CH) {
    int r = r0 + rl_t;
    if (r >= h) continue;
    T vrow[NB];
#pragma unroll
    for (int i = 0; i < NB; ++i) vrow[i] = (r == i) ? T(1) : (r > i ? V.at(r, c0 + i) : T(0));
#pragma unroll
    for (int k = 0; k < TW / 4; ++k) {
      int c = cgp * (TW / 4) + k;
      if (c >= ncols) break;
      T s = 0;
#pragma unroll
      for (int i = 0; i < NB; ++i) s += vrow[i] * Wp[0][i][c];
      C.at(r, col0 + c) -= s;
    }
  }
}

// --------------------------------------------------------------------------- helpers
// Copy the upper triangle of a leaf's R (rows 0..d-1 of the leaf in Y) into a d x d slot
// (zero below the diagonal), converting precision.
template <typename S, typename T>
__global__ void k_copy_leaf_r(const S *Y, int64_t ldy, const int64_t *leaf_row0, int d,
                              T *slots) {
  int slot = blockIdx.y;
  const S *src = Y + leaf_row0[slot];
  T *dst = slots + (int64_t)slot * d * d;
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < d * d; e += gridDim.x * blockDim.x) {
    int r = e % d, c = e / d;
    dst[e] = (r <= c) ? (T)src[r + (int64_t)c * ldy] : T(0);
  }
}

template <typename S, typename D>
__global__ void k_convert_slots(const S *src, D *dst, const int *slots, int d) {
  int slot = slots[blockIdx.y];
  const S *s = src + (int64_t)slot * d * d;
  D *t = dst + (int64_t)slot * d * d;
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < d * d; e += gridDim.x * blockDim.x)
    t[e] = (D)s[e];
}

template <typename T>
__global__ void k_zero_slots(T *dst, const int *slots, int d) {
  int slot = slots[blockIdx.y];
  T *t = dst + (int64_t)slot * d * d;
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < d * d; e += gridDim.x * blockDim.x) t[e] = 0;
}

// R_out = D R_root (D = sign(diag R_root), 0 -> +1); X_root = D.
template <typename T>
__global__ void k_finish_root(const T *Rroot, int d, double *Rout, T *Xroot) {
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < d * d; e += gridDim.x * blockDim.x) {
    int r = e % d, c = e / d;
    double s = ((double)Rroot[r + (int64_t)r * d] < 0.0) ? -1.0 : 1.0;
    Rout[e] = (r <= c) ? s * (double)Rroot[e] : 0.0;
    Xroot[e] = (r == c) ? (T)s : T(0);
  }
}

// Leaf block of Q_hat before the leaf reflectors: rows 0..d-1 = X_slot, rest 0.
template <typename T>
__global__ void k_init_leaf_q(T *Q, int64_t ldq, const int64_t *leaf_row0, const int *leaf_rows,
                              const T *X, int d) {
  int leaf = blockIdx.y;
  int64_t row0 = leaf_row0[leaf];
  int m = leaf_rows[leaf];
  const T *x = X + (int64_t)leaf * d * d;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < (int64_t)m * d;
       e += (int64_t)gridDim.x * blockDim.x) {
    int r = (int)(e % m), c = (int)(e / m);
    Q[row0 + r + (int64_t)c * ldq] = (r < d) ? x[r + (int64_t)c * d] : T(0);
  }
}

// Column-major copy with conversion (n x d, ld -> ld2).
template <typename S, typename D>
__global__ void k_convert_matrix(int64_t n, int d, const S *src, int64_t lds, D *dst, int64_t ldd) {
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < n * d;
       e += (int64_t)gridDim.x * blockDim.x) {
    int64_t r = e % n, c = e / n;
    dst[r + c * ldd] = (D)src[r + c * lds];
  }
}

template <typename T>
size_t panel_smem(int hmax) {
  int hp = hmax | 1;
  return sizeof(T) * ((size_t)NB * hp + (PF_THREADS / 32) * NB + NB + NB + NB * NB + 4);
}

template <typename T>
Error run_panel(const Prob<T> *probs, int nprob, int c0, int d, int hmax, T *tau, T *Tm,
                int npanels, cudaStream_t st) {
  size_t smem = panel_smem<T>(hmax);
  CK_CUDA(cudaFuncSetAttribute(k_panel<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  ::ckinv::note_launch(), k_panel<T><<<nprob, PF_THREADS, smem, st>>>(probs, c0, d, tau, Tm, npanels);
  CK_CUDA(cudaGetLastError());
  return ok();
}

template <typename T>
Error run_reflect(const Prob<T> *vp, const Prob<T> *cp, int nprob, int c0, int cbeg, int cend, int d,
                  const T *Tm, int npanels, int trans, cudaStream_t st) {
  if (cend <= cbeg) return ok();
  dim3 grid(nprob, (unsigned)ceil_div(cend - cbeg, TW));
  const size_t smem = sizeof(T) * (CH * (NB + 1) + TW * (CH + 1) + 9 * NB * TW + NB * NB);
  CK_CUDA(cudaFuncSetAttribute(k_reflect<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  ::ckinv::note_launch(), k_reflect<T><<<grid, BR_THREADS, smem, st>>>(vp, cp, c0, cbeg, cend, d, Tm, npanels, trans);
  CK_CUDA(cudaGetLastError());
  return ok();
}

struct Level {
  std::vector<int> top, bot;   // combines (top slot, bottom slot)
  bool fp64;
};

}  // namespace

// Tallest leaf whose NB-column panel fits in shared memory; a leaf may hold up to
// b + d - 1 rows after the short tail is merged, so b is capped at that minus d.
int max_block_rows(int d, bool leaf_fp64) {
  int h = 16;
  while ((leaf_fp64 ? panel_smem<double>(h + 16) : panel_smem<float>(h + 16)) <= kPanelSmemMax) h += 16;
  int b = h - d;
  return std::max(b, 0) / 16 * 16;
}

int auto_block_rows(int64_t n, int d, int sm_count) {
  (void)sm_count;
  int64_t b = 2048;
  if (n < 2 * b) b = std::max<int64_t>(d, (n + 1) / 2);
  if (b < d) b = d;
  return (int)b;
}

namespace {

template <typename TL>
Error tsqr_impl(ckinv_ctx *ctx, int64_t n, int d, int b, int fp64_levels, TL *Y, int64_t ldy, TL *Qout,
                int64_t ldq, double *Rout, cudaStream_t st) {
  constexpr bool LEAF64 = sizeof(TL) == 8;
  // ---- leaves
  std::vector<int64_t> row0;
  std::vector<int> rows;
  for (int64_t s = 0; s < n; s += b) {
    row0.push_back(s);
    rows.push_back((int)std::min<int64_t>(b, n - s));
  }
  if (rows.size() > 1 && rows.back() < d) {
    int last = rows.back();
    rows.pop_back();
    row0.pop_back();
    rows.back() += last;
  }
  const int L = (int)rows.size();
  int hmax = 0;
  for (int m : rows) hmax = std::max(hmax, m);
  if (panel_smem<TL>(hmax) > kPanelSmemMax)
    return fail(CKINV_EUNSUPPORTED, "tsqr: leaf height too large for the shared-memory panel");
  const int P = d / NB;
  // ---- tree levels
  std::vector<Level> levels;
  {
    std::vector<int> active(L);
    for (int i = 0; i < L; ++i) active[i] = i;
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
  const int H = (int)levels.size();
  int nf64 = (fp64_levels < 0) ? H : std::min(fp64_levels, H);
  if (LEAF64) nf64 = H;   // an FP64 leaf stage feeds an all-FP64 tree
  for (int l = 0; l < H; ++l) levels[l].fp64 = (l >= H - nf64);
  const bool first64 = (H == 0) ? true : levels[0].fp64;
  const bool root64 = (H == 0) ? true : levels[H - 1].fp64;

  // ---- device workspace (stream-ordered)
  const size_t slot = (size_t)d * d;
  float *Rf = nullptr, *tauf = nullptr, *Tf = nullptr, *Xf = nullptr;
  double *Rd = nullptr, *taud = nullptr, *Td = nullptr, *Xd = nullptr;
  TL *tauL = nullptr, *TLm = nullptr;
  int64_t *d_row0 = nullptr;
  int *d_rows = nullptr, *d_slots = nullptr;
  Prob<TL> *d_pl = nullptr;
  Prob<float> *d_pf = nullptr;
  Prob<double> *d_pd = nullptr;
  const bool need_f = !(LEAF64) && (nf64 < H || H == 0 || !first64);
  CK_CUDA(cudaMallocAsync((void **)&tauL, sizeof(TL) * d * L, st));
  CK_CUDA(cudaMallocAsync((void **)&TLm, sizeof(TL) * NB * NB * P * L, st));
  if (need_f || !LEAF64) {
    CK_CUDA(cudaMallocAsync((void **)&Rf, sizeof(float) * slot * L, st));
    CK_CUDA(cudaMallocAsync((void **)&Xf, sizeof(float) * slot * L, st));
    CK_CUDA(cudaMallocAsync((void **)&tauf, sizeof(float) * d * L, st));
    CK_CUDA(cudaMallocAsync((void **)&Tf, sizeof(float) * NB * NB * P * L, st));
  }
  if (nf64 > 0 || H == 0) {
    CK_CUDA(cudaMallocAsync((void **)&Rd, sizeof(double) * slot * L, st));
    CK_CUDA(cudaMallocAsync((void **)&Xd, sizeof(double) * slot * L, st));
    CK_CUDA(cudaMallocAsync((void **)&taud, sizeof(double) * d * L, st));
    CK_CUDA(cudaMallocAsync((void **)&Td, sizeof(double) * NB * NB * P * L, st));
  }
  // host-side descriptor tables: leaves (V = Y, C = Y) then (V = Y, C = Q); per level
  std::vector<Prob<TL>> hpl;
  for (int i = 0; i < L; ++i) hpl.push_back(Prob<TL>{Y + row0[i], nullptr, ldy, 0, rows[i], 0, i});
  for (int i = 0; i < L; ++i) hpl.push_back(Prob<TL>{Qout + row0[i], nullptr, ldq, 0, rows[i], 0, i});
  std::vector<Prob<float>> hpf;
  std::vector<Prob<double>> hpd;
  std::vector<size_t> lvl_off(H), lvl_xoff(H);
  for (int l = 0; l < H; ++l) {
    const Level &lv = levels[l];
    int nc = (int)lv.top.size();
    if (!lv.fp64) {
      lvl_off[l] = hpf.size();
      for (int c = 0; c < nc; ++c)
        hpf.push_back(Prob<float>{Rf + slot * lv.top[c], Rf + slot * lv.bot[c], d, d, d, 1, lv.bot[c]});
      lvl_xoff[l] = hpf.size();
      for (int c = 0; c < nc; ++c)
        hpf.push_back(Prob<float>{Xf + slot * lv.top[c], Xf + slot * lv.bot[c], d, d, d, 1, lv.bot[c]});
    } else {
      lvl_off[l] = hpd.size();
      for (int c = 0; c < nc; ++c)
        hpd.push_back(Prob<double>{Rd + slot * lv.top[c], Rd + slot * lv.bot[c], d, d, d, 1, lv.bot[c]});
      lvl_xoff[l] = hpd.size();
      for (int c = 0; c < nc; ++c)
        hpd.push_back(Prob<double>{Xd + slot * lv.top[c], Xd + slot * lv.bot[c], d, d, d, 1, lv.bot[c]});
    }
  }
  std::vector<int> hslots;
  std::vector<size_t> lvl_bslots(H);
  for (int l = 0; l < H; ++l) {
    lvl_bslots[l] = hslots.size();
    for (int s : levels[l].bot) hslots.push_back(s);
  }
  const size_t all_slots_off = hslots.size();
  for (int i = 0; i < L; ++i) hslots.push_back(i);
  CK_CUDA(cudaMallocAsync((void **)&d_row0, sizeof(int64_t) * L, st));
  CK_CUDA(cudaMallocAsync((void **)&d_rows, sizeof(int) * L, st));
  CK_CUDA(cudaMallocAsync((void **)&d_slots, sizeof(int) * hslots.size(), st));
  CK_CUDA(cudaMallocAsync((void **)&d_pl, sizeof(Prob<TL>) * hpl.size(), st));
  if (!hpf.empty()) CK_CUDA(cudaMallocAsync((void **)&d_pf, sizeof(Prob<float>) * hpf.size(), st));
  if (!hpd.empty()) CK_CUDA(cudaMallocAsync((void **)&d_pd, sizeof(Prob<double>) * hpd.size(), st));
  CK_TRY(stage_upload(ctx, row0.data(), sizeof(int64_t) * L, d_row0, st));
  CK_TRY(stage_upload(ctx, rows.data(), sizeof(int) * L, d_rows, st));
  CK_TRY(stage_upload(ctx, hslots.data(), sizeof(int) * hslots.size(), d_slots, st));
  CK_TRY(stage_upload(ctx, hpl.data(), sizeof(Prob<TL>) * hpl.size(), d_pl, st));
  if (!hpf.empty()) CK_TRY(stage_upload(ctx, hpf.data(), sizeof(Prob<float>) * hpf.size(), d_pf, st));
  if (!hpd.empty()) CK_TRY(stage_upload(ctx, hpd.data(), sizeof(Prob<double>) * hpd.size(), d_pd, st));

  // ---- 1. leaves
  for (int p = 0; p < P; ++p) {
    int c0 = p * NB;
    CK_TRY(run_panel<TL>(d_pl, L, c0, d, hmax, tauL, TLm, P, st));
    CK_TRY(run_reflect<TL>(d_pl, d_pl, L, c0, c0 + NB, d, d, TLm, P, 1, st));
  }
  // ---- 2. leaf R's into the tree slots
  {
    dim3 g((unsigned)std::min<int64_t>(ceil_div(slot, 256), 64), L);
    if (first64) ::ckinv::note_launch(), k_copy_leaf_r<TL, double><<<g, 256, 0, st>>>(Y, ldy, d_row0, d, Rd);
    else ::ckinv::note_launch(), k_copy_leaf_r<TL, float><<<g, 256, 0, st>>>(Y, ldy, d_row0, d, Rf);
    CK_CUDA(cudaGetLastError());
  }
  // ---- 3. tree, bottom-up
  for (int l = 0; l < H; ++l) {
    const Level &lv = levels[l];
    int nc = (int)lv.top.size();
    if (l > 0 && lv.fp64 && !levels[l - 1].fp64) {
      dim3 g((unsigned)std::min<int64_t>(ceil_div(slot, 256), 64), L);
      ::ckinv::note_launch(), k_convert_slots<float, double><<<g, 256, 0, st>>>(Rf, Rd, d_slots + all_slots_off, d);
      CK_CUDA(cudaGetLastError());
    }
    for (int p = 0; p < P; ++p) {
      int c0 = p * NB;
      if (lv.fp64) {
        CK_TRY(run_panel<double>(d_pd + lvl_off[l], nc, c0, d, d + NB, taud, Td, P, st));
        CK_TRY(run_reflect<double>(d_pd + lvl_off[l], d_pd + lvl_off[l], nc, c0, c0 + NB, d, d, Td, P, 1, st));
      } else {
        CK_TRY(run_panel<float>(d_pf + lvl_off[l], nc, c0, d, d + NB, tauf, Tf, P, st));
        CK_TRY(run_reflect<float>(d_pf + lvl_off[l], d_pf + lvl_off[l], nc, c0, c0 + NB, d, d, Tf, P, 1, st));
      }
    }
  }
  // ---- 4. root: R = D R_root, X_root = D
  {
    int g = (int)std::min<int64_t>(ceil_div(slot, 256), 256);
    if (root64) ::ckinv::note_launch(), k_finish_root<double><<<g, 256, 0, st>>>(Rd, d, Rout, Xd);
    else ::ckinv::note_launch(), k_finish_root<float><<<g, 256, 0, st>>>(Rf, d, Rout, Xf);
    CK_CUDA(cudaGetLastError());
  }
  // ---- 5. push X down the tree
  for (int l = H - 1; l >= 0; --l) {
    const Level &lv = levels[l];
    int nc = (int)lv.top.size();
    dim3 gz((unsigned)std::min<int64_t>(ceil_div(slot, 256), 64), nc);
    if (lv.fp64) ::ckinv::note_launch(), k_zero_slots<double><<<gz, 256, 0, st>>>(Xd, d_slots + lvl_bslots[l], d);
    else ::ckinv::note_launch(), k_zero_slots<float><<<gz, 256, 0, st>>>(Xf, d_slots + lvl_bslots[l], d);
    CK_CUDA(cudaGetLastError());
    for (int p = P - 1; p >= 0; --p) {
      int c0 = p * NB;
      if (lv.fp64)
        CK_TRY(run_reflect<double>(d_pd + lvl_off[l], d_pd + lvl_xoff[l], nc, c0, 0, d, d, Td, P, 0, st));
      else
        CK_TRY(run_reflect<float>(d_pf + lvl_off[l], d_pf + lvl_xoff[l], nc, c0, 0, d, d, Tf, P, 0, st));
    }
    if (l > 0 && lv.fp64 && !levels[l - 1].fp64) {
      dim3 g((unsigned)std::min<int64_t>(ceil_div(slot, 256), 64), L);
      ::ckinv::note_launch(), k_convert_slots<double, float><<<g, 256, 0, st>>>(Xd, Xf, d_slots + all_slots_off, d);
      CK_CUDA(cudaGetLastError());
    }
  }
  TL *XL = nullptr;
  if (LEAF64) {
    XL = reinterpret_cast<TL *>(Xd);
  } else {
    if (first64) {
      dim3 g((unsigned)std::min<int64_t>(ceil_div(slot, 256), 64), L);
      ::ckinv::note_launch(), k_convert_slots<double, float><<<g, 256, 0, st>>>(Xd, Xf, d_slots + all_slots_off, d);
      CK_CUDA(cudaGetLastError());
    }
    XL = reinterpret_cast<TL *>(Xf);
  }
  // ---- 6. leaves: Q_hat block = Q_leaf [X; 0]
  {
    dim3 g(64, L);
    ::ckinv::note_launch(), k_init_leaf_q<TL><<<g, 256, 0, st>>>(Qout, ldq, d_row0, d_rows, XL, d);
    CK_CUDA(cudaGetLastError());
  }
  for (int p = P - 1; p >= 0; --p) {
    int c0 = p * NB;
    CK_TRY(run_reflect<TL>(d_pl, d_pl + L, L, c0, 0, d, d, TLm, P, 0, st));
  }
  for (void *ptr : {(void *)Rf, (void *)Xf, (void *)tauf, (void *)Tf, (void *)tauL, (void *)TLm, (void *)Rd,
                    (void *)Xd, (void *)taud, (void *)Td, (void *)d_row0, (void *)d_rows, (void *)d_slots,
                    (void *)d_pl, (void *)d_pf, (void *)d_pd})
    if (ptr) CK_CUDA(cudaFreeAsync(ptr, st));
  return ok();
}

}  // namespace

Error tsqr_factor(ckinv_ctx *ctx, int64_t n, int d, int b, int fp64_levels, bool leaf_fp64, float *Y,
                  int64_t ldy, float *Qout, double *Rout, cudaStream_t st) {
  if (d % NB != 0) return fail(CKINV_EINVAL, "tsqr: d must be a multiple of 16");
  const int bmax = max_block_rows(d, leaf_fp64);
  if (bmax < d) return fail(CKINV_EUNSUPPORTED, "tsqr: d too large for a shared-memory panel");
  if (b > bmax) b = bmax;   // R and Q_hat do not depend on the leaf height
  if (!leaf_fp64) return tsqr_impl<float>(ctx, n, d, b, fp64_levels, Y, ldy, Qout, n, Rout, st);
  double *Y64 = nullptr, *Q64 = nullptr;
  CK_CUDA(cudaMallocAsync((void **)&Y64, sizeof(double) * n * d, st));
  CK_CUDA(cudaMallocAsync((void **)&Q64, sizeof(double) * n * d, st));
  unsigned g = (unsigned)std::min<int64_t>(ceil_div(n * d, 256), 65535);
  ::ckinv::note_launch(), k_convert_matrix<float, double><<<g, 256, 0, st>>>(n, d, Y, ldy, Y64, n);
  CK_CUDA(cudaGetLastError());
  Error e = tsqr_impl<double>(ctx, n, d, b, -1, Y64, n, Q64, n, Rout, st);
  if (e.st == CKINV_OK) {
    ::ckinv::note_launch(), k_convert_matrix<double, float><<<g, 256, 0, st>>>(n, d, Q64, n, Qout, n);
    cudaError_t c = cudaGetLastError();
    if (c != cudaSuccess) e = fail(CKINV_ECUDA, cudaGetErrorString(c));
  }
  cudaFreeAsync(Y64, st);
  cudaFreeAsync(Q64, st);
  return e;
}

}  // namespace ckinv
