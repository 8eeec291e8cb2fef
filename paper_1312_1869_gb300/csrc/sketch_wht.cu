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
// A warp owns two rows and evaluates them together, so that each point read from shared memory
// serves both.  Each lane owns up to 16 output slots; a small set-up kernel assigns the d
// outputs to the (slot, lane) grid so that the 32 lanes of one gather read 32 different banks
// (lane = bank of the output's U[p_b]), which makes the gather conflict-free.  A CTA of 4 warps
// owns 8 rows, three CTAs share an SM (12 warps of 167 registers), and each streams the
// pre-scaled points of every chunk, with each lane's sign masks for it (precomputed by a
// set-up kernel, one word each), into shared memory with asynchronous copies, the next chunk's
// in flight while the current one is transformed; at the end the 8 x d block of Y goes out
// through shared memory, each column's rows contiguous.
#include "internal.cuh"

namespace ckinv {
namespace {

constexpr int kWB = 1024;             // transform length (chunk of points)
constexpr int kPfAhead = 2;           // materialised K0: chunks prefetched into L2 ahead of the one in work
constexpr int kWMaxU = 16;            // output slots per lane: d <= 512
constexpr int kWPad = 33;             // padded row of the transpose buffers

// The points past n (the padding of K0 to order N) have zero kernel entries.  For the
// squared-exponential kernel they are placed at +infinity in every coordinate: their squared
// distance to any finite point is +infinity, whose exp2(-inf) is exactly 0, so the hot loop
// needs no mask.  The derivative's factor r^2 would make that inf * 0, so its scaled squared
// distance is first clamped at 1e4, which changes no entry (exp2(-x) is exactly 0 in FP32 for
// every x above ~150).  Matern-5/2, whose polynomial in r would overflow the same way at any
// clamp that is exact for every lengthscale, masks the last chunk's entries instead.
constexpr float kPadFar = __builtin_huge_valf();
constexpr float kSeClamp = 1e4f;
__host__ __device__ constexpr bool pad_far(int kind, bool) { return kind == CKINV_SE; }

// Shared memory of one CTA.  The transpose buffers double, after the last chunk, as the
// d x ROWS staging tile of the output (column stride ROWS + 1).  A materialised K0 (PTS
// false) stages no points.
template <int WARPS, int NB, int ROWS, bool PTS = true>
struct WhtSmem {
  float sp[2][PTS ? kWB * 3 : 4];        // the chunk's points (pre-scaled), two buffers
  uint32_t ssg[2][32];                   // lane l: bit t = sign bit of entry l + 32 t of the chunk
  uint32_t sgs[2][32];                   // lane l: bit u = gather sign of its slot u for the chunk
  static constexpr int kTPad = ROWS + 1;                 // staging tile: row stride of column j
  static constexpr int kBufFloats =
      WARPS * NB * 32 * kWPad > 32 * kWMaxU * kTPad ? WARPS * NB * 32 * kWPad : 32 * kWMaxU * kTPad;
  float buf[kBufFloats];                 // per warp NB transpose buffers of 32 x 33
  uint32_t gtab[32 * kWMaxU];            // slot: address of U[p_b] in a buffer | p_a << 11
  int jtab[32 * kWMaxU];                 // slot: output column j, or -1
};

__device__ __forceinline__ uint32_t smem_u32(const void *p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}
__device__ __forceinline__ void cp_async16(void *dst, const void *src) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(smem_u32(dst)), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
__device__ __forceinline__ void prefetch_l2(const void *p) { asm volatile("prefetch.global.L2 [%0];" ::"l"(p)); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_group 0;\n" ::: "memory"); }

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

// Each row's v (lane l, register t = entry l + 32 t) -> H_1024 v, left in that row's buffer as
// w[s * 33 + q] = U[32 s + q]: five stages over t, transpose, five stages over the former lane
// bits, one row after the other (interleaving the rows measured slower).  A lane reads back,
// and then overwrites, only its own row of the buffer, so the second half needs no barrier;
// the caller synchronises the warp before the gather.
template <int NR>
__device__ __forceinline__ void wht1024_rows(float (&v)[NR][32], float *w, int lane) {
  __syncwarp();                                      // the previous gather from w is done
#pragma unroll
  for (int r = 0; r < NR; ++r) {
    float *wr = w + r * 32 * kWPad;
    wht32(v[r]);
#pragma unroll
    for (int t = 0; t < 32; ++t) wr[t * kWPad + lane] = v[r][t];
    __syncwarp();
#pragma unroll
    for (int t = 0; t < 32; ++t) v[r][t] = wr[lane * kWPad + t];
    wht32(v[r]);
#pragma unroll
    for (int t = 0; t < 32; ++t) wr[lane * kWPad + t] = v[r][t];
  }
}

// x with its sign flipped iff bit b of m is 1 (no branch)
__device__ __forceinline__ float flip_if(float x, uint32_t m, int b) {
  return __uint_as_float(__float_as_uint(x) ^ ((m << (31 - b)) & 0x80000000u));
}

// The kernel entries of NR rows (coordinates x, pre-scaled) against the 32 points
// k_b = lane + 32 t of the chunk, Rademacher signs applied; each point read serves all NR
// rows.  With TAIL, entries at or past the end of the points (the zero padding of K0 to
// order N) are zero.
template <bool DERIV, int KIND, bool TAIL, int NR>
__device__ __forceinline__ void eval_rows(const float *P, int dim, const float (&x)[NR][3], float inv_l,
                                          uint32_t smask, int lane, int rem, float (&v)[NR][32]) {
#pragma unroll
  for (int t = 0; t < 32; ++t) {
    const int kb = lane + 32 * t;
    float q0, q1, q2;
    if (dim == 2) {
      const float2 q = reinterpret_cast<const float2 *>(P)[kb];
      q0 = q.x;
      q1 = q.y;
      q2 = 0.f;
    } else {
      q0 = P[dim * kb];
      q1 = dim > 1 ? P[dim * kb + 1] : 0.f;
      q2 = dim > 2 ? P[dim * kb + 2] : 0.f;
    }
#pragma unroll
    for (int r = 0; r < NR; ++r) {
      const float dx = x[r][0] - q0, dy = x[r][1] - q1;
      float r2 = fmaf(dy, dy, dx * dx);
      if (dim > 2) {
        const float dz = x[r][2] - q2;
        r2 = fmaf(dz, dz, r2);
      }
      if (DERIV && KIND == CKINV_SE) r2 = fminf(r2, kSeClamp);
      float e = dev::kernel_value(KIND, r2, inv_l, DERIV);
      if (TAIL) e = kb < rem ? e : 0.f;
      v[r][t] = flip_if(e, smask, t);
    }
  }
}

// A materialised K0: the entries of NR rows against the 32 points k_b = lane + 32 t of the
// chunk, read from HBM (row i of the symmetric K0 is its column i, contiguous, so a warp's
// loads are 128-byte lines; streamed, each entry is read once), Rademacher signs applied;
// with TAIL, entries at or past n are zero.
template <bool TAIL, int NR>
__device__ __forceinline__ void load_rows(const float *const (&kc)[NR], int64_t k0, uint32_t smask, int lane, int rem,
                                          float (&v)[NR][32]) {
#pragma unroll
  for (int t = 0; t < 32; ++t) {
    const int kb = lane + 32 * t;
#pragma unroll
    for (int r = 0; r < NR; ++r) {
      const float e = (!TAIL || kb < rem) ? __ldcs(kc[r] + k0 + kb) : 0.f;
      v[r][t] = flip_if(e, smask, t);
    }
  }
}

// rows (0, 1, ..., R-1) -> (S, S+1, ..., S-1) of the accumulators and coordinates
template <int R, int S>
__device__ __forceinline__ void rotate_rows(float (&acc)[R][kWMaxU], float (&xr)[R][3]) {
  if constexpr (S % R != 0) {
    float ta[R][kWMaxU], tx[R][3];
#pragma unroll
    for (int r = 0; r < R; ++r) {
#pragma unroll
      for (int u = 0; u < kWMaxU; ++u) ta[r][u] = acc[(r + S) % R][u];
#pragma unroll
      for (int c = 0; c < 3; ++c) tx[r][c] = xr[(r + S) % R][c];
    }
#pragma unroll
    for (int r = 0; r < R; ++r) {
#pragma unroll
      for (int u = 0; u < kWMaxU; ++u) acc[r][u] = ta[r][u];
#pragma unroll
      for (int c = 0; c < 3; ++c) xr[r][c] = tx[r][c];
    }
  }
}

// WARPS warps of RPW rows each, NR rows evaluated together; MINB CTAs resident per SM.
template <bool DERIV, int KIND, int WARPS, int RPW, int NR, int MINB>
__global__ void __launch_bounds__(WARPS * 32, MINB)
    k_sketch_wht(int64_t n, int64_t row0, int64_t m, int dim, int d, int nchunks, KernelParams kp,
                 const float *__restrict__ ps, const float *__restrict__ Kd, int64_t ldk,
                 const uint32_t *__restrict__ tsg, const uint32_t *__restrict__ gsw,
                 const uint32_t *__restrict__ gtab, const int *__restrict__ jtab, float *__restrict__ Y, int64_t ldy) {
  constexpr int kThreads = WARPS * 32, kRows = WARPS * RPW;
  constexpr bool kDense = KIND == CKINV_DENSE;   // entries read from a materialised K0
  static_assert(kRows <= 32 && RPW % NR == 0, "rows per CTA");
  static_assert(!kDense || RPW == NR, "a materialised K0 takes one group of rows per warp");
  extern __shared__ __align__(16) unsigned char wht_smem[];
  using Smem = WhtSmem<WARPS, NR, kRows, !kDense>;
  auto &S = *reinterpret_cast<Smem *>(wht_smem);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const float inv_l = kp.inv_l;
  const int nu = (d + 31) / 32;
  const int chunk_floats = kWB * dim;               // a 16-byte multiple for every dim

  // chunk ka's points and sign words into buffer b (asynchronous copies, one group); a
  // materialised K0 needs no points, and each warp reads its sign words itself
  auto stage = [&](int ka, int b) {
    if constexpr (kDense) return;
    const float *src = ps + (int64_t)ka * chunk_floats;
    for (int e = threadIdx.x * 4; e < chunk_floats; e += kThreads * 4) cp_async16(&S.sp[b][e], src + e);
    if (threadIdx.x < 8)
      cp_async16(&S.ssg[b][4 * threadIdx.x], tsg + (int64_t)ka * 32 + 4 * threadIdx.x);
    else if (threadIdx.x < 16)
      cp_async16(&S.sgs[b][4 * (threadIdx.x - 8)], gsw + (int64_t)ka * 32 + 4 * (threadIdx.x - 8));
    cp_async_commit();
  };
  stage(0, 0);
  for (int s = threadIdx.x; s < 32 * kWMaxU; s += kThreads) {
    S.gtab[s] = s < 32 * nu ? gtab[s] : 0u;
    S.jtab[s] = s < 32 * nu ? jtab[s] : -1;
  }
  // this warp's rows and their pre-scaled coordinates
  const int64_t rcta = (int64_t)blockIdx.x * kRows;
  const int64_t rbase = rcta + warp * RPW;
  float xr[RPW][3];
  const float *kc[NR];
#pragma unroll
  for (int r = 0; r < RPW; ++r) {
    const int64_t i = min(rbase + r, m - 1);
#pragma unroll
    for (int c = 0; c < 3; ++c) xr[r][c] = (!kDense && c < dim) ? ps[(row0 + i) * dim + c] : 0.f;
    if (r < NR) kc[r] = kDense ? Kd + (row0 + i) * ldk : nullptr;
  }
  float acc[RPW][kWMaxU];
#pragma unroll
  for (int r = 0; r < RPW; ++r)
#pragma unroll
    for (int u = 0; u < kWMaxU; ++u) acc[r][u] = 0.f;
  cp_async_wait_all();
  __syncthreads();
  // gather addresses of this lane's slots, two 16-bit fields a register (constant over chunks)
  uint32_t addr2[kWMaxU / 2];
#pragma unroll
  for (int h = 0; h < kWMaxU / 2; ++h)
    addr2[h] = (S.gtab[lane + 64 * h] & 0x7ffu) | ((S.gtab[lane + 64 * h + 32] & 0x7ffu) << 16);

  float *wb = S.buf + warp * NR * 32 * kWPad;
  // L2 prefetch of chunk ka's 4 KB of each of this warp's columns, issued kPfAhead chunks
  // before the chunk is read: lane l takes the 64-byte segments l and l + 32 (one prefetch
  // fills one 64-byte segment); segments past n are not touched
  auto prefetch_chunk = [&](int ka) {
    if constexpr (kDense) {
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        const int64_t kn = (int64_t)ka * kWB + 16 * (lane + 32 * h);
        if (kn < n) {
#pragma unroll
          for (int r = 0; r < NR; ++r) prefetch_l2(kc[r] + kn);
        }
      }
    }
  };
#pragma unroll 1
  for (int ka = 1; ka < kPfAhead; ++ka) prefetch_chunk(ka);
  // a materialised K0's sign words, read by each warp one chunk ahead (no block barrier in
  // its chunk loop: the warps run decoupled)
  uint32_t smask_next = 0, gsg_next = 0;
  if constexpr (kDense) {
    smask_next = __ldg(tsg + lane);
    gsg_next = __ldg(gsw + lane);
  }
  for (int ka = 0; ka < nchunks; ++ka) {
    const int b = ka & 1;
    if (ka + 1 < nchunks) stage(ka + 1, b ^ 1);
    const int64_t k0 = (int64_t)ka * kWB;
    const int rem = n - k0 < kWB ? (int)(n - k0) : kWB;   // live entries of this chunk
    prefetch_chunk(ka + kPfAhead);
    uint32_t smask, gsg;   // signs of this lane's 32 entries; (-1)^popcount(k_a & p_a) of its slots
    if constexpr (kDense) {
      smask = smask_next;
      gsg = gsg_next;
      if (ka + 1 < nchunks) {
        smask_next = __ldg(tsg + (int64_t)(ka + 1) * 32 + lane);
        gsg_next = __ldg(gsw + (int64_t)(ka + 1) * 32 + lane);
      }
    } else {
      smask = S.ssg[b][lane];
      gsg = S.sgs[b][lane];
    }
    const float *P = S.sp[b];
    // the warp's rows, NR at a time: the body is kept rolled (unrolled copies overflow the
    // instruction cache); the rows in work are always the first NR, rotated after each group
#pragma unroll 1
    for (int g = 0; g < RPW / NR; ++g) {
      float v[NR][32];
      const float(&xw)[NR][3] = *reinterpret_cast<const float(*)[NR][3]>(&xr[0][0]);
      if constexpr (kDense) {
        if (rem == kWB)
          load_rows<false, NR>(kc, k0, smask, lane, rem, v);
        else
          load_rows<true, NR>(kc, k0, smask, lane, rem, v);
      } else if (pad_far(KIND, DERIV) || rem == kWB) {
        eval_rows<DERIV, KIND, false, NR>(P, dim, xw, inv_l, smask, lane, rem, v);
      } else {
        eval_rows<DERIV, KIND, !pad_far(KIND, DERIV), NR>(P, dim, xw, inv_l, smask, lane, rem, v);
      }
      wht1024_rows<NR>(v, wb, lane);
      __syncwarp();
#pragma unroll
      for (int u = 0; u < kWMaxU; ++u) {
        if (u < nu) {
          const uint32_t a = (addr2[u >> 1] >> (16 * (u & 1))) & 0xffffu;
#pragma unroll
          for (int r = 0; r < NR; ++r) acc[r][u] += flip_if(wb[r * 32 * kWPad + a], gsg, u);
        }
      }
      rotate_rows<RPW, NR>(acc, xr);
    }
    if constexpr (!kDense) {
      cp_async_wait_all();
      __syncthreads();
    }
  }
  if constexpr (kDense) __syncthreads();   // the staging tile below overlaps other warps' buffers
  // Y = scale * acc: stage the CTA's rows x d block as T[j][row], then write each column's
  // rows as one contiguous segment
  float *T = S.buf;
#pragma unroll
  for (int u = 0; u < kWMaxU; ++u) {
    const int j = S.jtab[lane + 32 * u];
    if (u < nu && j >= 0) {
#pragma unroll
      for (int r = 0; r < RPW; ++r) T[j * Smem::kTPad + warp * RPW + r] = acc[r][u];
    }
  }
  __syncthreads();
  const float scale = (float)kp.scale;
  const int64_t i = rcta + lane;
  if (lane < kRows && i < m)
    for (int j = warp; j < d; j += WARPS) Y[i + (int64_t)j * ldy] = T[j * Smem::kTPad + lane] * scale;
}

// ps[e] = points[e] * coord_scale for the n * dim coordinates, `pad` up to `total`.
__global__ void k_wht_scale(const float *__restrict__ pts, int64_t count, int64_t total, float cs, float pad,
                            float *__restrict__ ps) {
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x)
    ps[e] = e < count ? pts[e] * cs : pad;
}

// Per chunk ka and lane l: tsg = the lane's 32 Rademacher sign bits (bit t for entry
// ka B + l + 32 t; zero past n), gsw = the gather signs (-1)^popcount(ka & p_a) of its slots.
__global__ void k_wht_masks(const uint32_t *__restrict__ bits, int64_t n, int nchunks, const uint32_t *__restrict__ gtab,
                            uint32_t *__restrict__ tsg, uint32_t *__restrict__ gsw) {
  const int64_t nwords = (n + 31) / 32;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < (int64_t)nchunks * 32;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t ka = e >> 5;
    const int l = (int)(e & 31);
    uint32_t m = 0;
    for (int t = 0; t < 32; ++t) {
      const int64_t w = ka * 32 + t;
      const uint32_t word = w < nwords ? bits[w] : 0u;
      m |= ((word >> l) & 1u) << t;
    }
    tsg[e] = m;
    uint32_t g = 0;
    for (int u = 0; u < kWMaxU; ++u) g |= (uint32_t)(__popc((uint32_t)ka & (gtab[l + 32 * u] >> 11)) & 1) << u;
    gsw[e] = g;
  }
}

// The output slots: output j reads U[p_b] at buffer address a_j = (p_b / 32) * 33 + p_b % 32,
// in bank a_j % 32.  Output j goes to lane bank(a_j), slot = its rank among the outputs of that
// bank; outputs past the last slot of their bank (rare) fill the empty slots in order.  One CTA;
// one warp ranks the outputs 32 at a time (match masks plus per-bank running counts) and pairs
// the k-th overflowing output with the k-th empty slot by ballot prefix counts.
__global__ void k_wht_slots(const int32_t *__restrict__ cols, int d, uint32_t *__restrict__ gtab,
                            int *__restrict__ jtab) {
  __shared__ uint32_t sa[32 * kWMaxU];
  __shared__ int slot[32 * kWMaxU];
  __shared__ int elist[32 * kWMaxU];
  __shared__ int cnt[32];
  const int nu = (d + 31) / 32;
  for (int j = threadIdx.x; j < d; j += blockDim.x) {
    const int p = cols[j], q = p & (kWB - 1);
    sa[j] = (uint32_t)((q >> 5) * kWPad + (q & 31)) | ((uint32_t)(p >> 10) << 11);
  }
  for (int s = threadIdx.x; s < 32 * kWMaxU; s += blockDim.x) {
    gtab[s] = 0u;
    jtab[s] = -1;
  }
  if (threadIdx.x < 32) cnt[threadIdx.x] = 0;
  __syncthreads();
  if (threadIdx.x < 32) {
    const int lane = threadIdx.x;
    const unsigned lt = (1u << lane) - 1u;
    // rank of output j: the outputs of its bank in earlier groups (cnt) and in lower lanes of
    // its own group; cnt[b] ends as the number of outputs in bank b
    for (int g = 0; g < d; g += 32) {
      const int j = g + lane;
      const bool v = j < d;
      const uint32_t bank = v ? (sa[j] & 31u) : 32u + (uint32_t)lane;   // lanes past d match none
      const unsigned peers = __match_any_sync(0xffffffffu, bank);
      const int base = v ? cnt[bank] : 0;
      __syncwarp();
      if (v) {
        const int rank = base + __popc(peers & lt);
        slot[j] = rank < nu ? rank * 32 + (int)bank : -1;
        if ((peers >> lane) == 1u) cnt[bank] = base + __popc(peers);   // the group's last of the bank
      }
      __syncwarp();
    }
    // the empty slots s = 32 u + l (empty iff u >= cnt[l]), in order of s
    int ne = 0;
    for (int g = 0; g < 32 * nu; g += 32) {
      const bool e = (g >> 5) >= cnt[lane];
      const unsigned m = __ballot_sync(0xffffffffu, e);
      if (e) elist[ne + __popc(m & lt)] = g + lane;
      ne += __popc(m);
    }
    __syncwarp();
    // the k-th overflowing output (in order of j) takes the k-th empty slot: 32 nu >= d leaves
    // at least as many empty slots as there are overflowing outputs
    int no = 0;
    for (int g = 0; g < d; g += 32) {
      const int j = g + lane;
      const bool o = j < d && slot[j] < 0;
      const unsigned m = __ballot_sync(0xffffffffu, o);
      if (o) slot[j] = elist[no + __popc(m & lt)];
      no += __popc(m);
    }
  }
  __syncthreads();
  for (int j = threadIdx.x; j < d; j += blockDim.x) {
    if (slot[j] < 0) continue;
    gtab[slot[j]] = sa[j];
    jtab[slot[j]] = j;
  }
}

// The launch configuration: 4 warps of 2 rows (evaluated as a pair), 3 CTAs per SM (167
// registers a thread: 12 warps an SM).  Measured at 262144 points, d = 512, against 8 warps of
// 4 rows (252 registers, 8 warps an SM): 65.7 ms against 84 ms; 12 warps of 2 rows in one CTA
// 73 ms, 6 warps x 2 CTAs 67.6 ms, 3 warps x 4 CTAs 67.0 ms.
constexpr int kCfgWarps = 4, kCfgRowsPerWarp = 2, kCfgPair = 2, kCfgMinBlocks = 3;
// A materialised K0: one row a warp (96 registers), 5 CTAs = 20 warps resident per SM to
// cover the streaming loads (2 rows a warp at 168 registers held 12: 3.3 against 3.0 ms for
// the 17.2 GB K of 65536 points; 4 CTAs at 124 registers: 3.06 ms; 6 spill).
constexpr int kDnWarps = 4, kDnRowsPerWarp = 1, kDnMinBlocks = 5;

template <bool DERIV, int KIND>
Error launch_wht(int64_t n, int64_t row0, int64_t m, int dim, int d, int nchunks, const KernelParams &kp,
                 const float *ps, const float *Kd, int64_t ldk, const uint32_t *tsg, const uint32_t *gsw,
                 const uint32_t *gtab, const int *jtab, float *Y, int64_t ldy, cudaStream_t st) {
  constexpr bool kDense = KIND == CKINV_DENSE;
  constexpr int W = kDense ? kDnWarps : kCfgWarps, RPW = kDense ? kDnRowsPerWarp : kCfgRowsPerWarp;
  constexpr int NR = kDense ? kDnRowsPerWarp : kCfgPair, MINB = kDense ? kDnMinBlocks : kCfgMinBlocks;
  auto kfn = k_sketch_wht<DERIV, KIND, W, RPW, NR, MINB>;
  constexpr size_t smem = sizeof(WhtSmem<W, NR, W * RPW, !kDense>);
  CK_CUDA(cudaFuncSetAttribute(kfn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  CK_CUDA(cudaFuncSetAttribute(kfn, cudaFuncAttributePreferredSharedMemoryCarveout, 100));
  const dim3 grid((unsigned)ceil_div(m, W * RPW));
  note_launch();
  kfn<<<grid, W * 32, smem, st>>>(n, row0, m, dim, d, nchunks, kp, ps, Kd, ldk, tsg, gsw, gtab, jtab, Y, ldy);
  CK_CUDA(cudaGetLastError());
  return ok();
}

}  // namespace

bool sketch_wht_supported(int64_t n, int d) { return padded_order(n) >= kWB && d <= 32 * kWMaxU; }

Error sketch_wht(ckinv_ctx *ctx, int64_t n, int dim, int d, const KernelParams &kp, const float *points, bool deriv,
                 float *Y, int64_t ldy, cudaStream_t st, int64_t row0, int64_t m) {
  if (m < 0) m = n;
  if (!sketch_wht_supported(n, d)) return fail(CKINV_EUNSUPPORTED, "structured sketch: needs N >= 1024, d <= 512");
  if (m == 0) return ok();
  // chunks wholly past n hold only padding (zero entries) and are skipped
  const int nchunks = (int)ceil_div(n, kWB);
  const int64_t total = (int64_t)nchunks * kWB * dim;
  // scratch, each part on a 256-byte boundary: the pre-scaled points padded to whole chunks,
  // the two slot tables, the two per-chunk mask tables
  auto up = [](size_t b) { return (b + 255) / 256 * 256; };
  const size_t ps_bytes = up(sizeof(float) * (size_t)total);
  const size_t tab_bytes = up(sizeof(uint32_t) * 32 * kWMaxU);
  const size_t mask_bytes = up(sizeof(uint32_t) * 32 * (size_t)nchunks);
  unsigned char *scratch = nullptr;
  CK_CUDA(dev_alloc(&scratch, ps_bytes + 2 * tab_bytes + 2 * mask_bytes, st));
  float *ps = reinterpret_cast<float *>(scratch);
  uint32_t *gtab = reinterpret_cast<uint32_t *>(scratch + ps_bytes);
  int *jtab = reinterpret_cast<int *>(scratch + ps_bytes + tab_bytes);
  uint32_t *tsg = reinterpret_cast<uint32_t *>(scratch + ps_bytes + 2 * tab_bytes);
  uint32_t *gsw = reinterpret_cast<uint32_t *>(scratch + ps_bytes + 2 * tab_bytes + mask_bytes);
  const int sgrid = (int)std::min<int64_t>(ceil_div(total, 256), (int64_t)ctx->sm_count * 8);
  note_launch();
  k_wht_scale<<<sgrid, 256, 0, st>>>(points, n * dim, total, kp.coord_scale,
                                     pad_far(kp.kind, deriv) ? kPadFar : 0.f, ps);
  note_launch();
  k_wht_slots<<<1, 256, 0, st>>>(ctx->om.cols, d, gtab, jtab);
  note_launch();
  k_wht_masks<<<(unsigned)ceil_div((int64_t)nchunks * 32, 256), 256, 0, st>>>(ctx->om.bits, n, nchunks, gtab, tsg, gsw);
  Error e = ok();
  if (cudaGetLastError() != cudaSuccess) e = fail(CKINV_ECUDA, "structured sketch: set-up launch failed");
  if (e.st == CKINV_OK) {
    if (kp.kind == CKINV_SE)
      e = deriv ? launch_wht<true, CKINV_SE>(n, row0, m, dim, d, nchunks, kp, ps, nullptr, 0, tsg, gsw, gtab, jtab, Y,
                                             ldy, st)
                : launch_wht<false, CKINV_SE>(n, row0, m, dim, d, nchunks, kp, ps, nullptr, 0, tsg, gsw, gtab, jtab, Y,
                                              ldy, st);
    else
      e = deriv ? launch_wht<true, CKINV_MATERN52>(n, row0, m, dim, d, nchunks, kp, ps, nullptr, 0, tsg, gsw, gtab,
                                                   jtab, Y, ldy, st)
                : launch_wht<false, CKINV_MATERN52>(n, row0, m, dim, d, nchunks, kp, ps, nullptr, 0, tsg, gsw, gtab,
                                                    jtab, Y, ldy, st);
  }
  cudaFreeAsync(scratch, st);
  return e;
}

Error sketch_wht_dense(ckinv_ctx *ctx, int64_t n, int d, const KernelParams &kp, const float *K, int64_t ldk, float *Y,
                       int64_t ldy, cudaStream_t st, int64_t row0, int64_t m, const uint32_t *bits,
                       const int32_t *cols) {
  if (m < 0) m = n;
  if (!bits) bits = ctx->om.bits;
  if (!cols) cols = ctx->om.cols;
  if (!sketch_wht_supported(n, d)) return fail(CKINV_EUNSUPPORTED, "structured sketch: needs N >= 1024, d <= 512");
  if (m == 0) return ok();
  const int nchunks = (int)ceil_div(n, kWB);
  auto up = [](size_t b) { return (b + 255) / 256 * 256; };
  const size_t tab_bytes = up(sizeof(uint32_t) * 32 * kWMaxU);
  const size_t mask_bytes = up(sizeof(uint32_t) * 32 * (size_t)nchunks);
  unsigned char *scratch = nullptr;
  CK_CUDA(dev_alloc(&scratch, 2 * tab_bytes + 2 * mask_bytes, st));
  uint32_t *gtab = reinterpret_cast<uint32_t *>(scratch);
  int *jtab = reinterpret_cast<int *>(scratch + tab_bytes);
  uint32_t *tsg = reinterpret_cast<uint32_t *>(scratch + 2 * tab_bytes);
  uint32_t *gsw = reinterpret_cast<uint32_t *>(scratch + 2 * tab_bytes + mask_bytes);
  note_launch();
  k_wht_slots<<<1, 256, 0, st>>>(cols, d, gtab, jtab);
  note_launch();
  k_wht_masks<<<(unsigned)ceil_div((int64_t)nchunks * 32, 256), 256, 0, st>>>(bits, n, nchunks, gtab, tsg, gsw);
  Error e = ok();
  if (cudaGetLastError() != cudaSuccess) e = fail(CKINV_ECUDA, "structured sketch: set-up launch failed");
  if (e.st == CKINV_OK)
    e = launch_wht<false, CKINV_DENSE>(n, row0, m, 1, d, nchunks, kp, nullptr, K, ldk, tsg, gsw, gtab, jtab, Y, ldy, st);
  cudaFreeAsync(scratch, st);
  return e;
}

namespace {
// B[j + i d] = (double) Bt[i + j d]
__global__ void k_transpose_widen(int d, const float *__restrict__ Bt, double *__restrict__ B) {
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < d * d; e += gridDim.x * blockDim.x) {
    const int i = e % d, j = e / d;
    B[j + (int64_t)i * d] = (double)Bt[e];
  }
}
}  // namespace

Error omega_t_times_wht(ckinv_ctx *ctx, int64_t n, int d, const float *X, int64_t ldx, const uint32_t *bits,
                        const int32_t *cols, double scale, double *B, cudaStream_t st) {
  float *Bt = nullptr;
  CK_CUDA(dev_alloc(&Bt, sizeof(float) * (size_t)d * d, st));
  KernelParams kp{};
  kp.kind = CKINV_DENSE;
  kp.scale = scale;
  Error e = sketch_wht_dense(ctx, n, d, kp, X, ldx, Bt, d, st, 0, d, bits, cols);
  if (e.st == CKINV_OK) {
    note_launch();
    k_transpose_widen<<<(unsigned)std::min<int64_t>(ceil_div((int64_t)d * d, 256), 1024), 256, 0, st>>>(d, Bt, B);
    if (cudaGetLastError() != cudaSuccess) e = fail(CKINV_ECUDA, "transpose launch failed");
  }
  cudaFreeAsync(Bt, st);
  return e;
}

}  // namespace ckinv
