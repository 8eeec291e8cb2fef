// Fused sketch Y = K0 Omega (Sec. 3.1-3.3) on the 5th-generation tensor cores.
//
// One CTA owns 128 rows of Y and all d <= 512 columns; the FP32 accumulator lives in
// TMEM (128 lanes x d columns).  The contraction runs over the n points in blocks of 64:
//   * warps 2..9 evaluate the 128 x 64 kernel tile in FP32 (exp2 on the MUFU), split it
//     into 1-3 BF16 terms and store them straight into the 128B-swizzled K-major SMEM
//     layout the MMA reads (no HBM traffic for K0 at all);
//   * warp 0 streams the 64 x d tile of the +-1 Omega pattern (BF16, exact) by TMA;
//   * warp 1 issues tcgen05.mma (M = 128, N = min(d, 256) per instruction, K = 16) and
//     commits each stage back to the producers through mbarriers;
//   * after the last block, warps 2..9 read TMEM with tcgen05.ld, scale by variance * c
//     and write Y (coalesced along rows: Y is column-major).
// Every mbarrier wait is bounded; on timeout the CTA records DERR_TIMEOUT, drains its
// own TMA copies and MMAs, frees TMEM and returns.
#include <cuda.h>
#include <cudaTypedefs.h>
#include <cstring>

#include "internal.cuh"

namespace ckinv {
namespace {

constexpr int BM = 128;
constexpr int BK = 64;
constexpr int kThreads = 320;          // 10 warps
constexpr int kProducerThreads = 256;  // warps 2..9
constexpr uint32_t kATileBytes = BM * BK * 2;  // 16 KB per BF16 term

// ------------------------------------------------------------------ PTX wrappers
__device__ __forceinline__ uint32_t smem_u32(const void *p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count));
}
__device__ __forceinline__ void mbar_arrive(uint32_t bar) {
  asm volatile("{\n .reg .b64 st;\n mbarrier.arrive.shared::cta.b64 st, [%0];\n}\n" ::"r"(bar)
               : "memory");
}
__device__ __forceinline__ void mbar_arrive_expect_tx(uint32_t bar, uint32_t bytes) {
  asm volatile(
      "{\n .reg .b64 st;\n mbarrier.arrive.expect_tx.shared::cta.b64 st, [%0], %1;\n}\n" ::"r"(bar),
      "r"(bytes)
      : "memory");
}
// try_wait with a suspend-time hint: the thread sleeps until the phase completes or the
// hint (ns) elapses, instead of spinning on the issue slots.
__device__ __forceinline__ bool mbar_try_wait(uint32_t bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, %3;\n"
      " selp.b32 %0, 1, 0, p;\n}\n"
      : "=r"(ok)
      : "r"(bar), "r"(parity), "r"(20000u)
      : "memory");
  return ok != 0;
}
__device__ __forceinline__ uint64_t global_ns() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}
// Bounded wait: gives up after ~1 s or when another warp has flagged an abort.
__device__ __noinline__ bool mbar_wait(uint32_t bar, uint32_t parity, volatile int *abort_flag) {
  if (mbar_try_wait(bar, parity)) return true;
  const uint64_t t0 = global_ns();
  for (uint32_t it = 0;; ++it) {
    if (mbar_try_wait(bar, parity)) return true;
    if ((it & 15u) == 15u) {
      if (*abort_flag) return false;
      if (global_ns() - t0 > 1000000000ull) {
        *abort_flag = 1;
        return false;
      }
    }
  }
}

// Warp-uniform bounded wait: lane 0 polls, the warp agrees on the outcome.
__device__ __forceinline__ bool mbar_wait_warp(uint32_t bar, uint32_t parity, volatile int *abort_flag) {
  int ok = 0;
  if ((threadIdx.x & 31) == 0) ok = mbar_wait(bar, parity, abort_flag) ? 1 : 0;
  ok = __shfl_sync(0xffffffffu, ok, 0);
  __syncwarp();
  return ok != 0;
}
__device__ __forceinline__ void fence_async_smem() {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}
__device__ __forceinline__ void tma_load_2d(uint32_t dst, const CUtensorMap *map, uint32_t bar,
                                            int x, int y) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%3, %4}], [%2];" ::"r"(dst),
      "l"(map), "r"(bar), "r"(x), "r"(y)
      : "memory");
}
__device__ __forceinline__ void tc_fence_before() {
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void tc_fence_after() {
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void tc_commit(uint32_t bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar)
               : "memory");
}
__device__ __forceinline__ void tc_mma(uint32_t dtmem, uint64_t adesc, uint64_t bdesc, uint32_t idesc,
                                       uint32_t accum) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
      " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(dtmem),
      "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accum));
}
__device__ __forceinline__ void tmem_ld8(uint32_t taddr, float *v) {
  uint32_t r[8];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%8];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
        "=r"(r[7])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int i = 0; i < 8; ++i) v[i] = __uint_as_float(r[i]);
}

// SMEM matrix descriptor: K-major, 128B swizzle, 8-row groups 1024 B apart.
__device__ __forceinline__ uint64_t sw128_desc(uint32_t saddr) {
  uint64_t desc = 0;
  desc |= (uint64_t)((saddr & 0x3FFFFu) >> 4);        // start address
  desc |= (uint64_t)1 << 16;                          // leading byte offset (unused)
  desc |= (uint64_t)(1024 >> 4) << 32;                // stride byte offset
  desc |= (uint64_t)1 << 46;                          // descriptor version (sm_100 family)
  desc |= (uint64_t)2 << 61;                          // swizzle: 128B
  return desc;
}
// Instruction descriptor, kind::f16: D = F32, A = B = BF16, both K-major, M = 128.
__host__ __device__ constexpr uint32_t idesc_bf16(int N) {
  return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(BM >> 4) << 24);
}

struct TcArgs {
  int64_t n;       // contraction length (points); also the row count in kernel mode
  int64_t m;       // output rows (dense mode: rows of A)
  int dim;
  int d;
  int num_kb;      // 64-point blocks in total
  int kb_per_cta;  // blocks per CTA along the contraction (split over gridDim.y)
  int stages;
  int box_rows;    // rows of Omega^T per TMA box
  KernelParams kp;
  const float *pts;
  const float *A;  // dense mode: row i of A at A + i * lda (K-major)
  int64_t lda;
  float *Y;        // store mode: Y = scale * acc (column-major, ld ldy)
  int64_t ldy;
  float *part;     // partial mode: part[split][i + j * ldp] = acc
  int64_t ldp;
  int *err;
};

// MODE 0: A = kernel tile evaluated from the points;  MODE 1: A = a dense FP32 matrix.
template <int NSPLIT, bool DERIV, int MODE>
__global__ void __launch_bounds__(kThreads, 1)
    k_sketch_tc(const __grid_constant__ CUtensorMap tmapB, const TcArgs a) {
  extern __shared__ uint8_t smem_raw[];
  // layout: [barriers | tmem slot | abort flag][per-warp point buffers] then the
  // 1024-aligned stage tiles
  uint64_t *bars = reinterpret_cast<uint64_t *>(smem_raw);
  const int S = a.stages;
  uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(bars + 26);
  volatile int *abort_flag = reinterpret_cast<volatile int *>(tmem_slot + 1);
  float4 *xs_all = reinterpret_cast<float4 *>(smem_raw + 512);   // 8 warps x 32 points
  uintptr_t tiles_u =
      (reinterpret_cast<uintptr_t>(smem_raw) + 512 + 8 * 32 * 16 + 1023) & ~(uintptr_t)1023;
  uint8_t *tiles = reinterpret_cast<uint8_t *>(tiles_u);
  const uint32_t b_bytes = (uint32_t)a.d * BK * 2;
  const uint32_t stage_bytes = NSPLIT * kATileBytes + b_bytes;

  auto fullA = [&](int s) { return smem_u32(bars + s); };
  auto fullB = [&](int s) { return smem_u32(bars + 8 + s); };
  auto empty = [&](int s) { return smem_u32(bars + 16 + s); };
  const uint32_t accum_bar = smem_u32(bars + 24);
  const uint32_t drain_bar = smem_u32(bars + 25);
  auto a_tile = [&](int s, int t) {
    return smem_u32(tiles + (size_t)s * stage_bytes + (size_t)t * kATileBytes);
  };
  auto b_tile = [&](int s) { return smem_u32(tiles + (size_t)s * stage_bytes + NSPLIT * kATileBytes); };

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int64_t i0 = (int64_t)blockIdx.x * BM;
  const int kb_begin = blockIdx.y * a.kb_per_cta;
  const int nkb = max(0, min(a.num_kb, kb_begin + a.kb_per_cta) - kb_begin);
  uint32_t tmem_cols = 32;
  while ((int)tmem_cols < a.d) tmem_cols <<= 1;

  if (threadIdx.x == 0) {
    for (int s = 0; s < S; ++s) {
      mbar_init(fullA(s), kProducerThreads / 32);
      mbar_init(fullB(s), 1);
      mbar_init(empty(s), 1);
    }
    mbar_init(accum_bar, 1);
    mbar_init(drain_bar, 1);
    *abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 1) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     smem_u32(tmem_slot)),
                 "r"(tmem_cols));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem_base = *tmem_slot;

  if (warp == 0) {
    // ------------------------------------------------------------ TMA producer (Omega)
    if (lane == 0) {
      int issued = 0;
      for (int kb = 0; kb < nkb; ++kb) {
        int s = kb % S;
        uint32_t ph = (uint32_t)(kb / S) & 1u;
        if (!mbar_wait(empty(s), ph ^ 1u, abort_flag)) break;
        mbar_arrive_expect_tx(fullB(s), b_bytes);
        const int kx = (kb_begin + kb) * BK;
        tma_load_2d(b_tile(s), &tmapB, fullB(s), kx, 0);
        if (a.box_rows < a.d)
          tma_load_2d(b_tile(s) + (uint32_t)a.box_rows * 128u, &tmapB, fullB(s), kx, a.box_rows);
        ++issued;
      }
      // every copy this CTA issued must land before its shared memory is released
      volatile int never = 0;
      int first = issued - S < 0 ? 0 : issued - S;
      for (int kb = first; kb < issued; ++kb)
        mbar_wait(fullB(kb % S), (uint32_t)(kb / S) & 1u, &never);
    }
    __syncwarp();
  } else if (warp == 1) {
    // ------------------------------------------------------------ MMA issuer
    if (lane == 0) {
      const uint32_t id0 = idesc_bf16(a.d < 256 ? a.d : 256);
      const uint32_t id1 = idesc_bf16(a.d > 256 ? a.d - 256 : 16);
      bool good = true;
      int issued = 0;
      for (int kb = 0; kb < nkb; ++kb) {
        int s = kb % S;
        uint32_t ph = (uint32_t)(kb / S) & 1u;
        if (!mbar_wait(fullA(s), ph, abort_flag) || !mbar_wait(fullB(s), ph, abort_flag)) {
          good = false;
          break;
        }
        tc_fence_after();
#pragma unroll
        for (int t = 0; t < NSPLIT; ++t) {
#pragma unroll
          for (int kk = 0; kk < BK / 16; ++kk) {
            uint64_t ad = sw128_desc(a_tile(s, t) + kk * 32);
            uint64_t bd = sw128_desc(b_tile(s) + kk * 32);
            uint32_t acc = (kb > 0 || t > 0 || kk > 0) ? 1u : 0u;
            tc_mma(tmem_base, ad, bd, id0, acc);
            if (a.d > 256) {
              uint64_t bd1 = sw128_desc(b_tile(s) + 256u * 128u + kk * 32);
              tc_mma(tmem_base + 256u, ad, bd1, id1, acc);
            }
          }
        }
        tc_commit(empty(s));
        ++issued;
      }
      if (good) tc_commit(accum_bar);
      if (issued > 0) {
        // all MMAs of this CTA must finish before TMEM is released
        volatile int never = 0;
        tc_commit(drain_bar);
        mbar_wait(drain_bar, 0u, &never);
      }
    }
    __syncwarp();
  } else {
    // ------------------------------------------------------------ A-tile producers
    // producer warp pw = warp - 2 handles tile rows 32 (pw % 4) .. +31 and the k-half
    // pw / 4 of every 64-point block; each lane owns one row.
    const int pw = warp - 2;
    const int r = (pw & 3) * 32 + lane;
    const int h = pw >> 2;
    float4 *xw = xs_all + pw * 32;
    const int64_t irow = min(i0 + r, (MODE == 0 ? a.n : a.m) - 1);
    const float cs = a.kp.coord_scale;
    float x0 = 0.f, x1 = 0.f, x2 = 0.f;
    if (MODE == 0) {
      x0 = a.pts[irow * a.dim] * cs;
      if (a.dim > 1) x1 = a.pts[irow * a.dim + 1] * cs;
      if (a.dim > 2) x2 = a.pts[irow * a.dim + 2] * cs;
    }
    const float *arow = (MODE == 1) ? a.A + irow * a.lda : nullptr;
    const bool row_ok = (MODE == 1) ? (i0 + r < a.m) : true;
    const int kind = a.kp.kind;
    const float inv_l = a.kp.inv_l;
    const uint32_t rowbase = (uint32_t)r * 128u;
    const uint32_t swz = (uint32_t)(r & 7);
    bool good = true;
    // the point this lane stages for the next block, fetched one block ahead
    auto load_point = [&](int kb) {
      float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
      int64_t k = (int64_t)(kb_begin + kb) * BK + h * 32 + lane;
      if (MODE == 0 && kb < nkb && k < a.n) {
        v.x = a.pts[k * a.dim] * cs;
        if (a.dim > 1) v.y = a.pts[k * a.dim + 1] * cs;
        if (a.dim > 2) v.z = a.pts[k * a.dim + 2] * cs;
        v.w = 1.0f;                        // marks a real point
      }
      return v;
    };
    float4 pnext = load_point(0);
    for (int kb = 0; kb < nkb; ++kb) {
      int s = kb % S;
      uint32_t ph = (uint32_t)(kb / S) & 1u;
      const int64_t kbase = (int64_t)(kb_begin + kb) * BK + h * 32;
      const bool full_block = (kbase + 32 <= (MODE == 0 ? a.n : a.n));
      if (MODE == 0) {
        __syncwarp();                      // previous block's reads of xw are done
        xw[lane] = pnext;
        __syncwarp();
        pnext = load_point(kb + 1);
      }
      if (!mbar_wait_warp(empty(s), ph ^ 1u, abort_flag)) { good = false; break; }
#pragma unroll
      for (int c = 0; c < 4; ++c) {
        float kv[8];
        if (MODE == 0) {
          if (full_block && a.dim <= 2) {
#pragma unroll
            for (int u = 0; u < 8; ++u) {
              float4 p = xw[c * 8 + u];
              float dx = x0 - p.x, dy = x1 - p.y;
              kv[u] = dev::kernel_value(kind, fmaf(dy, dy, dx * dx), inv_l, DERIV);
            }
          } else {
#pragma unroll
            for (int u = 0; u < 8; ++u) {
              float4 p = xw[c * 8 + u];
              float dx = x0 - p.x, dy = x1 - p.y, dz = x2 - p.z;
              float r2 = fmaf(dz, dz, fmaf(dy, dy, dx * dx));
              float v = dev::kernel_value(kind, r2, inv_l, DERIV);
              kv[u] = (p.w != 0.0f) ? v : 0.0f;
            }
          }
        } else {
          const int64_t k0 = kbase + c * 8;
          if (row_ok && k0 + 8 <= a.n) {
            float4 lo = *reinterpret_cast<const float4 *>(arow + k0);
            float4 hi = *reinterpret_cast<const float4 *>(arow + k0 + 4);
            kv[0] = lo.x; kv[1] = lo.y; kv[2] = lo.z; kv[3] = lo.w;
            kv[4] = hi.x; kv[5] = hi.y; kv[6] = hi.z; kv[7] = hi.w;
          } else {
#pragma unroll
            for (int u = 0; u < 8; ++u) kv[u] = (row_ok && k0 + u < a.n) ? arow[k0 + u] : 0.0f;
          }
        }
        const uint32_t chunk = (uint32_t)(h * 4 + c);
        const uint32_t off = rowbase + ((chunk ^ swz) << 4);
#pragma unroll
        for (int t = 0; t < NSPLIT; ++t) {
          uint32_t w[4];
#pragma unroll
          for (int u = 0; u < 4; ++u) {
            __nv_bfloat162 b2 = __floats2bfloat162_rn(kv[2 * u], kv[2 * u + 1]);
            w[u] = *reinterpret_cast<uint32_t *>(&b2);
            if (t + 1 < NSPLIT) {
              float2 back = __bfloat1622float2(b2);
              kv[2 * u] -= back.x;
              kv[2 * u + 1] -= back.y;
            }
          }
          const uint32_t dst = a_tile(s, t) + off;
          asm volatile("st.shared.v4.b32 [%0], {%1, %2, %3, %4};" ::"r"(dst), "r"(w[0]), "r"(w[1]),
                       "r"(w[2]), "r"(w[3])
                       : "memory");
        }
      }
      fence_async_smem();
      __syncwarp();
      if (lane == 0) mbar_arrive(fullA(s));
    }
    // ------------------------------------------------------------ epilogue
    bool e_ok = good && nkb > 0 && mbar_wait_warp(accum_bar, 0u, abort_flag);
    if (e_ok) {
      tc_fence_after();
      const int q = warp & 3;                 // TMEM lane quadrant this warp may access
      const int half = pw >> 2;               // two warps per quadrant split the columns
      const int cols_half = a.d / 2;
      const int64_t i = i0 + q * 32 + lane;
      const float scale = (float)a.kp.scale;
      const int64_t mrows = (MODE == 0) ? a.n : a.m;
      float *pout = a.part ? a.part + (int64_t)blockIdx.y * a.ldp * a.d : nullptr;
      for (int j = half * cols_half; j < (half + 1) * cols_half; j += 8) {
        float v[8];
        tmem_ld8(tmem_base + ((uint32_t)(q * 32) << 16) + (uint32_t)j, v);
        if (i < mrows) {
          if (pout) {
#pragma unroll
            for (int t = 0; t < 8; ++t) pout[i + (int64_t)(j + t) * a.ldp] = nkb > 0 ? v[t] : 0.0f;
          } else {
#pragma unroll
            for (int t = 0; t < 8; ++t) a.Y[i + (int64_t)(j + t) * a.ldy] = v[t] * scale;
          }
        }
      }
    }
  }
  tc_fence_before();
  __syncthreads();
  if (*abort_flag && threadIdx.x == 0) atomicOr(a.err, DERR_TIMEOUT);
  if (warp == 1) {
    tc_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem_base),
                 "r"(tmem_cols));
  }
}

PFN_cuTensorMapEncodeTiled_v12000 get_encode() {
  static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
  if (!fn) {
    cudaDriverEntryPointQueryResult q;
    void *p = nullptr;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
            cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
  }
  return fn;
}

template <int NSPLIT, bool DERIV, int MODE>
Error launch(const CUtensorMap &map, const TcArgs &a, size_t smem, dim3 grid, cudaStream_t st) {
  auto kfn = k_sketch_tc<NSPLIT, DERIV, MODE>;
  CK_CUDA(cudaFuncSetAttribute(kfn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  ::ckinv::note_launch();
  kfn<<<grid, kThreads, smem, st>>>(map, a);
  CK_CUDA(cudaGetLastError());
  return ok();
}

// Tensor map over the BF16 Omega^T of the context and the launch geometry.
Error prepare(ckinv_ctx *ctx, int d, int nsplit, CUtensorMap *map, TcArgs *a, size_t *smem) {
  if (d % 16 != 0 || d > 512 || d < 16) return fail(CKINV_EINVAL, "sketch_tc: d must be 16..512, d % 16 == 0");
  if (nsplit < 1 || nsplit > 3) return fail(CKINV_EINVAL, "sketch_tc: 1..3 BF16 terms");
  const OmegaCache &om = ctx->om;
  PFN_cuTensorMapEncodeTiled_v12000 enc = get_encode();
  if (!enc) return fail(CKINV_ECUDA, "cuTensorMapEncodeTiled entry point unavailable");
  const int box_rows = d <= 256 ? d : d / 2;
  cuuint64_t gdim[2] = {(cuuint64_t)om.kpad, (cuuint64_t)d};
  cuuint64_t gstride[1] = {(cuuint64_t)om.kpad * 2};
  cuuint32_t box[2] = {(cuuint32_t)BK, (cuuint32_t)box_rows};
  cuuint32_t estr[2] = {1, 1};
  CUresult cr = enc(map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, (void *)om.omegaT, gdim, gstride, box, estr,
                    CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                    CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (cr != CUDA_SUCCESS) return fail(CKINV_ECUDA, "cuTensorMapEncodeTiled failed");
  memset(a, 0, sizeof(*a));
  a->d = d;
  a->num_kb = (int)(om.kpad / BK);
  a->kb_per_cta = a->num_kb;
  a->box_rows = box_rows;
  a->err = ctx->d_err;
  const size_t stage_bytes = (size_t)nsplit * kATileBytes + (size_t)d * BK * 2;
  const size_t head = 512 + 8 * 32 * 16 + 1024;   // barriers, point buffers, alignment slack
  const size_t limit = 227 * 1024;
  int S = (int)((limit - head) / stage_bytes);
  if (S > 4) S = 4;
  if (S < 1) return fail(CKINV_EUNSUPPORTED, "sketch_tc: stage does not fit in shared memory");
  a->stages = S;
  *smem = head + (size_t)S * stage_bytes;
  return ok();
}

template <int MODE>
Error dispatch(int nsplit, bool deriv, const CUtensorMap &map, const TcArgs &a, size_t smem, dim3 grid,
               cudaStream_t st) {
  switch (nsplit * 2 + (deriv ? 1 : 0)) {
    case 2: return launch<1, false, MODE>(map, a, smem, grid, st);
    case 3: return launch<1, true, MODE>(map, a, smem, grid, st);
    case 4: return launch<2, false, MODE>(map, a, smem, grid, st);
    case 5: return launch<2, true, MODE>(map, a, smem, grid, st);
    case 6: return launch<3, false, MODE>(map, a, smem, grid, st);
    case 7: return launch<3, true, MODE>(map, a, smem, grid, st);
  }
  return fail(CKINV_EINVAL, "sketch_tc: nsplit must be 1..3");
}

// G[i * si + j * sj] = scale * sum_s part[s][i + j * ldp]   (FP64 sum over the splits)
__global__ void k_reduce_parts(int m, int d, int splits, const float *part, int64_t ldp, double scale, double *G,
                               int64_t si, int64_t sj) {
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < (int64_t)m * d;
       e += (int64_t)gridDim.x * blockDim.x) {
    int64_t i = e % m, j = e / m;
    double acc = 0.0;
    for (int s = 0; s < splits; ++s) acc += (double)part[(int64_t)s * ldp * d + i + j * ldp];
    G[i * si + j * sj] = scale * acc;
  }
}

}  // namespace

Error sketch_tc(ckinv_ctx *ctx, int64_t n, int dim, int d, int nsplit, const KernelParams &kp, const float *points,
                bool deriv, float *Y, int64_t ldy, cudaStream_t st) {
  CK_TRY(omega_materialise_bf16(ctx, st));
  CUtensorMap map;
  TcArgs a;
  size_t smem = 0;
  CK_TRY(prepare(ctx, d, nsplit, &map, &a, &smem));
  a.n = n;
  a.m = n;
  a.dim = dim;
  a.kp = kp;
  a.pts = points;
  a.Y = Y;
  a.ldy = ldy;
  return dispatch<0>(nsplit, deriv, map, a, smem, dim3((unsigned)ceil_div(n, BM), 1), st);
}

Error dense_tc(ckinv_ctx *ctx, int64_t m, int64_t n, int d, int nsplit, const float *A, int64_t lda, double scale,
               float *Y, int64_t ldy, double *G, int64_t si, int64_t sj, cudaStream_t st) {
  if (lda % 4 != 0 || (reinterpret_cast<uintptr_t>(A) & 15) != 0)
    return fail(CKINV_EINVAL, "dense_tc: A must be 16-byte aligned with lda % 4 == 0");
  CK_TRY(omega_materialise_bf16(ctx, st));
  CUtensorMap map;
  TcArgs a;
  size_t smem = 0;
  CK_TRY(prepare(ctx, d, nsplit, &map, &a, &smem));
  a.n = n;
  a.m = m;
  a.A = A;
  a.lda = lda;
  a.kp.scale = scale;
  const int mt = (int)ceil_div(m, BM);
  if (Y) {
    a.Y = Y;
    a.ldy = ldy;
    return dispatch<1>(nsplit, false, map, a, smem, dim3(mt, 1), st);
  }
  // split the contraction so that the grid covers every SM, then reduce in FP64
  int splits = std::max(1, std::min(a.num_kb, (ctx->sm_count + mt - 1) / mt));
  a.kb_per_cta = (int)ceil_div(a.num_kb, splits);
  splits = (int)ceil_div(a.num_kb, a.kb_per_cta);
  const int64_t ldp = (int64_t)mt * BM;
  float *part = nullptr;
  CK_CUDA(cudaMallocAsync((void **)&part, sizeof(float) * (size_t)splits * ldp * d, st));
  a.part = part;
  a.ldp = ldp;
  Error e = dispatch<1>(nsplit, false, map, a, smem, dim3(mt, splits), st);
  if (e.st == CKINV_OK) {
    note_launch();
    k_reduce_parts<<<(unsigned)std::min<int64_t>(ceil_div(m * d, 256), 2048), 256, 0, st>>>(
        (int)m, d, splits, part, ldp, scale, G, si, sj);
    cudaError_t c = cudaGetLastError();
    if (c != cudaSuccess) e = fail(CKINV_ECUDA, cudaGetErrorString(c));
  }
  cudaFreeAsync(part, st);
  return e;
}

}  // namespace ckinv
