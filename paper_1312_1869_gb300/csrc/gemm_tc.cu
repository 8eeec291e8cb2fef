// FP32 strided-batched GEMM on the 5th-generation tensor cores, for the TSQR trailing
// updates and the formation of Q_hat (Sec. 3.3: the Householder block updates of each
// leaf and the products with the compact-WY factors):
//   C_b = alpha * op(A_b) * B_b + beta * C_b,   op(A) = A or A^T,   column-major, FP32.
//
// FP32 accuracy from BF16 tensor cores: every FP32 operand x is split into three BF16 terms
// x = x0 + x1 + x2 (each term the BF16 rounding of what is left, 24 significant bits in
// all), and a product a b is taken as the six term products whose order is at most 2
// (a0b0, a0b1, a1b0, a1b1, a0b2, a2b0); the dropped ones are below 2^-24 |a b|.  The
// products accumulate in FP32 in TMEM.
//
// One CTA computes a 128 x 128 tile of C: warp 1 owns TMEM (128 FP32 columns) and issues
// tcgen05.mma (M = 128, N = 128, K = 16, kind::f16); warps 2..9 load the 128 x 64 blocks of
// op(A) and B from global memory, split them and store the terms into 128B-swizzled
// K-major shared memory, two stages deep; after the last block they read TMEM back and
// write C.  Every mbarrier wait is bounded; on timeout the CTA records DERR_TIMEOUT, waits
// for its own MMAs, frees TMEM and returns.
#include <cuda_bf16.h>

#include "internal.cuh"

namespace ckinv {
namespace {

constexpr int GBM = 128, GBN = 128, GBK = 64;
constexpr int kTerms = 3;
constexpr int kPairs = 6;
constexpr int kGStages = 2;
constexpr int kGThreads = 320;
constexpr int kGProducers = 256;
constexpr uint32_t kGTile = GBM * GBK * 2;                   // one BF16 term of a 128 x 64 tile: 16 KB
constexpr uint32_t kGStage = 2 * kTerms * kGTile;            // A and B terms of one stage: 96 KB
constexpr size_t kGSmem = 1024 + 1024 + (size_t)kGStages * kGStage;

__device__ __forceinline__ uint32_t su32(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }
__device__ __forceinline__ void g_mbar_init(uint32_t bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count));
}
__device__ __forceinline__ void g_mbar_arrive(uint32_t bar) {
  asm volatile("{\n .reg .b64 st;\n mbarrier.arrive.shared::cta.b64 st, [%0];\n}\n" ::"r"(bar) : "memory");
}
__device__ __forceinline__ bool g_try_wait(uint32_t bar, uint32_t parity) {
  const uint32_t hint_ns = 20000u;
  uint32_t ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, %3;\n"
      " selp.b32 %0, 1, 0, p;\n}\n"
      : "=r"(ok)
      : "r"(bar), "r"(parity), "r"(hint_ns)
      : "memory");
  return ok != 0;
}
__device__ __forceinline__ uint64_t g_ns() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}
__device__ __forceinline__ bool g_test_wait(uint32_t bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.test_wait.parity.shared::cta.b64 p, [%1], %2;\n"
      " selp.b32 %0, 1, 0, p;\n}\n"
      : "=r"(ok)
      : "r"(bar), "r"(parity)
      : "memory");
  return ok != 0;
}
// A limit of at least 100 us polls with try_wait (20 us suspend hint) and checks the clock
// every 16 polls; a shorter one polls without suspending and checks after every poll.
__device__ __forceinline__ bool g_poll(uint32_t bar, uint32_t parity, uint64_t limit_ns) {
  return limit_ns < 100000ull ? g_test_wait(bar, parity) : g_try_wait(bar, parity);
}
// Bounded single-thread wait (gives up after limit_ns, or when another warp flags an abort).
__device__ __noinline__ bool g_wait_slow(uint32_t bar, uint32_t parity, volatile int *abort_flag, uint64_t limit_ns) {
  const uint64_t t0 = g_ns();
  const uint32_t every = limit_ns < 100000ull ? 0u : 15u;
  for (uint32_t it = 0;; ++it) {
    if (g_poll(bar, parity, limit_ns)) return true;
    if ((it & every) == every) {
      if (*abort_flag) return false;
      if (g_ns() - t0 > limit_ns) {
        *abort_flag = 1;
        return false;
      }
    }
  }
}
__device__ __forceinline__ bool g_wait(uint32_t bar, uint32_t parity, volatile int *abort_flag, uint64_t limit_ns) {
  return g_poll(bar, parity, limit_ns) || g_wait_slow(bar, parity, abort_flag, limit_ns);
}
// Warp-wide bounded wait: every lane polls (each acquires the phase), the warp leaves together.
__device__ __forceinline__ bool g_wait_lanes(uint32_t bar, uint32_t parity, volatile int *abort_flag,
                                             uint64_t limit_ns) {
  if (__all_sync(0xffffffffu, g_poll(bar, parity, limit_ns))) return true;
  const uint64_t t0 = g_ns();
  const uint32_t every = limit_ns < 100000ull ? 0u : 15u;
  for (uint32_t it = 0;; ++it) {
    if (__all_sync(0xffffffffu, g_poll(bar, parity, limit_ns))) return true;
    if ((it & every) == every) {
      int stop = 0;
      if ((threadIdx.x & 31) == 0) {
        if (*abort_flag) stop = 1;
        else if (g_ns() - t0 > limit_ns) {
          *abort_flag = 1;
          stop = 1;
        }
      }
      if (__shfl_sync(0xffffffffu, stop, 0)) return false;
    }
  }
}
__device__ __forceinline__ void g_fence_async() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }
__device__ __forceinline__ void g_tc_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void g_tc_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void g_commit(uint32_t bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar) : "memory");
}
__device__ __forceinline__ void g_mma(uint32_t dtmem, uint64_t adesc, uint64_t bdesc, uint32_t idesc, uint32_t acc) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
      " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(dtmem),
      "l"(adesc), "l"(bdesc), "r"(idesc), "r"(acc));
}
__device__ __forceinline__ void g_tmem_ld8(uint32_t taddr, float *v) {
  uint32_t r[8];
  asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%8];"
               : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7])
               : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int i = 0; i < 8; ++i) v[i] = __uint_as_float(r[i]);
}
// K-major, 128-byte rows, 128B swizzle, 8-row groups 1024 B apart.
__device__ __forceinline__ uint64_t g_desc(uint32_t saddr) {
  uint64_t desc = 0;
  desc |= (uint64_t)((saddr & 0x3FFFFu) >> 4);
  desc |= (uint64_t)1 << 16;
  desc |= (uint64_t)(1024 >> 4) << 32;
  desc |= (uint64_t)1 << 46;
  desc |= (uint64_t)2 << 61;
  return desc;
}
// kind::f16: D = F32, A = B = BF16, both K-major, M = 128, N = 128.
constexpr uint32_t kGIdesc = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(GBN >> 3) << 17) |
                             ((uint32_t)(GBM >> 4) << 24);

// The three BF16 terms of eight FP32 values, as packed BF16 pairs.
__device__ __forceinline__ void split3(const float (&x)[8], uint32_t (&w)[kTerms][4]) {
#pragma unroll
  for (int u = 0; u < 4; ++u) {
    float a = x[2 * u], b = x[2 * u + 1];
#pragma unroll
    for (int t = 0; t < kTerms; ++t) {
      __nv_bfloat162 h = __floats2bfloat162_rn(a, b);
      w[t][u] = *reinterpret_cast<uint32_t *>(&h);
      float2 back = __bfloat1622float2(h);
      a -= back.x;
      b -= back.y;
    }
  }
}

// The three BF16 terms of four FP32 values, as packed BF16 pairs.
__device__ __forceinline__ void split3_4(const float *x, uint32_t (&w)[kTerms][2]) {
#pragma unroll
  for (int u = 0; u < 2; ++u) {
    float a = x[2 * u], b = x[2 * u + 1];
#pragma unroll
    for (int t = 0; t < kTerms; ++t) {
      __nv_bfloat162 h = __floats2bfloat162_rn(a, b);
      w[t][u] = *reinterpret_cast<uint32_t *>(&h);
      float2 back = __bfloat1622float2(h);
      a -= back.x;
      b -= back.y;
    }
  }
}

// Row (within a warp's 32) of lane l's quad t in the coalesced K-major layout: the four rows
// of one step are r, r + 4, r + 1, r + 5, whose 128B-swizzled chunks fill both halves of the
// shared-memory banks (rows r..r+3 would all land in the same half).
__device__ __forceinline__ int kq_row(int t, int lane) {
  return 8 * (t >> 1) + 2 * (t & 1) + 4 * ((lane >> 3) & 1) + (lane >> 4);
}

// A 32-row x 32-K block of a K-major operand (element (row, k) at P[k + row * ld]) read so
// that each warp load touches four rows of 128 bytes: lane l takes K values k0 + 4 (l % 8)
// .. +3 of rows rbase + kq_row(t, l), t < 8, into x[4 t .. 4 t + 3] (zero past K or the last
// row).  Reading a whole row per lane instead made every load touch 32 lines and left the
// kernel bound by L1 throughput.
__device__ __forceinline__ void load_kmajor_c(const float *P, int64_t ld, int rbase, int rows, int k0, int K,
                                              bool vec, int lane, float (&x)[32]) {
  const int kk = k0 + 4 * (lane & 7);
#pragma unroll
  for (int t = 0; t < 8; ++t) {
    const int row = rbase + kq_row(t, lane);
    if (row < rows && vec && kk + 4 <= K) {
      const float4 v = *reinterpret_cast<const float4 *>(P + (int64_t)row * ld + kk);
      x[4 * t] = v.x; x[4 * t + 1] = v.y; x[4 * t + 2] = v.z; x[4 * t + 3] = v.w;
    } else {
#pragma unroll
      for (int u = 0; u < 4; ++u) x[4 * t + u] = (row < rows && kk + u < K) ? P[(int64_t)row * ld + kk + u] : 0.f;
    }
  }
}

// 32 consecutive K values of row `row` of a K-major operand (element (row, k) at
// P[k + row * ld]), zero past K or past the last row.
__device__ __forceinline__ void load_kmajor(const float *P, int64_t ld, int row, int rows, int k0, int K, bool vec,
                                            float (&x)[32]) {
  if (row < rows && vec && k0 + 32 <= K) {
    const float4 *p = reinterpret_cast<const float4 *>(P + (int64_t)row * ld + k0);
#pragma unroll
    for (int q = 0; q < 8; ++q) {
      float4 v = p[q];
      x[4 * q] = v.x; x[4 * q + 1] = v.y; x[4 * q + 2] = v.z; x[4 * q + 3] = v.w;
    }
  } else {
#pragma unroll
    for (int u = 0; u < 32; ++u) x[u] = (row < rows && k0 + u < K) ? P[(int64_t)row * ld + k0 + u] : 0.f;
  }
}
// The same for an M-major operand (element (row, k) at P[row + k * ld]): lanes take
// consecutive rows, so each of the 32 loads is coalesced across the warp.
__device__ __forceinline__ void load_mmajor(const float *P, int64_t ld, int row, int rows, int k0, int K,
                                            float (&x)[32]) {
#pragma unroll
  for (int u = 0; u < 32; ++u) x[u] = (row < rows && k0 + u < K) ? P[row + (int64_t)(k0 + u) * ld] : 0.f;
}

template <bool TRANSA>
__global__ void __launch_bounds__(kGThreads, 1)
    k_gemm_tc(int M, int N, int K, float alpha, const float *__restrict__ A, int64_t lda, int64_t sA,
              const float *__restrict__ B, int64_t ldb, int64_t sB, float beta, float *C, int64_t ldc, int64_t sC,
              int vecA, int vecB, int *err, uint64_t wait_ns) {
  extern __shared__ uint8_t smem_raw[];
  uint64_t *bars = reinterpret_cast<uint64_t *>(smem_raw);
  uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(bars + 8);
  volatile int *abort_flag = reinterpret_cast<volatile int *>(tmem_slot + 1);
  uint8_t *tiles = reinterpret_cast<uint8_t *>((reinterpret_cast<uintptr_t>(smem_raw) + 1024 + 1023) &
                                               ~(uintptr_t)1023);
  auto full = [&](int s) { return su32(bars + s); };
  auto empty = [&](int s) { return su32(bars + 2 + s); };
  const uint32_t accum_bar = su32(bars + 4);
  const uint32_t drain_bar = su32(bars + 5);
  auto a_tile = [&](int s, int t) { return su32(tiles + (size_t)s * kGStage + (size_t)t * kGTile); };
  auto b_tile = [&](int s, int t) { return su32(tiles + (size_t)s * kGStage + (size_t)(kTerms + t) * kGTile); };

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int b = blockIdx.z;
  A += (int64_t)b * sA;
  B += (int64_t)b * sB;
  C += (int64_t)b * sC;
  const int m0 = blockIdx.x * GBM, n0 = blockIdx.y * GBN;
  const int nkb = (K + GBK - 1) / GBK;

  if (threadIdx.x == 0) {
    for (int s = 0; s < kGStages; ++s) {
      g_mbar_init(full(s), kGProducers);
      g_mbar_init(empty(s), 1);
    }
    g_mbar_init(accum_bar, 1);
    g_mbar_init(drain_bar, 1);
    *abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 1) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(su32(tmem_slot)),
                 "r"((uint32_t)GBN));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  g_tc_before();
  __syncthreads();
  g_tc_after();
  const uint32_t tmem = *tmem_slot;

  if (warp == 1) {
    if (lane == 0) {
      bool good = true;
      int issued = 0;
      // the six term products of order <= 2, small ones first
      const int ta[kPairs] = {2, 1, 0, 1, 0, 0}, tb[kPairs] = {0, 1, 2, 0, 1, 0};
      for (int kb = 0; kb < nkb; ++kb) {
        const int s = kb % kGStages;
        const uint32_t ph = (uint32_t)(kb / kGStages) & 1u;
        if (!g_wait(full(s), ph, abort_flag, wait_ns)) {
          good = false;
          break;
        }
        g_tc_after();
#pragma unroll
        for (int kk = 0; kk < GBK / 16; ++kk)
#pragma unroll
          for (int q = 0; q < kPairs; ++q) {
            const uint64_t ad = g_desc(a_tile(s, ta[q])) + 2 * kk;   // +32 bytes per K step
            const uint64_t bd = g_desc(b_tile(s, tb[q])) + 2 * kk;
            g_mma(tmem, ad, bd, kGIdesc, (kb > 0 || kk > 0 || q > 0) ? 1u : 0u);
          }
        g_commit(empty(s));
        ++issued;
      }
      if (good) g_commit(accum_bar);
      if (issued > 0) {
        volatile int never = 0;
        g_commit(drain_bar);
        g_wait(drain_bar, 0u, &never, kDefaultWaitNs);   // the MMAs always drain
      }
    }
    __syncwarp();
  } else if (warp >= 2) {
    // producer warp pw: tile rows 32 (pw % 4) + lane, K half pw / 4 of every block
    const int pw = warp - 2;
    const int r = (pw & 3) * 32 + lane;
    const int h = pw >> 2;
    const uint32_t rowoff = (uint32_t)r * 128u;
    bool good = true;
    // both operands of block kb + 1 are loaded while block kb is stored and the MMAs of the
    // previous stage run, so neither load's latency sits between two stages
    float xa[32], xb[32];
    const int rb = (pw & 3) * 32;                  // this warp's 32 tile rows
    auto load_block = [&](int kb) {
      const int k0 = kb * GBK + h * 32;
      if (TRANSA) load_kmajor_c(A, lda, m0 + rb, M, k0, K, vecA != 0, lane, xa);   // rows of op(A)
      else load_mmajor(A, lda, m0 + r, M, k0, K, xa);
      load_kmajor_c(B, ldb, n0 + rb, N, k0, K, vecB != 0, lane, xb);               // columns of B
    };
    // a whole row's 32 K values (M-major loads): four 16-byte chunks per term
    auto store_row = [&](const float (&x)[32], uint32_t tile0) {
#pragma unroll
      for (int c = 0; c < 4; ++c) {
        float v[8];
#pragma unroll
        for (int u = 0; u < 8; ++u) v[u] = x[8 * c + u];
        uint32_t w[kTerms][4];
        split3(v, w);
        const uint32_t off = rowoff + ((((uint32_t)(h * 4 + c)) ^ ((uint32_t)r & 7u)) << 4);
#pragma unroll
        for (int t = 0; t < kTerms; ++t)
          asm volatile("st.shared.v4.b32 [%0], {%1, %2, %3, %4};" ::"r"(tile0 + t * kGTile + off), "r"(w[t][0]),
                       "r"(w[t][1]), "r"(w[t][2]), "r"(w[t][3])
                       : "memory");
      }
    };
    // eight rows x 4 K values (coalesced K-major loads): half of a 16-byte chunk per term and row
    auto store_quads = [&](const float (&x)[32], uint32_t tile0) {
      const uint32_t chunk = (uint32_t)(h * 4 + ((lane & 7) >> 1)), half = (uint32_t)(lane & 1) * 8u;
#pragma unroll
      for (int t = 0; t < 8; ++t) {
        const uint32_t row = (uint32_t)(rb + kq_row(t, lane));
        uint32_t w[kTerms][2];
        split3_4(&x[4 * t], w);
        const uint32_t off = row * 128u + ((chunk ^ (row & 7u)) << 4) + half;
#pragma unroll
        for (int q = 0; q < kTerms; ++q)
          asm volatile("st.shared.v2.b32 [%0], {%1, %2};" ::"r"(tile0 + q * kGTile + off), "r"(w[q][0]), "r"(w[q][1])
                       : "memory");
      }
    };
    if (nkb > 0) load_block(0);
    for (int kb = 0; kb < nkb; ++kb) {
      const int s = kb % kGStages;
      const uint32_t ph = (uint32_t)(kb / kGStages) & 1u;
      if (!g_wait_lanes(empty(s), ph ^ 1u, abort_flag, wait_ns)) { good = false; break; }
      if (TRANSA) store_quads(xa, a_tile(s, 0));
      else store_row(xa, a_tile(s, 0));
      store_quads(xb, b_tile(s, 0));
      g_fence_async();
      g_mbar_arrive(full(s));
      if (kb + 1 < nkb) load_block(kb + 1);
    }
    // epilogue: TMEM lane quadrant warp % 4, columns split between the two warps of a quadrant
    if (good && nkb > 0 && g_wait_lanes(accum_bar, 0u, abort_flag, wait_ns)) {
      g_tc_after();
      const int q = warp & 3;
      const int m = m0 + q * 32 + lane;
      for (int j = (pw >> 2) * 64; j < (pw >> 2) * 64 + 64; j += 8) {
        float v[8];
        g_tmem_ld8(tmem + ((uint32_t)(q * 32) << 16) + (uint32_t)j, v);
        if (m < M) {
#pragma unroll
          for (int t = 0; t < 8; ++t) {
            const int n = n0 + j + t;
            if (n < N) {
              float *c = C + m + (int64_t)n * ldc;
              *c = alpha * v[t] + (beta == 0.f ? 0.f : beta * *c);
            }
          }
        }
      }
    }
  }
  g_tc_before();
  __syncthreads();
  if (*abort_flag && threadIdx.x == 0) atomicOr(err, DERR_TIMEOUT);
  if (warp == 1) {
    g_tc_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"((uint32_t)GBN));
  }
}

}  // namespace

Error gemm_tc_f32(const ckinv_ctx *ctx, bool transA, int M, int N, int K, float alpha, const float *A, int64_t lda,
                  int64_t sA, const float *B, int64_t ldb, int64_t sB, float beta, float *C, int64_t ldc, int64_t sC,
                  int batch, cudaStream_t st) {
  if (M <= 0 || N <= 0 || batch <= 0) return ok();
  if (batch > 65535) return fail(CKINV_EUNSUPPORTED, "gemm_tc: batch above 65535");
  // 16-byte vector loads of K-major rows when every row start is 16-byte aligned
  auto aligned = [](const float *p, int64_t ld, int64_t s, int nb) {
    return (reinterpret_cast<uintptr_t>(p) & 15) == 0 && ld % 4 == 0 && (nb == 1 || s % 4 == 0);
  };
  const int vecA = transA && aligned(A, lda, sA, batch);
  const int vecB = aligned(B, ldb, sB, batch);
  dim3 grid((unsigned)ceil_div(M, GBM), (unsigned)ceil_div(N, GBN), (unsigned)batch);
  note_launch();
  if (transA) {
    CK_CUDA(cudaFuncSetAttribute(k_gemm_tc<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kGSmem));
    k_gemm_tc<true><<<grid, kGThreads, kGSmem, st>>>(M, N, K, alpha, A, lda, sA, B, ldb, sB, beta, C, ldc, sC, vecA,
                                                     vecB, ctx->d_err, ctx->wait_ns);
  } else {
    CK_CUDA(cudaFuncSetAttribute(k_gemm_tc<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kGSmem));
    k_gemm_tc<false><<<grid, kGThreads, kGSmem, st>>>(M, N, K, alpha, A, lda, sA, B, ldb, sB, beta, C, ldc, sC, vecA,
                                                      vecB, ctx->d_err, ctx->wait_ns);
  }
  CK_CUDA(cudaGetLastError());
  return ok();
}

}  // namespace ckinv
