// Fused sketch Y = K0 Omega (Sec. 3.1-3.3) on the 5th-generation tensor cores.
//
// The CTAs run in pairs (clusters of two) that share each MMA: a pair owns 256 rows of Y
// (128 per CTA) and all d <= 512 columns, its FP32 accumulator in TMEM (128 lanes x d
// columns in each CTA).  The contraction runs over the n points in blocks of BK = 64:
//   * warps 2..9 of each CTA evaluate its 128 x 64 kernel tile in FP32 (exp2 on the MUFU)
//     from the block's points, split it into 1-3 BF16 terms and store them straight into
//     the 128B-swizzled K-major SMEM layout the MMA reads (no HBM traffic for K0 at all);
//   * warp 0, lane 0 of each CTA bulk-copies the raw coordinates of upcoming blocks into a
//     shared ring and fetches by TMA its half of the block's 64 x d tile of the +-1 Omega
//     pattern (BF16, exact);
//   * warp 1, lane 0 of the first CTA issues tcgen05.mma.cta_group::2 (M = 256, N <= 256 per
//     instruction, K = 16) once both CTAs' tiles of a stage are ready - the second CTA's
//     warp 1 relays its readiness with one cluster-scope arrival - and commits each stage
//     back to both CTAs' producers through mbarriers;
//   * after the last block, warps 2..9 read TMEM with tcgen05.ld, scale by variance * c and
//     write Y (coalesced along rows: Y is column-major).
// MODE 1 takes the A operand from a dense FP32 matrix instead of evaluating kernel entries
// (a materialised K, and the products B = Omega^T Q_hat and Omega^T Y' of the core and the
// gradient).  Every mbarrier wait is bounded (the context's limit for waits on another
// role's progress, one second for the CTA's own copies and MMAs to drain); on timeout the
// CTA records DERR_TIMEOUT, drains its own copies and MMAs, frees TMEM and returns.
#include <cuda.h>
#include <cudaTypedefs.h>
#include <cstring>

#include "internal.cuh"

namespace ckinv {
namespace {

constexpr int BM = 128;
constexpr int BK = 64;                  // points per pipeline stage
constexpr uint32_t kRowBytes = BK * 2;  // one K-major row of a BF16 tile: 128 B, 128B-swizzled
constexpr int kProducerWarps = 8;       // warps 2 .. 9
constexpr int kRowsPerLane = 1;         // tile rows per producer lane
constexpr int kPtSlots = 12;            // shared-memory slots of raw block coordinates (>= stages + 4)
constexpr uint32_t kPtSlotBytes = BK * 3 * 4;   // one block of up to 3-D points
constexpr int kKParts = kProducerWarps / 4;   // epilogue warps sharing one 32-row TMEM quadrant
constexpr int kThreads = 64 + 32 * kProducerWarps;
constexpr uint32_t kATileBytes = BM * BK * 2;  // 16 KB per BF16 term
static_assert(kProducerWarps % 4 == 0, "epilogue split");

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
__device__ __forceinline__ bool mbar_try_wait(uint32_t bar, uint32_t parity, uint32_t hint_ns) {
  uint32_t ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, %3;\n"
      " selp.b32 %0, 1, 0, p;\n}\n"
      : "=r"(ok)
      : "r"(bar), "r"(parity), "r"(hint_ns)
      : "memory");
  return ok != 0;
}
// The same with cluster-scope acquire, for barriers that threads of the peer CTA arrive on.
__device__ __forceinline__ bool mbar_try_wait_cl(uint32_t bar, uint32_t parity, uint32_t hint_ns) {
  uint32_t ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.acquire.cluster.shared::cta.b64 p, [%1], %2, %3;\n"
      " selp.b32 %0, 1, 0, p;\n}\n"
      : "=r"(ok)
      : "r"(bar), "r"(parity), "r"(hint_ns)
      : "memory");
  return ok != 0;
}
__device__ __forceinline__ uint64_t global_ns() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}
// Limit of a wait, in ns: the context's limit for waits on another role's progress (a kernel
// parameter, read where it is used so that the hot loops keep no register for it), the
// default second for waits on the CTA's own copies and MMAs to drain.  Every poll suspends
// for up to 20 us, or not at all under a limit below 100 us, whose loop then reads the clock
// after every poll so that it runs out after about its own length.
__device__ __forceinline__ uint32_t wait_hint(uint64_t limit_ns) { return limit_ns < 100000ull ? 0u : 20000u; }
// Bounded wait: gives up after the limit or when another warp has flagged an abort.  The
// first poll is inline; the loop is not.
__device__ __noinline__ bool mbar_wait_slow(uint32_t bar, uint32_t parity, volatile int *abort_flag,
                                            bool cluster_scope, uint64_t limit_ns) {
  const uint64_t t0 = global_ns();
  const uint32_t hint = wait_hint(limit_ns);
  const uint32_t every = hint ? 15u : 0u;
  for (uint32_t it = 0;; ++it) {
    if (cluster_scope ? mbar_try_wait_cl(bar, parity, hint) : mbar_try_wait(bar, parity, hint)) return true;
    if ((it & every) == every) {
      if (*abort_flag) return false;
      if (global_ns() - t0 > limit_ns) {
        *abort_flag = 1;
        return false;
      }
    }
  }
}
__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity, volatile int *abort_flag,
                                          bool cluster_scope, uint64_t limit_ns) {
  const uint32_t hint = wait_hint(limit_ns);
  if (cluster_scope ? mbar_try_wait_cl(bar, parity, hint) : mbar_try_wait(bar, parity, hint)) return true;
  return mbar_wait_slow(bar, parity, abort_flag, cluster_scope, limit_ns);
}

// Warp-wide bounded wait: every lane polls, so that each lane acquires the phase itself (no
// __syncwarp, whose memory ordering costs ~200 clocks), and the warp leaves together.
__device__ __noinline__ bool mbar_wait_lanes_slow(uint32_t bar, uint32_t parity, volatile int *abort_flag,
                                                   uint64_t limit_ns) {
  const uint32_t hint = wait_hint(limit_ns);
  const uint64_t t0 = global_ns();
  const uint32_t every = hint ? 15u : 0u;
  for (uint32_t it = 0;; ++it) {
    if (__all_sync(0xffffffffu, mbar_try_wait(bar, parity, hint))) return true;
    if ((it & every) == every) {
      int stop = 0;
      if ((threadIdx.x & 31) == 0) {
        if (*abort_flag) stop = 1;
        else if (global_ns() - t0 > limit_ns) {
          *abort_flag = 1;
          stop = 1;
        }
      }
      if (__shfl_sync(0xffffffffu, stop, 0)) return false;
    }
  }
}
__device__ __forceinline__ bool mbar_wait_lanes(uint32_t bar, uint32_t parity, volatile int *abort_flag,
                                                uint64_t limit_ns) {
  if (__all_sync(0xffffffffu, mbar_try_wait(bar, parity, wait_hint(limit_ns)))) return true;
  return mbar_wait_lanes_slow(bar, parity, abort_flag, limit_ns);
}
// Contiguous bulk copy global -> shared (async proxy), completion counted on an mbarrier;
// both addresses 16-byte aligned, bytes a multiple of 16.
__device__ __forceinline__ void bulk_load(uint32_t dst, const void *src, uint32_t bytes, uint32_t bar) {
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(dst),
               "l"(src), "r"(bytes), "r"(bar)
               : "memory");
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
__device__ __forceinline__ uint32_t cluster_rank() {
  uint32_t r;
  asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
  return r;
}
__device__ __forceinline__ void cluster_sync_all() {
  asm volatile("barrier.cluster.arrive.release.aligned;\nbarrier.cluster.wait.acquire.aligned;" ::: "memory");
}
__device__ __forceinline__ void tc_fence_before() {
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void tc_fence_after() {
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}
// Arrive on the mbarrier at this offset in each CTA of the pair named by ctaMask once all
// prior MMAs of the pair are done.
__device__ __forceinline__ void tc_commit_pair(uint32_t bar, uint16_t mask) {
  asm volatile(
      "tcgen05.commit.cta_group::2.mbarrier::arrive::one.shared::cluster.multicast::cluster.b64 [%0], %1;" ::"r"(bar),
      "h"(mask)
      : "memory");
}
// D[256 x N] (+)= A[256 x 16] B[16 x N] over the CTA pair: A rows 0-127 and B columns
// 0 .. N/2-1 from this CTA's shared memory, the rest from the peer's at the same offsets;
// D rows 0-127 in this CTA's TMEM, 128-255 in the peer's.
__device__ __forceinline__ void tc_mma_pair(uint32_t dtmem, uint64_t adesc, uint64_t bdesc, uint32_t idesc,
                                            uint32_t accum) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
      " tcgen05.mma.cta_group::2.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(dtmem),
      "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accum));
}
// Shared::cluster address of the same shared-memory offset in CTA `rank` of the cluster.
__device__ __forceinline__ uint32_t map_to_rank(uint32_t saddr, uint32_t rank) {
  uint32_t r;
  asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(r) : "r"(saddr), "r"(rank));
  return r;
}
__device__ __forceinline__ void mbar_arrive_remote(uint32_t cluster_addr) {
  asm volatile("mbarrier.arrive.release.cluster.shared::cluster.b64 _, [%0];" ::"r"(cluster_addr) : "memory");
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

// SMEM matrix descriptor: K-major rows of kRowBytes, swizzled by the matching mode,
// 8-row groups 8 * kRowBytes apart.
__device__ __forceinline__ uint64_t sw_desc(uint32_t saddr) {
  constexpr uint64_t layout = (kRowBytes == 128) ? 2 : (kRowBytes == 64 ? 4 : 6);   // 128B / 64B / 32B
  uint64_t desc = 0;
  desc |= (uint64_t)((saddr & 0x3FFFFu) >> 4);        // start address
  desc |= (uint64_t)1 << 16;                          // leading byte offset (unused)
  desc |= (uint64_t)((8 * kRowBytes) >> 4) << 32;     // stride byte offset
  desc |= (uint64_t)1 << 46;                          // descriptor version (sm_100 family)
  desc |= layout << 61;                               // swizzle mode
  return desc;
}
// Physical 16-byte chunk of logical chunk c in row r under that swizzle.
__device__ __forceinline__ uint32_t swz_chunk(uint32_t c, uint32_t r) {
  return (kRowBytes == 128) ? (c ^ (r & 7u)) : (kRowBytes == 64 ? (c ^ ((r >> 1) & 3u)) : (c ^ ((r >> 2) & 1u)));
}
// Instruction descriptor, kind::f16: D = F32, A = B = BF16, both K-major, M = 256 (pair).
__host__ __device__ constexpr uint32_t idesc_bf16(int N) {
  return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)((2 * BM) >> 4) << 24);
}

struct TcArgs {
  int64_t n;       // contraction length (points)
  int64_t m;       // output rows (dense mode: rows of A; kernel mode: points row0 .. row0 + m - 1)
  int64_t row0;    // kernel mode: first point of the output rows
  int dim;
  int d;
  int num_kb;      // BK-point blocks in total
  int kb_per_cta;  // blocks per CTA along the contraction (split over gridDim.y)
  int stages;
  int n0, n1;      // N of the first and second MMA column chunk (n1 = 0: a single chunk)
  int box_rows;    // rows of Omega^T per TMA box (divides n0 / 2 and n1 / 2)
  KernelParams kp;
  const float *pts;
  const float *A;  // dense mode: row i of A at A + i * lda (K-major)
  int64_t lda;
  float *Y;        // store mode: Y = scale * acc (column-major, ld ldy)
  int64_t ldy;
  float *part;     // partial mode: part[split][i + j * ldp] = acc (+= when accumulate)
  int64_t ldp;
  int accumulate;
  int *err;
  uint64_t wait_ns;  // limit of the waits on another role's progress
};

// MODE 0: A = kernel tile evaluated from the points;  MODE 1: A = a dense FP32 matrix.
// KIND is the covariance function of MODE 0 (fixed at compile time so that the inner
// loop carries no branch).
template <int NSPLIT, bool DERIV, int MODE, int KIND>
__global__ void __launch_bounds__(kThreads, 1)
    k_sketch_tc(const __grid_constant__ CUtensorMap tmapB, const TcArgs a) {
  extern __shared__ uint8_t smem_raw[];
  // layout: [barriers | tmem slot | abort flag][per-warp point buffers] then the
  // 1024-aligned stage tiles
  uint64_t *bars = reinterpret_cast<uint64_t *>(smem_raw);
  const int S = a.stages;
  uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(bars + 34 + kPtSlots);
  volatile int *abort_flag = reinterpret_cast<volatile int *>(tmem_slot + 1);
  const float *pt_slots = reinterpret_cast<const float *>(smem_raw + 512);   // kPtSlots blocks of raw points
  uintptr_t tiles_u =
      (reinterpret_cast<uintptr_t>(smem_raw) + 512 + kPtSlots * kPtSlotBytes + 1023) & ~(uintptr_t)1023;
  uint8_t *tiles = reinterpret_cast<uint8_t *>(tiles_u);
  // this CTA's half of the Omega tile: n0/2 rows of chunk 0, then n1/2 rows of chunk 1
  const uint32_t b_bytes = (uint32_t)(a.n0 + a.n1) / 2 * kRowBytes;
  const uint32_t stage_bytes = NSPLIT * kATileBytes + b_bytes;
  const uint32_t b1_off = (uint32_t)(a.n0 / 2) * kRowBytes;
  const uint32_t rank = cluster_rank();       // 0: the CTA that issues the pair's MMAs

  // full: this CTA's A tiles are written (one arrival per producer thread) and its Omega
  //   half has landed (the TMA thread's expect-tx arrival plus the bytes);
  // peerB (rank 0): the peer's A tiles and Omega half are ready (one cluster-scope arrival
  //   from the peer, made by a thread that does nothing else);
  // empty: the pair's MMAs are done with the stage (committed to both CTAs).
  auto full = [&](int s) { return smem_u32(bars + s); };
  auto empty = [&](int s) { return smem_u32(bars + 16 + s); };
  auto peerB = [&](int s) { return smem_u32(bars + 24 + s); };
  const uint32_t accum_bar = smem_u32(bars + 32);
  const uint32_t drain_bar = smem_u32(bars + 33);
  // fullP(j): the raw coordinates of the block in point slot j have landed
  auto fullP = [&](int j) { return smem_u32(bars + 34 + j); };
  auto pt_slot = [&](int j) { return smem_u32(pt_slots) + (uint32_t)j * kPtSlotBytes; };
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
      mbar_init(full(s), 32 * kProducerWarps + 1);
      mbar_init(empty(s), 1);
      mbar_init(peerB(s), 1);
    }
    for (int j = 0; j < kPtSlots; ++j) mbar_init(fullP(j), 1);
    mbar_init(accum_bar, 1);
    mbar_init(drain_bar, 1);
    *abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 1) {
    // collective over the pair: one warp of each CTA, the same columns in both
    asm volatile("tcgen05.alloc.cta_group::2.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     smem_u32(tmem_slot)),
                 "r"(tmem_cols));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::2.sync.aligned;");
  }
  tc_fence_before();
  cluster_sync_all();   // every barrier of the cluster is initialised before any remote arrival
  tc_fence_after();
  const uint32_t tmem_base = *tmem_slot;
  // limits: a.wait_ns for waits on another role's progress, kDefaultWaitNs for this CTA's
  // own copies and MMAs to land

  if (warp == 0) {
    // ------------------------------------------------------------ TMA producer (Omega)
    if (lane == 0) {
      // Points: the raw coordinates of block kb go to slot kb % kPtSlots, L = kPtSlots - S
      // blocks ahead of the stage being fetched. The slot's previous block (kb - S) was read
      // by the producers before they released its stage, which the empty wait below
      // observes, so the slot is free when the copy is issued.
      const int L = kPtSlots - S;
      auto issue_points = [&](int kb) {
        if (MODE != 0 || kb >= nkb) return;
        const int j = kb % kPtSlots;
        const int64_t k0 = (int64_t)(kb_begin + kb) * BK;
        if (k0 + BK <= a.n) {
          const uint32_t bytes = (uint32_t)(BK * a.dim * 4);
          mbar_arrive_expect_tx(fullP(j), bytes);
          bulk_load(pt_slot(j), a.pts + k0 * a.dim, bytes, fullP(j));
        } else {
          mbar_arrive(fullP(j));     // the last, partial block: producers read global memory
        }
      };
      for (int kb = 0; kb < L; ++kb) issue_points(kb);
      // this CTA fetches its half of each column chunk: rows c n0 + rank n_c/2 + [0, n_c/2)
      int issued = 0, pts_issued = L;
      for (int kb = 0; kb < nkb; ++kb) {
        int s = kb % S;
        uint32_t ph = (uint32_t)(kb / S) & 1u;
        if (!mbar_wait(empty(s), ph ^ 1u, abort_flag, false, a.wait_ns)) break;
        issue_points(kb + L);
        pts_issued = kb + L + 1;
        mbar_arrive_expect_tx(full(s), b_bytes);
        const int kx = (kb_begin + kb) * BK;
        const int h0 = a.n0 / 2, h1 = a.n1 / 2;
        for (int o = 0; o < h0; o += a.box_rows)
          tma_load_2d(b_tile(s) + (uint32_t)o * kRowBytes, &tmapB, full(s), kx, (int)rank * h0 + o);
        for (int o = 0; o < h1; o += a.box_rows)
          tma_load_2d(b_tile(s) + b1_off + (uint32_t)o * kRowBytes, &tmapB, full(s), kx, a.n0 + (int)rank * h1 + o);
        ++issued;
      }
      // every copy this CTA issued must land before shared memory is released
      volatile int never = 0;
      int first = issued - S < 0 ? 0 : issued - S;
      for (int kb = first; kb < issued; ++kb)
        mbar_wait(full(kb % S), (uint32_t)(kb / S) & 1u, &never, false, kDefaultWaitNs);
      if (MODE == 0) {
        const int last = min(pts_issued, nkb);
        for (int kb = max(0, last - kPtSlots); kb < last; ++kb)
          mbar_wait(fullP(kb % kPtSlots), (uint32_t)(kb / kPtSlots) & 1u, &never, false, kDefaultWaitNs);
      }
    }
    __syncwarp();
  } else if (warp == 1) {
    // ------------------------------------------------------------ MMA issuer (rank 0)
    if (lane == 0 && rank == 0) {
      const uint32_t id0 = idesc_bf16(a.n0);
      const uint32_t id1 = idesc_bf16(a.n1 > 0 ? a.n1 : 16);
      bool good = true;
      int issued = 0;
      for (int kb = 0; kb < nkb; ++kb) {
        int s = kb % S;
        uint32_t ph = (uint32_t)(kb / S) & 1u;
        if (!mbar_wait(full(s), ph, abort_flag, false, a.wait_ns) || !mbar_wait(peerB(s), ph, abort_flag, true, a.wait_ns)) {
          good = false;
          break;
        }
        tc_fence_after();
        // a K step of 16 elements (32 bytes) adds 2 to the descriptor's start-address field
        const uint64_t b0 = sw_desc(b_tile(s)), b1 = sw_desc(b_tile(s) + b1_off);
#pragma unroll
        for (int t = 0; t < NSPLIT; ++t) {
          const uint64_t a0 = sw_desc(a_tile(s, t));
#pragma unroll
          for (int kk = 0; kk < BK / 16; ++kk) {
            uint32_t acc = (kb > 0 || t > 0 || kk > 0) ? 1u : 0u;
            tc_mma_pair(tmem_base, a0 + 2 * kk, b0 + 2 * kk, id0, acc);
            if (a.n1 > 0) tc_mma_pair(tmem_base + (uint32_t)a.n0, a0 + 2 * kk, b1 + 2 * kk, id1, acc);
          }
        }
        tc_commit_pair(empty(s), 0x3);
        ++issued;
      }
      if (good) tc_commit_pair(accum_bar, 0x3);
      if (issued > 0) {
        // all MMAs of the pair must finish before either CTA releases TMEM or shared memory
        volatile int never = 0;
        tc_commit_pair(drain_bar, 0x1);
        mbar_wait(drain_bar, 0u, &never, false, kDefaultWaitNs);
      }
    } else if (lane == 0) {
      // rank 1: tell the MMA issuer when this CTA's A tiles and Omega half of each stage are
      // ready (acquire here, release at cluster scope to rank 0)
      const uint32_t peer_bar0 = map_to_rank(peerB(0), 0);
      for (int kb = 0; kb < nkb; ++kb) {
        int s = kb % S;
        uint32_t ph = (uint32_t)(kb / S) & 1u;
        if (!mbar_wait(full(s), ph, abort_flag, false, a.wait_ns)) break;
        mbar_arrive_remote(peer_bar0 + 8u * (uint32_t)s);
      }
    }
    __syncwarp();
  } else {
    // ------------------------------------------------------------ A-tile producers
    // Lane l of producer warp pw owns the kRowsPerLane tile rows l + 32 j (+ the warp's row
    // group) and, of every block, the KH points of k-part h: each staged point is read
    // once from shared memory and used for kRowsPerLane kernel entries.
    constexpr int RG = BM / (32 * kRowsPerLane);   // row groups
    constexpr int KP = kProducerWarps / RG;        // k-parts
    constexpr int KH = BK / KP;                    // points per k-part
    constexpr int CH = KH / 8;                     // 16-byte chunks per k-part and row
    static_assert(RG * KP == kProducerWarps && KH % 8 == 0 && KH <= 32, "producer layout");
    const int pw = warp - 2;
    const int g = pw % RG, h = pw / RG;
    const int64_t rows_total = a.m;
    const float cs = a.kp.coord_scale;
    const float inv_l = a.kp.inv_l;
    float xr[kRowsPerLane][3];
    const float *arow[kRowsPerLane];
    bool rok[kRowsPerLane];
#pragma unroll
    for (int j = 0; j < kRowsPerLane; ++j) {
      const int r = g * 32 * kRowsPerLane + j * 32 + lane;
      const int64_t irow = min(i0 + r, rows_total - 1);
      xr[j][0] = xr[j][1] = xr[j][2] = 0.f;
      if (MODE == 0) {
        const int64_t ip = a.row0 + irow;
        xr[j][0] = a.pts[ip * a.dim] * cs;
        if (a.dim > 1) xr[j][1] = a.pts[ip * a.dim + 1] * cs;
        if (a.dim > 2) xr[j][2] = a.pts[ip * a.dim + 2] * cs;
      }
      arow[j] = (MODE == 1) ? a.A + irow * a.lda : nullptr;
      rok[j] = (i0 + r < rows_total);
    }
    // rows l + 32 j share l mod 8, hence the swizzle of their 16-byte chunks
    const uint32_t lane_base = (uint32_t)(g * 32 * kRowsPerLane + lane) * kRowBytes;
    bool good = true;
    // one block: wait for its points and for the stage, fill the stage's A tiles
    // dense mode: the 32 entries of this lane's row for block kb, into nxt (zero past n)
    float nxt[kRowsPerLane][CH * 8];
    auto load_dense = [&](int kb) {
      const int64_t kbase = (int64_t)(kb_begin + kb) * BK + h * KH;
#pragma unroll
      for (int r = 0; r < kRowsPerLane; ++r) {
#pragma unroll
        for (int c = 0; c < CH; ++c) {
          const int64_t k0 = kbase + c * 8;
          if (rok[r] && k0 + 8 <= a.n) {
            const float4 lo = *reinterpret_cast<const float4 *>(arow[r] + k0);
            const float4 hi = *reinterpret_cast<const float4 *>(arow[r] + k0 + 4);
            nxt[r][c * 8 + 0] = lo.x; nxt[r][c * 8 + 1] = lo.y; nxt[r][c * 8 + 2] = lo.z; nxt[r][c * 8 + 3] = lo.w;
            nxt[r][c * 8 + 4] = hi.x; nxt[r][c * 8 + 5] = hi.y; nxt[r][c * 8 + 6] = hi.z; nxt[r][c * 8 + 7] = hi.w;
          } else {
#pragma unroll
            for (int u = 0; u < 8; ++u) nxt[r][c * 8 + u] = (rok[r] && k0 + u < a.n) ? arow[r][k0 + u] : 0.0f;
          }
        }
      }
    };
    if (MODE == 1 && nkb > 0) load_dense(0);
    auto produce = [&](int kb) -> bool {
      int s = kb % S;
      uint32_t ph = (uint32_t)(kb / S) & 1u;
      const int64_t kbase = (int64_t)(kb_begin + kb) * BK + h * KH;
      const bool full_block = ((int64_t)(kb_begin + kb) * BK + BK <= a.n);
      const int j = kb % kPtSlots;
      if (MODE == 0 && !mbar_wait_lanes(fullP(j), (uint32_t)(kb / kPtSlots) & 1u, abort_flag, a.wait_ns)) return false;
      if (!mbar_wait_lanes(empty(s), ph ^ 1u, abort_flag, a.wait_ns)) return false;
      const float *ps = pt_slots + (size_t)j * (kPtSlotBytes / 4) + (size_t)h * KH * a.dim;
      // Phase 1: all CH * 8 entries of this lane's rows (no shared-memory store in between,
      // so that the loads and the arithmetic of different entries overlap freely).
      float kv[kRowsPerLane][CH * 8];
      if (MODE == 0) {
        // differences in scaled coordinates: x cs - p cs, with p raw and x pre-scaled
        if (full_block && a.dim == 2) {
#pragma unroll
          for (int u = 0; u < CH * 8; u += 2) {
            const float4 p2 = *reinterpret_cast<const float4 *>(ps + u * 2);   // points u, u + 1
#pragma unroll
            for (int r = 0; r < kRowsPerLane; ++r) {
              float dx = fmaf(-cs, p2.x, xr[r][0]), dy = fmaf(-cs, p2.y, xr[r][1]);
              kv[r][u] = dev::kernel_value(KIND, fmaf(dy, dy, dx * dx), inv_l, DERIV);
              dx = fmaf(-cs, p2.z, xr[r][0]);
              dy = fmaf(-cs, p2.w, xr[r][1]);
              kv[r][u + 1] = dev::kernel_value(KIND, fmaf(dy, dy, dx * dx), inv_l, DERIV);
            }
          }
        } else {
          // other dimensions, or the last, partial block (points from global memory, zero
          // past n)
#pragma unroll
          for (int u = 0; u < CH * 8; ++u) {
            const int64_t k = kbase + u;
            const bool valid = full_block || k < a.n;
            const float *q = full_block ? ps + u * a.dim : a.pts + (valid ? k : 0) * a.dim;
            const float px = q[0], py = a.dim > 1 ? q[1] : 0.f, pz = a.dim > 2 ? q[2] : 0.f;
#pragma unroll
            for (int r = 0; r < kRowsPerLane; ++r) {
              float dx = fmaf(-cs, px, xr[r][0]), dy = fmaf(-cs, py, xr[r][1]), dz = fmaf(-cs, pz, xr[r][2]);
              float v = dev::kernel_value(KIND, fmaf(dz, dz, fmaf(dy, dy, dx * dx)), inv_l, DERIV);
              kv[r][u] = valid ? v : 0.0f;
            }
          }
        }
      } else {
        // dense mode: this block's rows of A were loaded while the previous block was stored;
        // the next block's loads go out now and land during this block's stores and waits
#pragma unroll
        for (int r = 0; r < kRowsPerLane; ++r)
#pragma unroll
          for (int u = 0; u < CH * 8; ++u) kv[r][u] = nxt[r][u];
        if (kb + 1 < nkb) load_dense(kb + 1);
      }
      // Phase 2: split into BF16 terms and store each 16-byte chunk at its swizzled place.
      uint8_t *stage_base = tiles + (size_t)s * stage_bytes;
#pragma unroll
      for (int c = 0; c < CH; ++c) {
        const uint32_t off = lane_base + (swz_chunk((uint32_t)(h * CH + c), (uint32_t)lane) << 4);
#pragma unroll
        for (int r = 0; r < kRowsPerLane; ++r) {
#pragma unroll
          for (int t = 0; t < NSPLIT; ++t) {
            uint32_t w[4];
#pragma unroll
            for (int u = 0; u < 4; ++u) {
              __nv_bfloat162 b2 = __floats2bfloat162_rn(kv[r][c * 8 + 2 * u], kv[r][c * 8 + 2 * u + 1]);
              w[u] = *reinterpret_cast<uint32_t *>(&b2);
              if (t + 1 < NSPLIT) {
                float2 back = __bfloat1622float2(b2);
                kv[r][c * 8 + 2 * u] -= back.x;
                kv[r][c * 8 + 2 * u + 1] -= back.y;
              }
            }
            *reinterpret_cast<uint4 *>(stage_base + (size_t)t * kATileBytes + off + (uint32_t)(r * 32) * kRowBytes) =
                make_uint4(w[0], w[1], w[2], w[3]);
          }
        }
      }
      fence_async_smem();                  // this thread's tile writes -> visible to the tensor core
      mbar_arrive(full(s));
      return true;
    };
    for (int kb = 0; kb < nkb; ++kb) {
      if (!produce(kb)) { good = false; break; }
    }
    // ------------------------------------------------------------ epilogue
    bool e_ok = good && nkb > 0 && mbar_wait_lanes(accum_bar, 0u, abort_flag, a.wait_ns);
    if (e_ok) {
      tc_fence_after();
      const int q = warp & 3;                 // TMEM lane quadrant this warp may access
      const int part = pw >> 2;               // kKParts warps per quadrant split the columns
      const int64_t i = i0 + q * 32 + lane;
      const float scale = (float)a.kp.scale;
      const int64_t mrows = a.m;
      float *pout = a.part ? a.part + (int64_t)blockIdx.y * a.ldp * a.d : nullptr;
      for (int j = part * 8; j < a.d; j += 8 * kKParts) {
        float v[8];
        tmem_ld8(tmem_base + ((uint32_t)(q * 32) << 16) + (uint32_t)j, v);
        if (i < mrows) {
          if (pout) {
#pragma unroll
            for (int t = 0; t < 8; ++t) {
              float *q = pout + i + (int64_t)(j + t) * a.ldp;
              *q = (a.accumulate ? *q : 0.0f) + (nkb > 0 ? v[t] : 0.0f);
            }
          } else {
#pragma unroll
            for (int t = 0; t < 8; ++t) a.Y[i + (int64_t)(j + t) * a.ldy] = v[t] * scale;
          }
        }
      }
    }
  }
  tc_fence_before();
  // no peer may still multicast into, or arrive on, this CTA's shared memory after it exits
  cluster_sync_all();
  if (*abort_flag && threadIdx.x == 0) atomicOr(a.err, DERR_TIMEOUT);
  if (warp == 1) {
    tc_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::2.sync.aligned.b32 %0, %1;" ::"r"(tmem_base),
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

template <int NSPLIT, bool DERIV, int MODE, int KIND>
Error launch(const CUtensorMap &map, const TcArgs &a, size_t smem, dim3 grid, cudaStream_t st) {
  auto kfn = k_sketch_tc<NSPLIT, DERIV, MODE, KIND>;
  CK_CUDA(cudaFuncSetAttribute(kfn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  grid.x = (unsigned)(ceil_div((int64_t)grid.x, 2) * 2);   // whole pairs; an extra CTA stores nothing
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = grid;
  cfg.blockDim = dim3(kThreads);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = 2;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  ::ckinv::note_launch();
  CK_CUDA(cudaLaunchKernelEx(&cfg, kfn, map, a));
  return ok();
}

// Tensor map over a BF16 right factor Bt (d x kpad, row j = column j of the right factor,
// contiguous over the contraction; the context's Omega^T by default) and the launch geometry.
Error prepare_b(ckinv_ctx *ctx, const __nv_bfloat16 *Bt, int64_t kpad, int d, int nsplit, CUtensorMap *map,
                TcArgs *a, size_t *smem) {
  if (d % 16 != 0 || d > 512 || d < 16) return fail(CKINV_EINVAL, "sketch_tc: d must be 16..512, d % 16 == 0");
  if (nsplit < 1 || nsplit > 3) return fail(CKINV_EINVAL, "sketch_tc: 1..3 BF16 terms");
  struct {
    const __nv_bfloat16 *omegaT;
    int64_t kpad;
  } om{Bt, kpad};
  PFN_cuTensorMapEncodeTiled_v12000 enc = get_encode();
  if (!enc) return fail(CKINV_ECUDA, "cuTensorMapEncodeTiled entry point unavailable");
  // MMA column chunks: N = d for d <= 256, else two chunks (equal when d % 32 == 0) of
  // N <= 256; each CTA of the pair holds N/2 rows of each chunk (a multiple of 8, so every
  // half starts on a 1024-byte swizzle atom)
  const int n0 = d <= 256 ? d : (d % 32 == 0 ? d / 2 : 256);
  const int n1 = d - n0;
  int box_rows = n0 / 2;
  if (n1 > 0) {
    int x = n0 / 2, y = n1 / 2;
    while (y) { int t = x % y; x = y; y = t; }
    box_rows = x;
  }
  cuuint64_t gdim[2] = {(cuuint64_t)om.kpad, (cuuint64_t)d};
  cuuint64_t gstride[1] = {(cuuint64_t)om.kpad * 2};
  cuuint32_t box[2] = {(cuuint32_t)BK, (cuuint32_t)box_rows};
  cuuint32_t estr[2] = {1, 1};
  CUresult cr = enc(map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, (void *)om.omegaT, gdim, gstride, box, estr,
                    CU_TENSOR_MAP_INTERLEAVE_NONE, (kRowBytes == 128 ? CU_TENSOR_MAP_SWIZZLE_128B : CU_TENSOR_MAP_SWIZZLE_64B),
                    CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                    CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (cr != CUDA_SUCCESS) return fail(CKINV_ECUDA, "cuTensorMapEncodeTiled failed");
  memset(a, 0, sizeof(*a));
  a->d = d;
  a->num_kb = (int)(om.kpad / BK);
  a->kb_per_cta = a->num_kb;
  a->box_rows = box_rows;
  a->n0 = n0;
  a->n1 = n1;
  a->err = ctx->d_err;
  a->wait_ns = ctx->wait_ns;
  const size_t stage_bytes = (size_t)nsplit * kATileBytes + (size_t)d / 2 * kRowBytes;
  const size_t head = 512 + kPtSlots * kPtSlotBytes + 1024;   // barriers, point slots, alignment slack
  const size_t limit = 227 * 1024;
  int S = (int)((limit - head) / stage_bytes);
  if (S > 8) S = 8;   // also keeps kPtSlots - S >= 4 blocks of point prefetch
  if (S < 1) return fail(CKINV_EUNSUPPORTED, "sketch_tc: a stage does not fit in shared memory");
  a->stages = S;
  *smem = head + (size_t)S * stage_bytes;
  // A CTA with d > 256 holds all 512 TMEM columns; never let two of them share an SM (the
  // second would block in tcgen05.alloc until the first exits).
  if (d > 256) *smem = std::max(*smem, (size_t)(120 * 1024));
  return ok();
}

Error prepare(ckinv_ctx *ctx, int d, int nsplit, CUtensorMap *map, TcArgs *a, size_t *smem) {
  return prepare_b(ctx, ctx->om.omegaT, ctx->om.kpad, d, nsplit, map, a, smem);
}

template <int KIND>
Error dispatch_kernel(int nsplit, bool deriv, const CUtensorMap &map, const TcArgs &a, size_t smem, dim3 grid,
                      cudaStream_t st) {
  switch (nsplit * 2 + (deriv ? 1 : 0)) {
    case 2: return launch<1, false, 0, KIND>(map, a, smem, grid, st);
    case 3: return launch<1, true, 0, KIND>(map, a, smem, grid, st);
    case 4: return launch<2, false, 0, KIND>(map, a, smem, grid, st);
    case 5: return launch<2, true, 0, KIND>(map, a, smem, grid, st);
    case 6: return launch<3, false, 0, KIND>(map, a, smem, grid, st);
    case 7: return launch<3, true, 0, KIND>(map, a, smem, grid, st);
  }
  return fail(CKINV_EINVAL, "sketch_tc: nsplit must be 1..3");
}

Error dispatch_dense(int nsplit, const CUtensorMap &map, const TcArgs &a, size_t smem, dim3 grid, cudaStream_t st) {
  switch (nsplit) {
    case 1: return launch<1, false, 1, 0>(map, a, smem, grid, st);
    case 2: return launch<2, false, 1, 0>(map, a, smem, grid, st);
    case 3: return launch<3, false, 1, 0>(map, a, smem, grid, st);
  }
  return fail(CKINV_EINVAL, "dense_tc: nsplit must be 1..3");
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
                bool deriv, float *Y, int64_t ldy, cudaStream_t st, int64_t row0, int64_t m) {
  if (m < 0) m = n;
  if ((reinterpret_cast<uintptr_t>(points) & 15) != 0)
    return fail(CKINV_EINVAL, "sketch: points must be 16-byte aligned for the tensor-core path");
  CK_TRY(omega_materialise_bf16(ctx, st));
  CUtensorMap map;
  TcArgs a;
  size_t smem = 0;
  CK_TRY(prepare(ctx, d, nsplit, &map, &a, &smem));
  a.n = n;
  a.m = m;
  a.row0 = row0;
  a.dim = dim;
  a.kp = kp;
  a.pts = points;
  a.Y = Y;
  a.ldy = ldy;
  const dim3 grid((unsigned)ceil_div(m, BM), 1);
  if (kp.kind == CKINV_SE) return dispatch_kernel<CKINV_SE>(nsplit, deriv, map, a, smem, grid, st);
  if (kp.kind == CKINV_MATERN52) return dispatch_kernel<CKINV_MATERN52>(nsplit, deriv, map, a, smem, grid, st);
  return fail(CKINV_EINVAL, "sketch_tc: covariance kind has no fused form");
}

Error sketch_tc_rhs(ckinv_ctx *ctx, int64_t n, int dim, int d, int nsplit, const KernelParams &kp, const float *points,
                    const __nv_bfloat16 *Bt, int64_t kpad, int splits, float *part, int64_t ldp, bool accumulate,
                    cudaStream_t st) {
  if ((reinterpret_cast<uintptr_t>(points) & 15) != 0)
    return fail(CKINV_EINVAL, "sketch: points must be 16-byte aligned for the tensor-core path");
  if (kpad < n || kpad % 64 != 0) return fail(CKINV_EINVAL, "sketch_tc_rhs: kpad must be >= n, a multiple of 64");
  CUtensorMap map;
  TcArgs a;
  size_t smem = 0;
  CK_TRY(prepare_b(ctx, Bt, kpad, d, nsplit, &map, &a, &smem));
  a.n = n;
  a.m = n;
  a.dim = dim;
  a.kp = kp;
  a.pts = points;
  a.kb_per_cta = (int)ceil_div(a.num_kb, std::max(1, splits));
  a.part = part;
  a.ldp = ldp;
  a.accumulate = accumulate ? 1 : 0;
  const dim3 grid((unsigned)ceil_div(n, BM), (unsigned)ceil_div(a.num_kb, a.kb_per_cta));
  if (kp.kind == CKINV_SE) return dispatch_kernel<CKINV_SE>(nsplit, false, map, a, smem, grid, st);
  if (kp.kind == CKINV_MATERN52) return dispatch_kernel<CKINV_MATERN52>(nsplit, false, map, a, smem, grid, st);
  return fail(CKINV_EINVAL, "sketch_tc_rhs: covariance kind has no fused form");
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
    return dispatch_dense(nsplit, map, a, smem, dim3(mt, 1), st);
  }
  // split the contraction so that the grid covers every SM, then reduce in FP64
  int splits = std::max(1, std::min(a.num_kb, (ctx->sm_count + mt - 1) / mt));
  a.kb_per_cta = (int)ceil_div(a.num_kb, splits);
  splits = (int)ceil_div(a.num_kb, a.kb_per_cta);
  const int64_t ldp = (int64_t)mt * BM;
  float *part = nullptr;
  CK_CUDA(dev_alloc((void **)&part, sizeof(float) * (size_t)splits * ldp * d, st));
  a.part = part;
  a.ldp = ldp;
  Error e = dispatch_dense(nsplit, map, a, smem, dim3(mt, splits), st);
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
