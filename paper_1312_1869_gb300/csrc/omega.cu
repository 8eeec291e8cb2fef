// Structured random matrix Omega = c R H_N P of Definition 1 (Sec. 3.2): the Rademacher
// diagonal R and the column subsample P drawn from a counter-based generator, and the
// BF16 copy of the unscaled +-1 pattern that the tensor-core sketch streams by TMA.
//
// Draw (reading; the paper names no generator): Philox4x32-10 with key (seed_lo,
// seed_hi) and counter (index_lo, index_hi, stream, 0).  r_k = -1 iff bit 0 of word 0 at
// stream 0 is set.  P = the d candidates c < N with the smallest 64-bit keys
// (word0 << 32 | word1) at stream 1, ties to the smaller c, sorted ascending.
#include "internal.cuh"

namespace ckinv {
namespace {

__global__ void k_signs(int64_t n, uint32_t k0, uint32_t k1, uint32_t *bits) {
  int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  uint32_t bit = 0;
  if (k < n) {
    uint4 w = dev::philox4x32_10((uint32_t)k, (uint32_t)(k >> 32), 0u, 0u, k0, k1);
    bit = w.x & 1u;
  }
  uint32_t word = __ballot_sync(0xffffffffu, bit);
  if ((threadIdx.x & 31) == 0 && k < n) bits[k >> 5] = word;
}

__device__ __forceinline__ unsigned long long cand_key(int64_t c, uint32_t k0, uint32_t k1) {
  uint4 w = dev::philox4x32_10((uint32_t)c, (uint32_t)(c >> 32), 1u, 0u, k0, k1);
  return ((unsigned long long)w.x << 32) | (unsigned long long)w.y;
}

// The d smallest of N keys by a two-level radix select: a histogram of the top 16 key bits
// gives the bin t that holds the d-th smallest key; a histogram of the next 16 bits of the
// keys in bin t gives the sub-bin t2 that holds it.  Every key below (t, t2) and the keys of
// sub-bin t2 are then collected (about d of them: a sub-bin holds N / 2^32 keys on average)
// and sorted in one block.
//
// level 0: histogram of key bits 63..48 over all N candidates;
// level 1: histogram of key bits 47..32 over the candidates whose top bits equal small[0].
__global__ void k_key_hist(int64_t N, uint32_t k0, uint32_t k1, const uint32_t *small, int level, uint32_t *hist) {
  const uint32_t t = level ? small[0] : 0u;
  for (int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; c < N;
       c += (int64_t)gridDim.x * blockDim.x) {
    unsigned long long key = cand_key(c, k0, k1);
    if (level == 0) atomicAdd(&hist[key >> 48], 1u);
    else if ((uint32_t)(key >> 48) == t) atomicAdd(&hist[(key >> 32) & 0xffffu], 1u);
  }
}

// One block of 1024 threads: find the bin holding the target-th smallest key of the
// histogram.  Level 0 (target d): small[0] = bin t, small[3] = keys in the bins below t.
// Level 1 (target d - small[3], within bin t): small[4] = sub-bin t2.
__global__ void k_pick_bin(const uint32_t *hist, int d, int level, uint32_t *small) {
  __shared__ uint32_t part[1024];
  const uint32_t target = level ? (uint32_t)d - small[3] : (uint32_t)d;
  int t = threadIdx.x;
  uint32_t s = 0;
  for (int i = 0; i < 64; ++i) s += hist[t * 64 + i];
  part[t] = s;
  __syncthreads();
  // inclusive scan (Hillis-Steele)
  for (int off = 1; off < 1024; off <<= 1) {
    uint32_t v = (t >= off) ? part[t - off] : 0u;
    __syncthreads();
    part[t] += v;
    __syncthreads();
  }
  uint32_t before = (t == 0) ? 0u : part[t - 1];
  if (before < target && part[t] >= target) {
    uint32_t cum = before;
    for (int i = 0; i < 64; ++i) {
      const uint32_t h = hist[t * 64 + i];
      if (cum + h >= target) {
        if (level == 0) {
          small[0] = (uint32_t)(t * 64 + i);
          small[3] = cum;
        } else {
          small[4] = (uint32_t)(t * 64 + i);
        }
        break;
      }
      cum += h;
    }
  }
}

// Candidates: every key below bin (t, t2) of the two-level select, and the keys in it.
__global__ void k_collect(int64_t N, uint32_t k0, uint32_t k1, const uint32_t *small,
                          unsigned long long *cand, uint32_t *cand_idx, uint32_t cap,
                          uint32_t *counter) {
  const unsigned long long bound = ((unsigned long long)small[0] << 16) | small[4];   // key bits 63..32
  for (int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; c < N;
       c += (int64_t)gridDim.x * blockDim.x) {
    unsigned long long key = cand_key(c, k0, k1);
    if ((key >> 32) <= bound) {
      uint32_t pos = atomicAdd(counter, 1u);
      if (pos < cap) {
        cand[pos] = key;
        cand_idx[pos] = (uint32_t)c;
      }
    }
  }
}

// One block: sort the (key, index) candidates, keep the d smallest, sort their indices.
constexpr int kSortCap = 4096;
__global__ void k_finalize(const unsigned long long *cand, const uint32_t *cand_idx,
                           const uint32_t *counter, int d, int32_t *cols, int *err) {
  __shared__ unsigned long long skey[kSortCap];
  __shared__ uint32_t sidx[kSortCap];
  uint32_t cnt = *counter;
  if (cnt > (uint32_t)kSortCap || cnt < (uint32_t)d) {
    if (threadIdx.x == 0) atomicOr(err, DERR_CAPACITY);
    return;
  }
  int P = 1;
  while (P < (int)cnt) P <<= 1;
  for (int i = threadIdx.x; i < P; i += blockDim.x) {
    skey[i] = (i < (int)cnt) ? cand[i] : ~0ull;
    sidx[i] = (i < (int)cnt) ? cand_idx[i] : 0xffffffffu;
  }
  __syncthreads();
  // bitonic sort by (key, index)
  for (int k = 2; k <= P; k <<= 1) {
    for (int j = k >> 1; j > 0; j >>= 1) {
      for (int i = threadIdx.x; i < P; i += blockDim.x) {
        int ixj = i ^ j;
        if (ixj > i) {
          bool up = ((i & k) == 0);
          unsigned long long a = skey[i], b = skey[ixj];
          uint32_t ia = sidx[i], ib = sidx[ixj];
          bool gt = (a > b) || (a == b && ia > ib);
          if (gt == up) {
            skey[i] = b; skey[ixj] = a;
            sidx[i] = ib; sidx[ixj] = ia;
          }
        }
      }
      __syncthreads();
    }
  }
  // the first d entries are P; sort their indices ascending (reuse skey as index keys)
  int Q = 1;
  while (Q < d) Q <<= 1;
  for (int i = threadIdx.x; i < Q; i += blockDim.x)
    skey[i] = (i < d) ? (unsigned long long)sidx[i] : ~0ull;
  __syncthreads();
  for (int k = 2; k <= Q; k <<= 1) {
    for (int j = k >> 1; j > 0; j >>= 1) {
      for (int i = threadIdx.x; i < Q; i += blockDim.x) {
        int ixj = i ^ j;
        if (ixj > i) {
          bool up = ((i & k) == 0);
          unsigned long long a = skey[i], b = skey[ixj];
          if ((a > b) == up) { skey[i] = b; skey[ixj] = a; }
        }
      }
      __syncthreads();
    }
  }
  for (int i = threadIdx.x; i < d; i += blockDim.x) cols[i] = (int32_t)skey[i];
}

// omegaT[j * kpad + k] = bf16(+-1) = r_k (-1)^popc(k & p_j) for k < n, 0 for k >= n.
__global__ void k_omegaT(int64_t n, int64_t kpad, int d, const uint32_t *bits,
                         const int32_t *cols, __nv_bfloat16 *out) {
  int j = blockIdx.y;
  uint32_t p = (uint32_t)cols[j];
  int64_t k2 = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) * 2;
  if (k2 >= kpad) return;
  float v[2];
#pragma unroll
  for (int t = 0; t < 2; ++t) {
    int64_t k = k2 + t;
    if (k < n) {
      uint32_t s = (bits[k >> 5] >> (k & 31)) & 1u;
      s ^= (uint32_t)(__popcll((unsigned long long)k & (unsigned long long)p) & 1);
      v[t] = s ? -1.0f : 1.0f;
    } else {
      v[t] = 0.0f;
    }
  }
  __nv_bfloat162 pr = __floats2bfloat162_rn(v[0], v[1]);
  *reinterpret_cast<__nv_bfloat162 *>(out + (int64_t)j * kpad + k2) = pr;
}

// Launch sequence of the column draw (two-level select, collect, sort) on scratch that the
// caller provides: hist (65536 bins), small (>= 8 counters, zeroed here), the candidate
// list (cap entries) and the error word.
Error select_columns(int64_t N, int d, uint32_t k0, uint32_t k1, int grid, uint32_t *hist, uint32_t *small,
                     unsigned long long *cand, uint32_t *cand_idx, uint32_t cap, int32_t *cols, int *err,
                     cudaStream_t st) {
  CK_CUDA(cudaMemsetAsync(small, 0, sizeof(uint32_t) * 8, st));
  for (int level = 0; level < 2; ++level) {
    CK_CUDA(cudaMemsetAsync(hist, 0, sizeof(uint32_t) * 65536, st));
    note_launch();
    k_key_hist<<<grid, 256, 0, st>>>(N, k0, k1, small, level, hist);
    note_launch();
    k_pick_bin<<<1, 1024, 0, st>>>(hist, d, level, small);
  }
  note_launch();
  k_collect<<<grid, 256, 0, st>>>(N, k0, k1, small, cand, cand_idx, cap, small + 2);
  note_launch();
  k_finalize<<<1, 1024, 0, st>>>(cand, cand_idx, small + 2, d, cols, err);
  CK_CUDA(cudaGetLastError());
  return ok();
}

// Dense Omega (n x d FP32, column-major, ld n) of a given kind (Definition 1's c R T P with T
// the Walsh-Hadamard, discrete Hartley or cosine matrix, or the scaled Gaussian projection
// of Sec. 5.1), each entry evaluated in FP64 and rounded once.  Readings:
//   Walsh-Hadamard  c r_k (-1)^popcount(k & p_j),  c = N^-1/2
//   Hartley         n^-1/2 r_k cas(2 pi (k p_j mod n) / n),  cas = cos + sin
//   cosine          r_k s_p cos(pi ((2k + 1) p_j mod 4n) / (2n)),  s_0 = n^-1/2, s_p = (2/n)^1/2
//   Gaussian        z_kj / sqrt(n), z by Box-Muller from Philox words 0, 1 at (k d + j, stream 8)
__global__ void k_omega_dense(int64_t n, int d, int kind, double c, uint32_t k0, uint32_t k1,
                              const uint32_t *__restrict__ bits, const int32_t *__restrict__ cols,
                              float *__restrict__ Om) {
  const int j = blockIdx.y;
  const int64_t p = kind == 1 ? 0 : (int64_t)cols[j];
  for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < n; k += (int64_t)gridDim.x * blockDim.x) {
    double v;
    if (kind == 1) {
      const uint64_t idx = (uint64_t)k * (uint64_t)d + (uint64_t)j;
      const uint4 w = dev::philox4x32_10((uint32_t)idx, (uint32_t)(idx >> 32), 8u, 0u, k0, k1);
      const double u0 = ((double)w.x + 0.5) * (1.0 / 4294967296.0);
      const double u1 = ((double)w.y + 0.5) * (1.0 / 4294967296.0);
      v = sqrt(-2.0 * log(u0)) * cospi(2.0 * u1) * c;
    } else {
      const double r = ((bits[k >> 5] >> (k & 31)) & 1u) ? -1.0 : 1.0;
      if (kind == 0) {
        v = (__popcll((unsigned long long)(k & p)) & 1) ? -c * r : c * r;
      } else if (kind == 2) {
        const double a = (double)(((k % n) * (p % n)) % n) / (double)n;   // angle / (2 pi)
        v = c * r * (cospi(2.0 * a) + sinpi(2.0 * a));
      } else {
        const int64_t m = ((2 * k + 1) * p) % (4 * n);
        const double s = (p == 0) ? sqrt(1.0 / (double)n) : sqrt(2.0 / (double)n);
        v = r * s * cospi((double)m / (2.0 * (double)n));
      }
    }
    Om[k + (int64_t)j * n] = (float)v;
  }
}

}  // namespace

Error omega_dense(ckinv_ctx *ctx, int64_t n, int32_t d, uint64_t seed, int kind, float *Om, cudaStream_t st) {
  if (kind < 0 || kind > 3) return fail(CKINV_EINVAL, "unknown Omega kind");
  const uint32_t k0 = (uint32_t)seed, k1 = (uint32_t)(seed >> 32);
  // the signs of R and the column subsample: over N = 2^ceil(log2 n) candidates for the
  // Walsh-Hadamard matrix, over the n columns of the Hartley and cosine matrices
  const uint32_t *bits = nullptr;
  const int32_t *cols = nullptr;
  if (kind == 0) {
    CK_TRY(omega_draw(ctx, n, d, seed, st));
    bits = ctx->om.bits;
    cols = ctx->om.cols;
  } else if (kind >= 2) {
    if (d > n) return fail(CKINV_EINVAL, "d above n for a Hartley or cosine Omega");
    CK_TRY(omega_draw(ctx, n, d, seed, st));          // signs (and scratch) for this n
    bits = ctx->om.bits;
    int32_t *c2 = nullptr;
    CK_CUDA(dev_alloc(&c2, sizeof(int32_t) * d, st));
    const int grid = (int)std::min<int64_t>(ceil_div(n, 256), (int64_t)ctx->sm_count * 8);
    Error e = select_columns(n, d, k0, k1, grid, ctx->hist, ctx->small, ctx->cand, ctx->cand_idx,
                             (uint32_t)ctx->cand_cap, c2, ctx->d_err, st);
    if (e.st) {
      cudaFreeAsync(c2, st);
      return e;
    }
    cols = c2;
  }
  double c = 1.0;
  if (kind == 0) c = 1.0 / std::sqrt((double)padded_order(n));
  else if (kind == 1 || kind == 2) c = 1.0 / std::sqrt((double)n);
  dim3 grid((unsigned)std::min<int64_t>(ceil_div(n, 256), 256), (unsigned)d);
  note_launch();
  k_omega_dense<<<grid, 256, 0, st>>>(n, d, kind, c, k0, k1, bits, cols, Om);
  cudaError_t ce = cudaGetLastError();
  if (kind >= 2) cudaFreeAsync(const_cast<int32_t *>(cols), st);
  if (ce != cudaSuccess) return fail(CKINV_ECUDA, cudaGetErrorString(ce));
  return ok();
}

namespace {
template <typename T>
Error grow(T **p, size_t *cap, size_t need, cudaStream_t st) {
  if (*p && *cap >= need) return ok();
  if (*p) cudaFreeAsync(*p, st);
  *p = nullptr;
  *cap = 0;
  CK_CUDA(dev_alloc((void **)p, sizeof(T) * need, st));
  *cap = need;
  return ok();
}
}  // namespace

Error omega_reserve(ckinv_ctx *ctx, int64_t n, int32_t d, cudaStream_t st) {
  OmegaCache &om = ctx->om;
  CK_TRY(grow(&om.bits, &om.bits_cap, (size_t)ceil_div(n, 32), st));
  CK_TRY(grow(&om.cols, &om.cols_cap, (size_t)d, st));
  const int64_t kpad = ceil_div(n, 64) * 64;
  size_t cap = om.omegaT_cap / sizeof(__nv_bfloat16);
  CK_TRY(grow(&om.omegaT, &cap, (size_t)kpad * d, st));
  om.omegaT_cap = cap * sizeof(__nv_bfloat16);
  if (!ctx->hist) {
    CK_CUDA(cudaMalloc((void **)&ctx->hist, sizeof(uint32_t) * 65536));
    CK_CUDA(cudaMalloc((void **)&ctx->small, sizeof(uint32_t) * 16));
    ctx->cand_cap = kSortCap;
    CK_CUDA(cudaMalloc((void **)&ctx->cand, sizeof(unsigned long long) * ctx->cand_cap));
    CK_CUDA(cudaMalloc((void **)&ctx->cand_idx, sizeof(uint32_t) * ctx->cand_cap));
  }
  return ok();
}

Error omega_draw(ckinv_ctx *ctx, int64_t n, int32_t d, uint64_t seed, cudaStream_t st) {
  OmegaCache &om = ctx->om;
  if (om.n == n && om.d == d && om.seed == seed && om.bits) return ok();
  int64_t N = padded_order(n);
  uint32_t k0 = (uint32_t)seed, k1 = (uint32_t)(seed >> 32);
  om.n = -1;
  om.omegaT_valid = false;
  CK_TRY(grow(&om.bits, &om.bits_cap, (size_t)ceil_div(n, 32), st));
  CK_TRY(grow(&om.cols, &om.cols_cap, (size_t)d, st));
  if (!ctx->hist) {
    CK_CUDA(cudaMalloc((void **)&ctx->hist, sizeof(uint32_t) * 65536));
    CK_CUDA(cudaMalloc((void **)&ctx->small, sizeof(uint32_t) * 16));
    ctx->cand_cap = kSortCap;
    CK_CUDA(cudaMalloc((void **)&ctx->cand, sizeof(unsigned long long) * ctx->cand_cap));
    CK_CUDA(cudaMalloc((void **)&ctx->cand_idx, sizeof(uint32_t) * ctx->cand_cap));
  }
  ::ckinv::note_launch(), k_signs<<<(unsigned)ceil_div(n, 256), 256, 0, st>>>(n, k0, k1, om.bits);
  int grid = (int)std::min<int64_t>(ceil_div(N, 256), (int64_t)ctx->sm_count * 8);
  CK_TRY(select_columns(N, d, k0, k1, grid, ctx->hist, ctx->small, ctx->cand, ctx->cand_idx, (uint32_t)ctx->cand_cap,
                        om.cols, ctx->d_err, st));
  om.n = n;
  om.d = d;
  om.seed = seed;
  return ok();
}

Error omega_materialise_bf16(ckinv_ctx *ctx, cudaStream_t st) {
  OmegaCache &om = ctx->om;
  if (om.omegaT_valid) return ok();
  int64_t kpad = ceil_div(om.n, 64) * 64;
  size_t cap = om.omegaT_cap / sizeof(__nv_bfloat16);
  CK_TRY(grow(&om.omegaT, &cap, (size_t)kpad * om.d, st));
  om.omegaT_cap = cap * sizeof(__nv_bfloat16);
  om.kpad = kpad;
  dim3 grid((unsigned)ceil_div(kpad / 2, 256), (unsigned)om.d);
  ::ckinv::note_launch(), k_omegaT<<<grid, 256, 0, st>>>(om.n, kpad, om.d, om.bits, om.cols, om.omegaT);
  CK_CUDA(cudaGetLastError());
  om.omegaT_valid = true;
  return ok();
}

}  // namespace ckinv

// ===================================================================== no-allocation draw
// A variant of the Omega draw for callers that cannot allocate device memory: programs
// that hand all device memory to their own pool up front and leave nothing for the CUDA
// allocator, and code that must not take the implicit device synchronisation an allocation
// can cause.  Its scratch (the 65536-bin key histogram, the candidate list and a few
// counters) is one file-scope device array, so the entry point needs no context and calls
// no allocator.  The array exists once per device that loads the library and lives until
// the process exits; every call on a device reuses it, so calls whose work overlaps on the
// GPU (different streams, or different host threads) race on it and must be serialised by
// the caller.
namespace ckinv {
namespace {

constexpr size_t kNoAllocHistBytes = sizeof(uint32_t) * 65536;
constexpr size_t kNoAllocSmallBytes = 256;   // counters and the error word
constexpr size_t kNoAllocKeyBytes = sizeof(unsigned long long) * kSortCap;
constexpr size_t kNoAllocIdxBytes = sizeof(uint32_t) * kSortCap;
constexpr size_t kNoAllocBytes = kNoAllocHistBytes + kNoAllocSmallBytes + kNoAllocKeyBytes + kNoAllocIdxBytes;

static __device__ __align__(256) unsigned char g_omega_scratch[kNoAllocBytes];

constexpr int kMaxDevices = 64;
unsigned char *g_scratch_addr[kMaxDevices] = {};
int g_scratch_ready[kMaxDevices] = {};

// Device address of this device's scratch array, resolved once per device with that device
// current (the host-side symbol is only a stand-in, never a device address).
Error scratch_for_current_device(unsigned char **out) {
  int dev = 0;
  CK_CUDA(cudaGetDevice(&dev));
  if (dev < 0 || dev >= kMaxDevices) return fail(CKINV_EUNSUPPORTED, "device index above 63");
  if (!__atomic_load_n(&g_scratch_ready[dev], __ATOMIC_ACQUIRE)) {
    void *p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_omega_scratch);
    if (e != cudaSuccess)
      return fail(CKINV_ECUDA, std::string("cudaGetSymbolAddress of the Omega scratch: ") + cudaGetErrorString(e));
    g_scratch_addr[dev] = static_cast<unsigned char *>(p);
    __atomic_store_n(&g_scratch_ready[dev], 1, __ATOMIC_RELEASE);
  }
  *out = g_scratch_addr[dev];
  return ok();
}

}  // namespace
}  // namespace ckinv

extern "C" ckinv_status ckinv_omega_noalloc(int64_t n, int32_t d, uint64_t seed, uint32_t *sign_bits, int32_t *cols,
                                            ckinv_stream stream) {
  using namespace ckinv;
  if (!sign_bits || !cols) {
    set_static_error("ckinv_omega_noalloc: null output pointer");
    return CKINV_EINVAL;
  }
  if (n < 1 || n > ((int64_t)1 << 31) || d < 1 || d > 512 || (int64_t)d > padded_order(n)) {
    set_static_error("ckinv_omega_noalloc: need 1 <= n <= 2^31 and 1 <= d <= min(512, N); its fixed scratch "
                     "holds a 65536-bin histogram and 4096 candidates");
    return CKINV_EINVAL;
  }
  auto cuda_fail = [](const char *what, cudaError_t e) {
    set_static_error(std::string("ckinv_omega_noalloc: ") + what + ": " + cudaGetErrorString(e));
    return e == cudaErrorMemoryAllocation ? CKINV_ENOMEM : CKINV_ECUDA;
  };
  cudaStream_t st = (cudaStream_t)stream;
  unsigned char *base = nullptr;
  {
    Error e = scratch_for_current_device(&base);
    if (e.st != CKINV_OK) {
      set_static_error(e.msg);
      return e.st;
    }
  }
  uint32_t *hist = reinterpret_cast<uint32_t *>(base);
  uint32_t *small = reinterpret_cast<uint32_t *>(base + kNoAllocHistBytes);
  int *err = reinterpret_cast<int *>(small + 32);
  unsigned long long *cand = reinterpret_cast<unsigned long long *>(base + kNoAllocHistBytes + kNoAllocSmallBytes);
  uint32_t *cand_idx = reinterpret_cast<uint32_t *>(base + kNoAllocHistBytes + kNoAllocSmallBytes + kNoAllocKeyBytes);
  const int64_t N = padded_order(n);
  const uint32_t k0 = (uint32_t)seed, k1 = (uint32_t)(seed >> 32);
  // the array keeps the previous call's contents: clear what must start at zero (the
  // histogram and the counters are cleared again inside select_columns)
  cudaError_t ce = cudaMemsetAsync(base, 0, kNoAllocHistBytes + kNoAllocSmallBytes, st);
  if (ce != cudaSuccess) return cuda_fail("clearing the scratch array", ce);
  note_launch();
  k_signs<<<(unsigned)ceil_div(n, 256), 256, 0, st>>>(n, k0, k1, sign_bits);
  if ((ce = cudaGetLastError()) != cudaSuccess) return cuda_fail("launch of the sign draw", ce);
  int dev = 0, sms = 0;
  if ((ce = cudaGetDevice(&dev)) != cudaSuccess) return cuda_fail("cudaGetDevice", ce);
  if ((ce = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess)
    return cuda_fail("cudaDeviceGetAttribute", ce);
  const int grid = (int)std::min<int64_t>(ceil_div(N, 256), (int64_t)sms * 8);
  {
    Error e = select_columns(N, d, k0, k1, grid, hist, small, cand, cand_idx, (uint32_t)kSortCap, cols, err, st);
    if (e.st != CKINV_OK) {
      set_static_error("ckinv_omega_noalloc: " + e.msg);
      return e.st;
    }
  }
  // report a candidate-list overflow (a sub-bin of the two-level select holding more than
  // 4096 - d keys; about N / 2^32 are expected, so not at any supported n) before returning
  int herr = 0;
  if ((ce = cudaMemcpyAsync(&herr, err, sizeof(int), cudaMemcpyDeviceToHost, st)) != cudaSuccess)
    return cuda_fail("read-back of the error word", ce);
  if ((ce = cudaStreamSynchronize(st)) != cudaSuccess) return cuda_fail("stream synchronisation", ce);
  if (herr) {
    set_static_error("ckinv_omega_noalloc: more than 4096 candidate columns share the selection bin");
    return CKINV_EUNSUPPORTED;
  }
  return CKINV_OK;
}
