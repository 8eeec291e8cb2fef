// C ABI of the ckinv library: argument checking, workspace ownership and the order of the
// stages (sketch -> TSQR -> core -> solve -> likelihood and gradient).  All arithmetic of
// the method runs in the kernels of the other translation units.
#include <cmath>
#include <cstdio>
#include <cstring>
#include <map>
#include <mutex>
#include <tuple>
#include <vector>

#include "internal.cuh"

using namespace ckinv;

Error ckinv::stage_upload(ckinv_ctx *ctx, const void *src, size_t bytes, void *dst, cudaStream_t st) {
  if (ctx->capture_arena) {
    // inside a graph capture: the copy runs when the graph does, so its source bytes must
    // stay put until then
    UploadArena &ar = *ctx->capture_arena;
    size_t at = (ar.used + 15) & ~(size_t)15;
    if (at + bytes > ar.cap) return fail(CKINV_ENOMEM, "upload arena of the batched graph is full");
    memcpy(ar.host + at, src, bytes);
    ar.used = at + bytes;
    CK_CUDA(cudaMemcpyAsync(dst, ar.host + at, bytes, cudaMemcpyHostToDevice, st));
    return ok();
  }
  ckinv_ctx::Stage &sl = ctx->stage[ctx->stage_next];
  ctx->stage_next = (ctx->stage_next + 1) % 8;
  if (sl.done) CK_CUDA(cudaEventSynchronize(sl.done));
  else CK_CUDA(cudaEventCreateWithFlags(&sl.done, cudaEventDisableTiming));
  if (sl.cap < bytes) {
    if (sl.host) CK_CUDA(cudaFreeHost(sl.host));
    sl.host = nullptr;
    sl.cap = std::max<size_t>(bytes, 4096);
    CK_CUDA(cudaMallocHost(&sl.host, sl.cap));
  }
  memcpy(sl.host, src, bytes);
  CK_CUDA(cudaMemcpyAsync(dst, sl.host, bytes, cudaMemcpyHostToDevice, st));
  CK_CUDA(cudaEventRecord(sl.done, st));
  return ok();
}

unsigned long long &ckinv::launch_counter() {
  static unsigned long long c = 0;
  return c;
}

namespace {
// The library's own stream-ordered memory pools, one per device.  Freed blocks stay in the
// pool (release threshold: never) so that the workspaces of repeated solves (hundreds of MB
// each) are reused without remapping; the setting is private to these pools and leaves the
// device's default pool, which other code in the process may use, as it was.  When the last
// context on a device is destroyed its pool is trimmed back to the driver.
constexpr int kPoolDevices = 64;
std::mutex g_pool_mu;
cudaMemPool_t g_pool[kPoolDevices] = {};
int g_live_ctx[kPoolDevices] = {};

cudaError_t library_pool(int dev, cudaMemPool_t *out) {
  if (dev < 0 || dev >= kPoolDevices) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lk(g_pool_mu);
  if (!g_pool[dev]) {
    cudaMemPoolProps props = {};
    props.allocType = cudaMemAllocationTypePinned;
    props.handleTypes = cudaMemHandleTypeNone;
    props.location.type = cudaMemLocationTypeDevice;
    props.location.id = dev;
    cudaMemPool_t pool = nullptr;
    cudaError_t e = cudaMemPoolCreate(&pool, &props);
    if (e != cudaSuccess) return e;
    uint64_t keep = UINT64_MAX;
    e = cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &keep);
    if (e != cudaSuccess) {
      cudaMemPoolDestroy(pool);
      return e;
    }
    g_pool[dev] = pool;
  }
  *out = g_pool[dev];
  return cudaSuccess;
}
}  // namespace

cudaError_t ckinv::dev_alloc(void **p, size_t bytes, cudaStream_t st) {
  // inside a stream capture the allocation becomes a graph memory node of the device's
  // graph pool; everywhere else it comes from the library's pool
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  if (cudaStreamIsCapturing(st, &cs) != cudaSuccess) return cudaGetLastError();
  if (cs != cudaStreamCaptureStatusNone) return cudaMallocAsync(p, bytes, st);
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  cudaMemPool_t pool = nullptr;
  if ((e = library_pool(dev, &pool)) != cudaSuccess) return e;
  return cudaMallocFromPoolAsync(p, bytes, pool, st);
}

namespace {

thread_local std::string g_static_err;

struct DeviceGuard {
  int prev = -1;
  bool ok = false;
  explicit DeviceGuard(int dev) {
    if (cudaGetDevice(&prev) != cudaSuccess) prev = -1;
    ok = (cudaSetDevice(dev) == cudaSuccess);
  }
  ~DeviceGuard() {
    if (prev >= 0) cudaSetDevice(prev);
  }
};

ckinv_status finish(ckinv_ctx *ctx, const Error &e) {
  if (e.st != CKINV_OK) {
    if (ctx) ctx->err = e.msg;
    else g_static_err = e.msg;
  }
  return e.st;
}

Error check_plan(const ckinv_plan_desc *plan, const ckinv_kernel *kern, bool need_points) {
  if (!plan || !kern) return fail(CKINV_EINVAL, "null plan or kernel descriptor");
  if (plan->d < 16 || plan->d > 512 || plan->d % 16 != 0)
    return fail(CKINV_EINVAL, "d must satisfy 16 <= d <= 512 and d % 16 == 0");
  if (plan->n < plan->d) return fail(CKINV_EINVAL, "n must be >= d");
  if (plan->n > ((int64_t)1 << 31)) return fail(CKINV_EUNSUPPORTED, "n above 2^31");
  if (kern->kind != CKINV_SE && kern->kind != CKINV_MATERN52 && kern->kind != CKINV_DENSE)
    return fail(CKINV_EINVAL, "unknown kernel kind");
  if (kern->kind != CKINV_DENSE && need_points) {
    if (plan->dim < 1 || plan->dim > 3) return fail(CKINV_EINVAL, "dim must be 1, 2 or 3");
    if (!(kern->lengthscale > 0) || !(kern->variance > 0))
      return fail(CKINV_EINVAL, "lengthscale and variance must be > 0");
  }
  if (!(kern->nugget > 0)) return fail(CKINV_EINVAL, "nugget must be > 0");
  if (plan->prec < CKINV_FP32 || plan->prec > CKINV_FP32_WHT) return fail(CKINV_EINVAL, "unknown precision");
  if (plan->block_rows != 0 && plan->block_rows < plan->d) return fail(CKINV_EINVAL, "block_rows must be >= d");
  if (plan->refine_steps < 0 || plan->refine_steps > 4) return fail(CKINV_EINVAL, "refine_steps must be 0..4");
  if (plan->tree_fp64_levels < -1) return fail(CKINV_EINVAL, "tree_fp64_levels must be >= -1");
  if (plan->leaf_fp64 != 0 && plan->leaf_fp64 != 1) return fail(CKINV_EINVAL, "leaf_fp64 must be 0 or 1");
  if (plan->omega_kind < 0 || plan->omega_kind > 3) return fail(CKINV_EINVAL, "omega_kind must be 0..3");
  return ok();
}

// The BF16 form runs the TSQR's large FP32 GEMMs on the tensor cores (three BF16 terms per
// operand, FP32 accumulation in TMEM: R to ~5e-6, Q_hat orthonormal to ~1e-5 at d = 512,
// far below that form's 2^-9 kernel-entry rounding).  The forms that carry kernel entries to
// 16 or 24 bits (BF16x2, BF16x3), the FP32 form and FP64 leaves keep them on the CUDA cores
// (Q_hat orthonormal to ~5e-7): measured against the oracle, the tensor-core Q_hat alone put
// the BF16x3 form's K^-1 A 20x to 1000x above its kernel-entry floor.
bool tsqr_on_tensor_cores(const ckinv_plan_desc *plan) {
  return plan->prec == CKINV_BF16 && plan->leaf_fp64 == 0;
}

KernelParams make_params(const ckinv_plan_desc *plan, const ckinv_kernel *kern) {
  KernelParams kp;
  kp.kind = kern->kind;
  double l = kern->lengthscale > 0 ? kern->lengthscale : 1.0;
  kp.inv_l = (float)(1.0 / l);
  double cse = 1.4426950408889634 / (2.0 * l * l);
  kp.c_se = (float)cse;
  kp.coord_scale = (kern->kind == CKINV_SE) ? (float)std::sqrt(cse) : 1.0f;
  double c = 1.0 / std::sqrt((double)padded_order(plan->n));
  double var = (kern->kind == CKINV_DENSE) ? 1.0 : kern->variance;
  kp.scale = var * c;
  kp.ell = l;
  kp.var = var;
  return kp;
}

Error read_device_error(ckinv_ctx *ctx, cudaStream_t st) {
  int h = 0;
  CK_CUDA(cudaMemcpyAsync(&h, ctx->d_err, sizeof(int), cudaMemcpyDeviceToHost, st));
  CK_CUDA(cudaStreamSynchronize(st));
  if (h) {
    CK_CUDA(cudaMemsetAsync(ctx->d_err, 0, sizeof(int), st));
    if (h & DERR_TIMEOUT) return fail(CKINV_ETIMEOUT, "a bounded device-side wait ran out");
    if (h & DERR_NONFINITE) return fail(CKINV_EINVAL, "non-finite value (NaN or Inf) in the points, A or y");
    if (h & DERR_SINGULAR) return fail(CKINV_ESINGULAR, "zero or non-finite pivot in an LU factorisation");
    if (h & DERR_CAPACITY) return fail(CKINV_EUNSUPPORTED, "device list capacity exceeded (Omega draw)");
  }
  return ok();
}

// Flags DERR_NONFINITE when any of the `count` values (rows x cols, leading dimension ld)
// is a NaN or an infinity.  A cheap pass over inputs of O(n) size: the points, the right-hand
// sides and the targets.
__global__ void k_check_finite(const float *x, int64_t rows, int64_t cols, int64_t ld, int *err) {
  const int64_t count = rows * cols;
  bool bad = false;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < count; e += (int64_t)gridDim.x * blockDim.x) {
    const float v = x[(e % rows) + (e / rows) * ld];
    bad |= !(fabsf(v) <= 3.402823466e38f);
  }
  if (__any_sync(0xffffffffu, bad) && (threadIdx.x & 31) == 0) atomicOr(err, DERR_NONFINITE);
}

// dst = (float) src, n elements.
__global__ void k_narrow_f64(const double *src, int64_t n, float *dst) {
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x)
    dst[e] = (float)src[e];
}

Error check_finite(ckinv_ctx *ctx, const float *x, int64_t rows, int64_t cols, int64_t ld, cudaStream_t st) {
  if (rows <= 0 || cols <= 0) return ok();
  const unsigned g = (unsigned)std::min<int64_t>(ceil_div(rows * cols, 256), (int64_t)ctx->sm_count * 4);
  note_launch();
  k_check_finite<<<g, 256, 0, st>>>(x, rows, cols, ld, ctx->d_err);
  CK_CUDA(cudaGetLastError());
  return ok();
}

// Rows row0 .. row0 + m - 1 of the sketch (m < 0: all n rows).
Error do_sketch(ckinv_ctx *ctx, const ckinv_plan_desc *plan, const ckinv_kernel *kern, const float *points,
                const float *K, int64_t ldk, bool deriv, float *Y, int64_t ldy, cudaStream_t st, int64_t row0 = 0,
                int64_t m = -1) {
  CK_TRY(check_plan(plan, kern, true));
  if (m < 0) m = plan->n;
  if (row0 < 0 || m < 1 || row0 + m > plan->n) return fail(CKINV_EINVAL, "rows must lie in [0, n)");
  if (!Y || ldy < m) return fail(CKINV_EINVAL, "Y must be non-null with ldy >= its row count");
  if (kern->kind == CKINV_DENSE) {
    if (!K || ldk < plan->n) return fail(CKINV_EINVAL, "dense kernel needs K with ldk >= n");
    if (deriv) return fail(CKINV_EINVAL, "no derivative sketch for a materialised K");
  } else if (!points) {
    return fail(CKINV_EINVAL, "points must be non-null");
  }
  if (kern->kind != CKINV_DENSE) CK_TRY(check_finite(ctx, points, plan->dim, plan->n, plan->dim, st));
  KernelParams kp = make_params(plan, kern);
  if (plan->omega_kind != 0) {
    // a dense Omega (Gaussian, Hartley or cosine): materialised, then contracted
    if (deriv) return fail(CKINV_EINVAL, "the derivative sketch takes the Walsh-Hadamard Omega only");
    if (kern->kind != CKINV_DENSE && (row0 != 0 || m != plan->n))
      return fail(CKINV_EINVAL, "a row range of a matrix-free sketch takes the Walsh-Hadamard Omega only");
    float *Om = nullptr;
    CK_CUDA(dev_alloc(&Om, sizeof(float) * (size_t)plan->n * plan->d, st));
    Error e = omega_dense(ctx, plan->n, plan->d, plan->seed, plan->omega_kind, Om, st);
    if (e.st == CKINV_OK) {
      if (kern->kind == CKINV_DENSE)
        e = gemm_batched<float>(ctx, false, (int)m, plan->d, (int)plan->n, 1.0f, K + row0, ldk, 0, Om, plan->n, 0, 0.0f,
                                Y, ldy, 0, 1, st);
      else
        e = sketch_dense_omega(ctx, plan->n, plan->dim, plan->d, kp, points, Om, Y, ldy, st);
    }
    cudaFreeAsync(Om, st);
    return e;
  }
  CK_TRY(omega_draw(ctx, plan->n, plan->d, plan->seed, st));
  if (kern->kind == CKINV_DENSE) {
    if (plan->prec == CKINV_FP32_WHT && sketch_wht_supported(plan->n, plan->d))
      return sketch_wht_dense(ctx, plan->n, plan->d, kp, K, ldk, Y, ldy, st, row0, m);
    // K is symmetric: its column i is read as row i (16-byte rows for the tensor-core path)
    if (plan->prec != CKINV_FP32 && plan->prec != CKINV_FP32_WHT && ldk % 4 == 0 &&
        (reinterpret_cast<uintptr_t>(K) & 15) == 0)
      return dense_tc(ctx, m, plan->n, plan->d, plan->prec, K + row0 * ldk, ldk, kp.scale, Y, ldy, nullptr, 0, 0, st);
    return sketch_simt(ctx, plan->n, plan->dim, plan->d, kp, nullptr, K, ldk, false, Y, ldy, st, row0, m);
  }
  if (plan->prec == CKINV_FP32_WHT && sketch_wht_supported(plan->n, plan->d))
    return sketch_wht(ctx, plan->n, plan->dim, plan->d, kp, points, deriv, Y, ldy, st, row0, m);
  if (plan->prec == CKINV_FP32 || plan->prec == CKINV_FP32_WHT)
    return sketch_simt(ctx, plan->n, plan->dim, plan->d, kp, points, nullptr, 0, deriv, Y, ldy, st, row0, m);
  return sketch_tc(ctx, plan->n, plan->dim, plan->d, plan->prec, kp, points, deriv, Y, ldy, st, row0, m);
}

void factor_release(ckinv_factor *f) {
  if (!f) return;
  for (void *p : {(void *)f->Q, (void *)f->R, (void *)f->B, (void *)f->Cp, (void *)f->luB, (void *)f->pivB,
                  (void *)f->logdet_parts, (void *)f->bits, (void *)f->cols, (void *)f->S2, (void *)f->pivS,
                  (void *)f->logdet2, (void *)f->omega_dense})
    if (p) cudaFreeAsync(p, f->stream);
  delete f;
}

// ------------------------------------------------------------------ leaf-height autotuner
// Chosen TSQR leaf heights, keyed by (device, d, ceil(log2 n), FP64 tree levels, FP64 leaves,
// tensor-core GEMMs).
struct TuneKey {
  int device, d, log2n, fp64_levels, leaf_fp64, tc;
  bool operator<(const TuneKey &o) const {
    return std::tie(device, d, log2n, fp64_levels, leaf_fp64, tc) <
           std::tie(o.device, o.d, o.log2n, o.fp64_levels, o.leaf_fp64, o.tc);
  }
};
std::mutex g_tune_mu;
std::map<TuneKey, int> g_tuned;

TuneKey tune_key(const ckinv_ctx *ctx, const ckinv_plan_desc *plan) {
  int l = 0;
  while (((int64_t)1 << l) < plan->n) ++l;
  return TuneKey{ctx->device, plan->d, l, plan->tree_fp64_levels, plan->leaf_fp64, tsqr_on_tensor_cores(plan) ? 1 : 0};
}

int leaf_rows(const ckinv_ctx *ctx, const ckinv_plan_desc *plan) {
  if (plan->block_rows) return plan->block_rows;
  {
    std::lock_guard<std::mutex> lk(g_tune_mu);
    auto it = g_tuned.find(tune_key(ctx, plan));
    if (it != g_tuned.end()) return it->second;
  }
  return auto_block_rows(plan->n, plan->d, ctx->sm_count);
}

__global__ void k_fill_hash(int64_t count, uint32_t salt, float *Y) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < count; i += (int64_t)gridDim.x * blockDim.x) {
    uint32_t h = (uint32_t)i * 2654435761u ^ salt;
    h ^= h >> 16; h *= 0x7feb352du; h ^= h >> 15; h *= 0x846ca68bu; h ^= h >> 16;
    Y[i] = (float)(h >> 8) * (1.0f / 16777216.0f) - 0.5f;
  }
}

// Times the TSQR of an n x d matrix of pseudo-random entries at each candidate leaf height
// and records the fastest for the plan's shape class.
Error autotune_leaf_rows(ckinv_ctx *ctx, const ckinv_plan_desc *plan, cudaStream_t st, int *out) {
  const int64_t n = plan->n;
  const int d = plan->d;
  std::vector<int> cand;
  for (int b : {256, 512, 1024, 2048, 4096})
    if (b >= d && (int64_t)b * 2 <= n) cand.push_back(b);
  // the tallest leaf whose panels fit in shared memory (fewer leaves, fewer FP64 combines)
  const int bmax = max_leaf_rows(d, plan->leaf_fp64 != 0);
  if (bmax >= d && (int64_t)bmax * 2 <= n && std::find(cand.begin(), cand.end(), bmax) == cand.end())
    cand.push_back(bmax);
  if (cand.empty()) cand.push_back(auto_block_rows(n, d, ctx->sm_count));
  float *Y = nullptr, *Q = nullptr;
  double *R = nullptr;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  Error e = ok();
  int best = cand[0];
  float best_ms = 1e30f;
  do {
    if (dev_alloc((void **)&Y, sizeof(float) * n * d, st) != cudaSuccess ||
        dev_alloc((void **)&Q, sizeof(float) * n * d, st) != cudaSuccess ||
        dev_alloc((void **)&R, sizeof(double) * d * d, st) != cudaSuccess) {
      e = fail(CKINV_ENOMEM, "autotune workspace");
      break;
    }
    if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) {
      e = fail(CKINV_ECUDA, "autotune events");
      break;
    }
    note_launch();
    k_fill_hash<<<(unsigned)std::min<int64_t>(ceil_div(n * d, 256), 4096), 256, 0, st>>>(n * d, 0x9e3779b9u, Y);
    for (int b : cand) {
      if ((e = tsqr_factor(ctx, n, d, b, plan->tree_fp64_levels, plan->leaf_fp64 != 0, tsqr_on_tensor_cores(plan), Y, n, Q, R, st)).st) break;
      cudaEventRecord(e0, st);
      for (int r = 0; r < 2 && !e.st; ++r)
        e = tsqr_factor(ctx, n, d, b, plan->tree_fp64_levels, plan->leaf_fp64 != 0, tsqr_on_tensor_cores(plan), Y, n, Q, R, st);
      cudaEventRecord(e1, st);
      if (e.st) break;
      if (cudaEventSynchronize(e1) != cudaSuccess) {
        e = fail(CKINV_ECUDA, "autotune timing");
        break;
      }
      float ms = 0.f;
      cudaEventElapsedTime(&ms, e0, e1);
      if (ms < best_ms) {
        best_ms = ms;
        best = b;
      }
    }
  } while (0);
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  for (void *p : {(void *)Y, (void *)Q, (void *)R})
    if (p) cudaFreeAsync(p, st);
  if (e.st) return e;
  {
    std::lock_guard<std::mutex> lk(g_tune_mu);
    g_tuned[tune_key(ctx, plan)] = best;
  }
  *out = best;
  return ok();
}

Error do_tsqr(ckinv_ctx *ctx, const ckinv_plan_desc *plan, const ckinv_kernel *kern, float *Y, int64_t ldy,
              ckinv_factor **out, cudaStream_t st) {
  CK_TRY(check_plan(plan, kern, false));
  if (!Y || !out || ldy < plan->n) return fail(CKINV_EINVAL, "Y/out must be non-null, ldy >= n");
  *out = nullptr;
  const int64_t n = plan->n;
  const int d = plan->d;
  int b = leaf_rows(ctx, plan);
  CK_TRY(omega_draw(ctx, n, d, plan->seed, st));
  ckinv_factor *f = new ckinv_factor();
  f->ctx = ctx;
  f->device = ctx->device;
  f->stream = st;
  f->n = n;
  f->d = d;
  f->tau = kern->nugget;
  f->refine_steps = plan->refine_steps;
  f->prec = plan->prec;
  f->omega_scale = 1.0 / std::sqrt((double)padded_order(n));
  Error e = ok();
  auto alloc = [&](void **p, size_t bytes) {
    if (e.st != CKINV_OK) return;
    cudaError_t ce = dev_alloc(p, bytes, st);
    if (ce != cudaSuccess) e = fail(CKINV_ENOMEM, std::string("factor allocation: ") + cudaGetErrorString(ce));
  };
  const size_t dd = (size_t)d * d;
  alloc((void **)&f->Q, sizeof(float) * (size_t)n * d);
  alloc((void **)&f->R, sizeof(double) * dd);
  alloc((void **)&f->B, sizeof(double) * dd);
  alloc((void **)&f->Cp, sizeof(double) * dd);
  alloc((void **)&f->luB, sizeof(double) * dd * 2);     // luC = luB + d*d
  alloc((void **)&f->pivB, sizeof(int32_t) * d * 2);     // pivC = pivB + d
  if (e.st == CKINV_OK) {
    f->luC = f->luB + dd;
    f->pivC = f->pivB + d;
  }
  alloc((void **)&f->logdet_parts, sizeof(double) * 2);
  alloc((void **)&f->bits, sizeof(uint32_t) * ceil_div(n, 32));
  alloc((void **)&f->cols, sizeof(int32_t) * d);
  if (e.st == CKINV_OK) {
    cudaError_t c1 = cudaMemcpyAsync(f->bits, ctx->om.bits, sizeof(uint32_t) * ceil_div(n, 32),
                                     cudaMemcpyDeviceToDevice, st);
    cudaError_t c2 = cudaMemcpyAsync(f->cols, ctx->om.cols, sizeof(int32_t) * d, cudaMemcpyDeviceToDevice, st);
    if (c1 != cudaSuccess || c2 != cudaSuccess) e = fail(CKINV_ECUDA, "copy of Omega into the factor failed");
  }
  if (e.st == CKINV_OK && plan->omega_kind != 0) {
    f->omega_kind = plan->omega_kind;
    alloc((void **)&f->omega_dense, sizeof(float) * (size_t)n * d);
    if (e.st == CKINV_OK) e = omega_dense(ctx, n, d, plan->seed, plan->omega_kind, f->omega_dense, st);
  }
  if (e.st == CKINV_OK) {
    e = tsqr_factor(ctx, n, d, b, plan->tree_fp64_levels, plan->leaf_fp64 != 0, tsqr_on_tensor_cores(plan), Y, ldy, f->Q,
                    f->R, st);
  }
  if (e.st == CKINV_OK) e = lowrank_core(ctx, f, st);
  if (e.st != CKINV_OK) {
    factor_release(f);
    return e;
  }
  *out = f;
  return ok();
}

bool is_host_pointer(const void *p) {
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return true;
  }
  return a.type == cudaMemoryTypeHost || a.type == cudaMemoryTypeUnregistered;
}

// ------------------------------------------------------------------ small FP64 helpers
// out += x . y in one block (a fixed summation order, so results are reproducible)
__global__ void __launch_bounds__(1024) k_dot(int64_t n, const double *x, int64_t incx, const double *y,
                                              int64_t incy, double *out) {
  __shared__ double red[1024];
  double s = 0.0;
  for (int64_t i = threadIdx.x; i < n; i += blockDim.x) s = fma(x[i * incx], y[i * incy], s);
  red[threadIdx.x] = s;
  __syncthreads();
  for (int o = blockDim.x / 2; o > 0; o >>= 1) {
    if ((int)threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x == 0) *out += red[0];
}

__global__ void __launch_bounds__(1024) k_dot_f32(int64_t n, const float *x, const float *y, double *out) {
  __shared__ double red[1024];
  double s = 0.0;
  for (int64_t i = threadIdx.x; i < n; i += blockDim.x) s = fma((double)x[i], (double)y[i], s);
  red[threadIdx.x] = s;
  __syncthreads();
  for (int o = blockDim.x / 2; o > 0; o >>= 1) {
    if ((int)threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x == 0) *out += red[0];
}

// y = op(A) x  (d x d FP64, ld d)
__global__ void k_gemv(int d, const double *A, const double *x, double *y, int trans) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= d) return;
  double s = 0.0;
  for (int k = 0; k < d; ++k) s = fma(trans ? A[k + (int64_t)i * d] : A[i + (int64_t)k * d], x[k], s);
  y[i] = s;
}

__global__ void k_identity(int d, double *I) {
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < d * d; e += gridDim.x * blockDim.x)
    I[e] = (e % d == e / d) ? 1.0 : 0.0;
}

__global__ void k_transpose(int d, const double *A, double *At) {
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < d * d; e += gridDim.x * blockDim.x) {
    int i = e % d, j = e / d;
    At[j + (int64_t)i * d] = A[e];
  }
}

// Final assembly of the likelihood and its gradient from the reduced scalars:
//   s[0] = y^T alpha, s[1] = <E, G1>, s[2] = gamma^T g3, s[3] = <F, G2>, s[4] = gamma^T G2 gamma,
//   s[5] = <E, R>, s[6] = gamma^T R^T beta, s[7] = <F, B R>, s[8] = gamma^T B R gamma,
//   s[9] = tr(E B), s[10] = alpha^T alpha;  logdet parts lp = [ln|det B|, ln|det C'|].
__global__ void k_finish_nll(const double *s, const double *lp, int64_t n, int d, double tau, double *out) {
  const double two_pi = 6.283185307179586476925286766559;
  double logdet = (double)(n - d) * log(tau) + lp[1] - lp[0];
  out[0] = 0.5 * s[0] + 0.5 * logdet + 0.5 * (double)n * log(two_pi);
  out[1] = s[1] - s[2] - 0.5 * (s[3] - s[4]);
  out[2] = s[5] - s[6] - 0.5 * (s[7] - s[8]);
  double trki = (double)(n - d) / tau + s[9];
  out[3] = 0.5 * tau * (trki - s[10]);
}

// The whole likelihood pipeline enqueued on st, leaving [NLL, d/dlog l, d/dlog variance,
// d/dlog nugget] in out_dev (4 doubles, device memory).  Nothing here waits on the host or
// reads device memory back, so the sequence can be captured into a CUDA graph.
Error nll_grad_enqueue(ckinv_ctx *ctx, const ckinv_plan_desc *plan, const ckinv_kernel *kern, const float *points,
                       const float *y, double *out_dev, cudaStream_t st) {
  CK_TRY(check_plan(plan, kern, true));
  if (kern->kind == CKINV_DENSE) return fail(CKINV_EINVAL, "nll_grad needs a kernel function, not a matrix");
  if (!points || !y || !out_dev) return fail(CKINV_EINVAL, "null argument");
  if (plan->omega_kind != 0) return fail(CKINV_EINVAL, "the likelihood takes the Walsh-Hadamard Omega only");
  const int64_t n = plan->n;
  const int d = plan->d;
  const size_t dd = (size_t)d * d;
  float *Y = nullptr, *Yd = nullptr, *alpha = nullptr;
  double *ws = nullptr;
  ckinv_factor *f = nullptr;
  Error e = ok();
  do {
    if (dev_alloc((void **)&Y, sizeof(float) * n * d, st) != cudaSuccess ||
        dev_alloc((void **)&Yd, sizeof(float) * n * d, st) != cudaSuccess ||
        dev_alloc((void **)&alpha, sizeof(float) * n, st) != cudaSuccess) {
      e = fail(CKINV_ENOMEM, "nll workspace");
      break;
    }
    // ws: G1, G2, E, F, T1, T2 (d x d each), g3, beta, gamma, v1, v2 (d each), s[16]
    const size_t ws_elems = 6 * dd + 5 * (size_t)d + 16;
    if (dev_alloc((void **)&ws, sizeof(double) * ws_elems, st) != cudaSuccess) {
      e = fail(CKINV_ENOMEM, "nll workspace");
      break;
    }
    double *G1 = ws, *G2 = G1 + dd, *E = G2 + dd, *F = E + dd, *T1 = F + dd, *T2 = T1 + dd;
    double *g3 = T2 + dd, *beta = g3 + d, *gamma = beta + d, *v1 = gamma + d, *v2 = v1 + d;
    double *s = v2 + d;
    if (cudaMemsetAsync(s, 0, sizeof(double) * 16, st) != cudaSuccess) {
      e = fail(CKINV_ECUDA, "memset");
      break;
    }
    if ((e = check_finite(ctx, y, n, 1, n, st)).st) break;
    if ((e = do_sketch(ctx, plan, kern, points, nullptr, 0, false, Y, n, st)).st) break;
    if ((e = do_sketch(ctx, plan, kern, points, nullptr, 0, true, Yd, n, st)).st) break;
    if ((e = do_tsqr(ctx, plan, kern, Y, n, &f, st)).st) break;
    if ((e = lowrank_solve(ctx, f, y, n, 1, alpha, n, plan->refine_steps, st)).st) break;
    // beta = Q^T alpha, g3 = Yd^T alpha, G1 = Q^T Yd, G2 = Omega^T Yd
    if ((e = tsprod(ctx, n, d, 1, f->Q, n, nullptr, nullptr, 0, alpha, n, beta, st)).st) break;
    if ((e = tsprod(ctx, n, d, 1, Yd, n, nullptr, nullptr, 0, alpha, n, g3, st)).st) break;
    if ((e = tsprod(ctx, n, d, d, f->Q, n, nullptr, nullptr, 0, Yd, n, G1, st)).st) break;
    if (omega_by_transform(plan->prec, n, d)) {
      // G2 = Omega^T Yd through the fast transform over Yd's columns (FP32)
      if ((e = omega_t_times_wht(ctx, n, d, Yd, n, f->bits, f->cols, f->omega_scale, G2, st)).st) break;
    } else if (n % 4 == 0 && plan->prec == CKINV_BF16) {
      // G2 = Omega^T Yd on the tensor cores (rows of A are the columns of Yd)
      if ((e = omega_draw(ctx, n, d, plan->seed, st)).st) break;
      if ((e = dense_tc(ctx, d, n, d, 3, Yd, n, f->omega_scale, nullptr, 0, G2, d, 1, st)).st) break;
    } else if ((e = tsprod(ctx, n, d, d, nullptr, 0, f->bits, f->cols, f->omega_scale, Yd, n, G2, st)).st) {
      break;
    }
    // gamma = B^-T beta;  E = C'^-1;  F = B^-T E
    if (cudaMemcpyAsync(gamma, beta, sizeof(double) * d, cudaMemcpyDeviceToDevice, st) != cudaSuccess) {
      e = fail(CKINV_ECUDA, "copy");
      break;
    }
    if ((e = lu_solve_dev(d, 1, f->luB, f->pivB, gamma, 1, st)).st) break;
    ::ckinv::note_launch(), k_identity<<<64, 256, 0, st>>>(d, E);
    if ((e = lu_solve_dev(d, d, f->luC, f->pivC, E, 0, st)).st) break;
    if (cudaMemcpyAsync(F, E, sizeof(double) * dd, cudaMemcpyDeviceToDevice, st) != cudaSuccess) {
      e = fail(CKINV_ECUDA, "copy");
      break;
    }
    if ((e = lu_solve_dev(d, d, f->luB, f->pivB, F, 1, st)).st) break;
    // s0 = y^T alpha
    ::ckinv::note_launch(), k_dot_f32<<<1, 1024, 0, st>>>(n, y, alpha, s + 0);
    // s1 = <E, G1>, s3 = <F, G2>
    ::ckinv::note_launch(), k_dot<<<1, 1024, 0, st>>>((int64_t)dd, E, 1, G1, 1, s + 1);
    ::ckinv::note_launch(), k_dot<<<1, 1024, 0, st>>>((int64_t)dd, F, 1, G2, 1, s + 3);
    // s2 = gamma^T g3
    ::ckinv::note_launch(), k_dot<<<1, 1024, 0, st>>>(d, gamma, 1, g3, 1, s + 2);
    // s4 = gamma^T G2 gamma
    ::ckinv::note_launch(), k_gemv<<<(d + 127) / 128, 128, 0, st>>>(d, G2, gamma, v1, 0);
    ::ckinv::note_launch(), k_dot<<<1, 1024, 0, st>>>(d, gamma, 1, v1, 1, s + 4);
    // s5 = <E, R>, s6 = gamma^T R^T beta
    ::ckinv::note_launch(), k_dot<<<1, 1024, 0, st>>>((int64_t)dd, E, 1, f->R, 1, s + 5);
    ::ckinv::note_launch(), k_gemv<<<(d + 127) / 128, 128, 0, st>>>(d, f->R, beta, v1, 1);
    ::ckinv::note_launch(), k_dot<<<1, 1024, 0, st>>>(d, gamma, 1, v1, 1, s + 6);
    // T1 = B R;  s7 = <F, B R>;  s8 = gamma^T B R gamma
    if ((e = gemm_small_dev(d, d, f->B, f->R, T1, 0, st)).st) break;
    ::ckinv::note_launch(), k_dot<<<1, 1024, 0, st>>>((int64_t)dd, F, 1, T1, 1, s + 7);
    ::ckinv::note_launch(), k_gemv<<<(d + 127) / 128, 128, 0, st>>>(d, T1, gamma, v2, 0);
    ::ckinv::note_launch(), k_dot<<<1, 1024, 0, st>>>(d, gamma, 1, v2, 1, s + 8);
    // s9 = tr(E B) = <E^T, B>;  s10 = alpha^T alpha
    ::ckinv::note_launch(), k_transpose<<<64, 256, 0, st>>>(d, E, T2);
    ::ckinv::note_launch(), k_dot<<<1, 1024, 0, st>>>((int64_t)dd, T2, 1, f->B, 1, s + 9);
    ::ckinv::note_launch(), k_dot_f32<<<1, 1024, 0, st>>>(n, alpha, alpha, s + 10);
    ::ckinv::note_launch(), k_finish_nll<<<1, 1, 0, st>>>(s, f->logdet_parts, n, d, f->tau, out_dev);
    cudaError_t le = cudaGetLastError();
    if (le != cudaSuccess) e = fail(CKINV_ECUDA, cudaGetErrorString(le));
  } while (0);
  factor_release(f);
  for (void *p : {(void *)Y, (void *)Yd, (void *)alpha, (void *)ws})
    if (p) cudaFreeAsync(p, st);
  return e;
}

Error do_nll_grad(ckinv_ctx *ctx, const ckinv_plan_desc *plan, const ckinv_kernel *kern, const float *points,
                  const float *y, double *nll, double *grad, cudaStream_t st) {
  if (!nll || !grad) return fail(CKINV_EINVAL, "null argument");
  double *dout = nullptr;
  CK_CUDA(dev_alloc((void **)&dout, sizeof(double) * 4, st));
  Error e = nll_grad_enqueue(ctx, plan, kern, points, y, dout, st);
  double hout[4] = {0, 0, 0, 0};
  if (e.st == CKINV_OK && cudaMemcpyAsync(hout, dout, sizeof(hout), cudaMemcpyDeviceToHost, st) != cudaSuccess)
    e = fail(CKINV_ECUDA, "copy of the likelihood to the host failed");
  cudaFreeAsync(dout, st);
  if (cudaStreamSynchronize(st) != cudaSuccess && e.st == CKINV_OK)
    e = fail(CKINV_ECUDA, cudaGetErrorString(cudaGetLastError()));
  if (e.st == CKINV_OK) e = read_device_error(ctx, st);
  if (e.st == CKINV_OK) {
    *nll = hout[0];
    grad[0] = hout[1];
    grad[1] = hout[2];
    grad[2] = hout[3];
  }
  return e;
}

// ------------------------------------------------------------------ batched likelihood
// Every problem gets a context of its own (its Omega buffers are reserved here, so nothing
// allocates through the context during capture); the problems' pipelines are captured on
// kBatchStreams forked streams of one CUDA graph, which is instantiated and launched.  The
// instantiated graph is kept on the calling context with everything it refers to (the
// per-problem contexts, the pinned upload arena, the output buffer): a later call with the
// same problems - the same descriptors and the same input pointers - launches it again
// without capturing or instantiating anything.
constexpr int kBatchStreams = 8;

}  // namespace

struct ckinv_batch_graph {
  std::vector<unsigned char> key;            // descriptors and pointers of the captured batch
  std::vector<ckinv_ctx *> sub;
  ckinv::UploadArena arena;
  double *d_out = nullptr;
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  int nprob = 0;
};

namespace {

void batch_graph_release(ckinv_batch_graph *b) {
  if (!b) return;
  if (b->exec) cudaGraphExecDestroy(b->exec);
  if (b->graph) cudaGraphDestroy(b->graph);
  for (ckinv_ctx *c : b->sub) {
    if (!c) continue;
    for (void *q : {(void *)c->d_err, (void *)c->hist, (void *)c->cand, (void *)c->cand_idx, (void *)c->small,
                    (void *)c->om.bits, (void *)c->om.cols, (void *)c->om.omegaT})
      if (q) cudaFree(q);
    delete c;
  }
  if (b->arena.host) cudaFreeHost(b->arena.host);
  if (b->d_out) cudaFree(b->d_out);
  delete b;
}

std::vector<unsigned char> batch_key(int nprob, const ckinv_plan_desc *plans, const ckinv_kernel *kerns,
                                     const float *const *points, const float *const *y) {
  std::vector<unsigned char> k;
  auto put = [&](const void *p, size_t n) {
    const unsigned char *c = static_cast<const unsigned char *>(p);
    k.insert(k.end(), c, c + n);
  };
  put(&nprob, sizeof(nprob));
  put(plans, sizeof(ckinv_plan_desc) * nprob);
  put(kerns, sizeof(ckinv_kernel) * nprob);
  put(points, sizeof(const float *) * nprob);
  put(y, sizeof(const float *) * nprob);
  return k;
}

// Launch a captured batch and read its results and the problems' device errors.
Error batch_graph_run(ckinv_batch_graph *b, cudaStream_t st, double *nll, double *grad) {
  std::vector<double> hout((size_t)b->nprob * 4, 0.0);
  ::ckinv::note_launch();
  cudaError_t ce;
  if ((ce = cudaGraphLaunch(b->exec, st)) != cudaSuccess ||
      (ce = cudaMemcpyAsync(hout.data(), b->d_out, sizeof(double) * 4 * b->nprob, cudaMemcpyDeviceToHost, st)) !=
          cudaSuccess ||
      (ce = cudaStreamSynchronize(st)) != cudaSuccess)
    return fail(CKINV_ECUDA, std::string("batched graph: ") + cudaGetErrorString(ce));
  for (int p = 0; p < b->nprob; ++p) {
    Error pe = read_device_error(b->sub[p], st);
    if (pe.st) return fail(pe.st, "problem " + std::to_string(p) + ": " + pe.msg);
  }
  for (int p = 0; p < b->nprob; ++p) {
    nll[p] = hout[4 * p];
    for (int k = 0; k < 3; ++k) grad[3 * p + k] = hout[4 * p + 1 + k];
  }
  return ok();
}

Error do_nll_grad_batched(ckinv_ctx *ctx, int nprob, const ckinv_plan_desc *plans, const ckinv_kernel *kerns,
                          const float *const *points, const float *const *y, double *nll, double *grad,
                          cudaStream_t st) {
  std::vector<unsigned char> key = batch_key(nprob, plans, kerns, points, y);
  if (ctx->batch && ctx->batch->key == key) return batch_graph_run(ctx->batch, st, nll, grad);
  std::vector<ckinv_plan_desc> pl(plans, plans + nprob);
  for (int p = 0; p < nprob; ++p) {
    CK_TRY(check_plan(&pl[p], &kerns[p], true));
    if (kerns[p].kind == CKINV_DENSE) return fail(CKINV_EINVAL, "nll_grad needs a kernel function, not a matrix");
    if (!points[p] || !y[p]) return fail(CKINV_EINVAL, "null points or targets");
  }
  // leaf heights: the autotuner's choice for each shape class not tuned yet
  for (int p = 0; p < nprob; ++p) {
    if (pl[p].block_rows) continue;
    bool known;
    {
      std::lock_guard<std::mutex> lk(g_tune_mu);
      known = g_tuned.count(tune_key(ctx, &pl[p])) != 0;
    }
    int b = 0;
    if (!known) CK_TRY(autotune_leaf_rows(ctx, &pl[p], st, &b));
    pl[p].block_rows = leaf_rows(ctx, &pl[p]);
  }
  // a new batch replaces the kept one
  if (ctx->batch) {
    cudaStreamSynchronize(st);
    batch_graph_release(ctx->batch);
    ctx->batch = nullptr;
  }
  ckinv_batch_graph *bg = new ckinv_batch_graph();
  bg->key = key;
  bg->nprob = nprob;
  bg->sub.assign(nprob, nullptr);
  const int ns = std::min(nprob, kBatchStreams);
  std::vector<cudaStream_t> ws(ns, nullptr);
  std::vector<cudaEvent_t> join(ns, nullptr);
  cudaEvent_t fork = nullptr;
  cudaStream_t cap = nullptr;   // the capture origin (the caller's stream may be the legacy one)
  Error e = ok();
  do {
    for (int p = 0; p < nprob && !e.st; ++p) {
      bg->sub[p] = new ckinv_ctx();
      bg->sub[p]->device = ctx->device;
      bg->sub[p]->sm_count = ctx->sm_count;
      bg->sub[p]->wait_ns = ctx->wait_ns;
      if (cudaMalloc((void **)&bg->sub[p]->d_err, sizeof(int)) != cudaSuccess ||
          cudaMemsetAsync(bg->sub[p]->d_err, 0, sizeof(int), st) != cudaSuccess) {
        e = fail(CKINV_ENOMEM, "batch context");
        break;
      }
      e = omega_reserve(bg->sub[p], pl[p].n, pl[p].d, st);
    }
    if (e.st) break;
    bg->arena.cap = ((size_t)1 << 20) + (size_t)nprob * (256 << 10);
    if (cudaMallocHost((void **)&bg->arena.host, bg->arena.cap) != cudaSuccess ||
        cudaMalloc((void **)&bg->d_out, sizeof(double) * 4 * nprob) != cudaSuccess) {
      e = fail(CKINV_ENOMEM, "batch buffers");
      break;
    }
    if (cudaEventCreateWithFlags(&fork, cudaEventDisableTiming) != cudaSuccess ||
        cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking) != cudaSuccess) {
      e = fail(CKINV_ECUDA, "batch events");
      break;
    }
    for (int w = 0; w < ns && !e.st; ++w)
      if (cudaStreamCreateWithFlags(&ws[w], cudaStreamNonBlocking) != cudaSuccess ||
          cudaEventCreateWithFlags(&join[w], cudaEventDisableTiming) != cudaSuccess)
        e = fail(CKINV_ECUDA, "batch streams");
    if (e.st) break;
    if (cudaStreamSynchronize(st) != cudaSuccess) {   // reservations are in place
      e = fail(CKINV_ECUDA, cudaGetErrorString(cudaGetLastError()));
      break;
    }
    if (cudaStreamBeginCapture(cap, cudaStreamCaptureModeRelaxed) != cudaSuccess) {
      e = fail(CKINV_ECUDA, "cudaStreamBeginCapture failed");
      break;
    }
    cudaEventRecord(fork, cap);
    for (int w = 0; w < ns; ++w) cudaStreamWaitEvent(ws[w], fork, 0);
    for (int p = 0; p < nprob && !e.st; ++p) {
      bg->sub[p]->capture_arena = &bg->arena;
      e = nll_grad_enqueue(bg->sub[p], &pl[p], &kerns[p], points[p], y[p], bg->d_out + 4 * p, ws[p % ns]);
      bg->sub[p]->capture_arena = nullptr;
    }
    for (int w = 0; w < ns; ++w) {
      cudaEventRecord(join[w], ws[w]);
      cudaStreamWaitEvent(cap, join[w], 0);
    }
    cudaError_t ce = cudaStreamEndCapture(cap, &bg->graph);
    if (e.st) break;
    if (ce != cudaSuccess || !bg->graph) {
      e = fail(CKINV_ECUDA, std::string("graph capture of the batch failed: ") + cudaGetErrorString(ce));
      break;
    }
    if ((ce = cudaGraphInstantiate(&bg->exec, bg->graph, 0)) != cudaSuccess) {
      e = fail(CKINV_ECUDA, std::string("graph instantiation failed: ") + cudaGetErrorString(ce));
      break;
    }
    e = batch_graph_run(bg, st, nll, grad);
  } while (0);
  cudaStreamSynchronize(st);
  for (int w = 0; w < ns; ++w) {
    if (ws[w]) cudaStreamDestroy(ws[w]);
    if (join[w]) cudaEventDestroy(join[w]);
  }
  if (fork) cudaEventDestroy(fork);
  if (cap) cudaStreamDestroy(cap);
  if (e.st) {
    batch_graph_release(bg);
    return e;
  }
  ctx->batch = bg;
  return ok();
}

}  // namespace

void ckinv::set_static_error(const std::string &msg) { g_static_err = msg; }

// ====================================================================== exported ABI
extern "C" {

const char *ckinv_version(void) { return "ckinv 0.1 (sm_103a)"; }

unsigned long long ckinv_kernel_launches(void) { return __atomic_load_n(&launch_counter(), __ATOMIC_RELAXED); }

ckinv_status ckinv_create(ckinv_ctx **out, int device) {
  if (!out) return finish(nullptr, fail(CKINV_EINVAL, "ctx pointer is null"));
  *out = nullptr;
  int count = 0;
  if (cudaGetDeviceCount(&count) != cudaSuccess || count == 0) {
    cudaGetLastError();
    return finish(nullptr, fail(CKINV_EUNSUPPORTED, "no CUDA device"));
  }
  if (device < 0 || device >= count) return finish(nullptr, fail(CKINV_EINVAL, "device index out of range"));
  cudaDeviceProp prop;
  if (cudaGetDeviceProperties(&prop, device) != cudaSuccess)
    return finish(nullptr, fail(CKINV_ECUDA, "cudaGetDeviceProperties failed"));
  if (!(prop.major == 10 && prop.minor == 3))
    return finish(nullptr, fail(CKINV_EUNSUPPORTED, "this build targets sm_103 (GB300) only"));
  DeviceGuard g(device);
  ckinv_ctx *ctx = new ckinv_ctx();
  ctx->device = device;
  ctx->sm_count = prop.multiProcessorCount;
  if (cudaMalloc((void **)&ctx->d_err, sizeof(int)) != cudaSuccess || cudaMemset(ctx->d_err, 0, sizeof(int)) != cudaSuccess) {
    delete ctx;
    return finish(nullptr, fail(CKINV_ENOMEM, "context allocation failed"));
  }
  if (device < kPoolDevices) {
    std::lock_guard<std::mutex> lk(g_pool_mu);
    ++g_live_ctx[device];
  }
  *out = ctx;
  return CKINV_OK;
}

ckinv_status ckinv_destroy(ckinv_ctx *ctx) {
  if (!ctx) return CKINV_OK;
  DeviceGuard g(ctx->device);
  cudaDeviceSynchronize();
  for (auto &sl : ctx->stage) {
    if (sl.host) cudaFreeHost(sl.host);
    if (sl.done) cudaEventDestroy(sl.done);
  }
  for (void *p : {(void *)ctx->d_err, (void *)ctx->hist, (void *)ctx->cand, (void *)ctx->cand_idx,
                  (void *)ctx->small, (void *)ctx->om.bits, (void *)ctx->om.cols, (void *)ctx->om.omegaT})
    if (p) cudaFree(p);
  batch_graph_release(ctx->batch);
  if (ctx->device < kPoolDevices) {
    std::lock_guard<std::mutex> lk(g_pool_mu);
    if (--g_live_ctx[ctx->device] == 0 && g_pool[ctx->device]) cudaMemPoolTrimTo(g_pool[ctx->device], 0);
  }
  delete ctx;
  return CKINV_OK;
}

const char *ckinv_last_error(const ckinv_ctx *ctx) {
  return ctx ? ctx->err.c_str() : g_static_err.c_str();
}

ckinv_status ckinv_set_wait_limit(ckinv_ctx *ctx, uint64_t nanoseconds) {
  if (!ctx) return finish(nullptr, fail(CKINV_EINVAL, "null context"));
  if (nanoseconds > 60000000000ull) return finish(ctx, fail(CKINV_EINVAL, "wait limit above 60 s"));
  ctx->wait_ns = nanoseconds ? nanoseconds : kDefaultWaitNs;
  return CKINV_OK;
}

ckinv_status ckinv_check(ckinv_ctx *ctx, ckinv_stream stream) {
  if (!ctx) return finish(nullptr, fail(CKINV_EINVAL, "null context"));
  DeviceGuard g(ctx->device);
  Error e = read_device_error(ctx, (cudaStream_t)stream);
  if (e.st == CKINV_OK) {
    cudaError_t le = cudaGetLastError();
    if (le != cudaSuccess) e = fail(CKINV_ECUDA, cudaGetErrorString(le));
  }
  return finish(ctx, e);
}

ckinv_status ckinv_omega(ckinv_ctx *ctx, int64_t n, int32_t d, uint64_t seed, uint32_t *sign_bits, int32_t *cols,
                         ckinv_stream stream) {
  if (!ctx) return finish(nullptr, fail(CKINV_EINVAL, "null context"));
  if (d < 1 || n < 1 || (int64_t)d > padded_order(n) || d > 4096)
    return finish(ctx, fail(CKINV_EINVAL, "need 1 <= d <= min(N, 4096)"));
  DeviceGuard g(ctx->device);
  cudaStream_t st = (cudaStream_t)stream;
  Error e = omega_draw(ctx, n, d, seed, st);
  if (e.st == CKINV_OK && sign_bits) {
    cudaError_t c = cudaMemcpyAsync(sign_bits, ctx->om.bits, sizeof(uint32_t) * ceil_div(n, 32),
                                    cudaMemcpyDeviceToDevice, st);
    if (c != cudaSuccess) e = fail(CKINV_ECUDA, cudaGetErrorString(c));
  }
  if (e.st == CKINV_OK && cols) {
    cudaError_t c = cudaMemcpyAsync(cols, ctx->om.cols, sizeof(int32_t) * d, cudaMemcpyDeviceToDevice, st);
    if (c != cudaSuccess) e = fail(CKINV_ECUDA, cudaGetErrorString(c));
  }
  return finish(ctx, e);
}

ckinv_status ckinv_omega_matrix(ckinv_ctx *ctx, int64_t n, int32_t d, uint64_t seed, int32_t kind, float *Omega,
                                int64_t ldo, ckinv_stream stream) {
  if (!ctx) return finish(nullptr, fail(CKINV_EINVAL, "null context"));
  if (!Omega || n < 1 || d < 1 || ldo < n || kind < 0 || kind > 3 || d > 4096 ||
      (int64_t)d > (kind == 0 ? padded_order(n) : n))
    return finish(ctx, fail(CKINV_EINVAL, "need Omega, ldo >= n, 0 <= kind <= 3, 1 <= d <= min(4096, N or n)"));
  DeviceGuard g(ctx->device);
  cudaStream_t st = (cudaStream_t)stream;
  if (ldo == n) return finish(ctx, omega_dense(ctx, n, d, seed, kind, Omega, st));
  float *tmp = nullptr;
  if (dev_alloc(&tmp, sizeof(float) * (size_t)n * d, st) != cudaSuccess)
    return finish(ctx, fail(CKINV_ENOMEM, "Omega workspace"));
  Error e = omega_dense(ctx, n, d, seed, kind, tmp, st);
  if (e.st == CKINV_OK && cudaMemcpy2DAsync(Omega, sizeof(float) * ldo, tmp, sizeof(float) * n, sizeof(float) * n, d,
                                            cudaMemcpyDeviceToDevice, st) != cudaSuccess)
    e = fail(CKINV_ECUDA, "copy of Omega failed");
  cudaFreeAsync(tmp, st);
  return finish(ctx, e);
}

ckinv_status ckinv_sketch(ckinv_ctx *ctx, const ckinv_plan_desc *plan, const ckinv_kernel *kern, const float *points,
                          const float *K, int64_t ldk, float *Y, int64_t ldy, ckinv_stream stream) {
  if (!ctx) return finish(nullptr, fail(CKINV_EINVAL, "null context"));
  DeviceGuard g(ctx->device);
  return finish(ctx, do_sketch(ctx, plan, kern, points, K, ldk, false, Y, ldy, (cudaStream_t)stream));
}

ckinv_status ckinv_kernel_matrix(ckinv_ctx *ctx, const ckinv_plan_desc *plan, const ckinv_kernel *kern,
                                 const float *points, float *K, int64_t ldk, ckinv_stream stream) {
  if (!ctx) return finish(nullptr, fail(CKINV_EINVAL, "null context"));
  DeviceGuard g(ctx->device);
  Error e = check_plan(plan, kern, true);
  if (e.st == CKINV_OK && kern->kind == CKINV_DENSE) e = fail(CKINV_EINVAL, "a kernel function is needed");
  if (e.st == CKINV_OK && (!points || !K || ldk < plan->n)) e = fail(CKINV_EINVAL, "need points, K and ldk >= n");
  cudaStream_t st = (cudaStream_t)stream;
  if (e.st == CKINV_OK) e = check_finite(ctx, points, plan->dim, plan->n, plan->dim, st);
  if (e.st == CKINV_OK) e = kernel_matrix(ctx, plan->n, plan->dim, make_params(plan, kern), points, K, ldk, st);
  return finish(ctx, e);
}

ckinv_status ckinv_sketch_dlogl(ckinv_ctx *ctx, const ckinv_plan_desc *plan, const ckinv_kernel *kern,
                                const float *points, float *Yd, int64_t ldy, ckinv_stream stream) {
  if (!ctx) return finish(nullptr, fail(CKINV_EINVAL, "null context"));
  DeviceGuard g(ctx->device);
  return finish(ctx, do_sketch(ctx, plan, kern, points, nullptr, 0, true, Yd, ldy, (cudaStream_t)stream));
}

ckinv_status ckinv_tsqr(ckinv_ctx *ctx, const ckinv_plan_desc *plan, const ckinv_kernel *kern, float *Y, int64_t ldy,
                        ckinv_factor **out, ckinv_stream stream) {
  if (!ctx) return finish(nullptr, fail(CKINV_EINVAL, "null context"));
  DeviceGuard g(ctx->device);
  return finish(ctx, do_tsqr(ctx, plan, kern, Y, ldy, out, (cudaStream_t)stream));
}

ckinv_status ckinv_factor_free(ckinv_factor *f) {
  if (!f) return CKINV_OK;
  DeviceGuard g(f->device);
  factor_release(f);
  return CKINV_OK;
}

ckinv_status ckinv_factor_r(const ckinv_factor *f, double *R, ckinv_stream stream) {
  if (!f || !R) return finish(nullptr, fail(CKINV_EINVAL, "null argument"));
  DeviceGuard g(f->device);
  cudaError_t c = cudaMemcpyAsync(R, f->R, sizeof(double) * f->d * f->d, cudaMemcpyDeviceToDevice, (cudaStream_t)stream);
  return finish(f->ctx, c == cudaSuccess ? ok() : fail(CKINV_ECUDA, cudaGetErrorString(c)));
}

ckinv_status ckinv_factor_q(const ckinv_factor *f, float *Q, int64_t ldq, ckinv_stream stream) {
  if (!f || !Q || ldq < f->n) return finish(nullptr, fail(CKINV_EINVAL, "null argument or ldq < n"));
  DeviceGuard g(f->device);
  cudaError_t c = cudaMemcpy2DAsync(Q, sizeof(float) * ldq, f->Q, sizeof(float) * f->n, sizeof(float) * f->n, f->d,
                                    cudaMemcpyDeviceToDevice, (cudaStream_t)stream);
  return finish(f->ctx, c == cudaSuccess ? ok() : fail(CKINV_ECUDA, cudaGetErrorString(c)));
}

ckinv_status ckinv_factor_core(const ckinv_factor *f, double *B, double *Cp, double *logdet, ckinv_stream stream) {
  if (!f) return finish(nullptr, fail(CKINV_EINVAL, "null factor"));
  DeviceGuard g(f->device);
  cudaStream_t st = (cudaStream_t)stream;
  const size_t bytes = sizeof(double) * f->d * f->d;
  if (B && cudaMemcpyAsync(B, f->B, bytes, cudaMemcpyDeviceToDevice, st) != cudaSuccess)
    return finish(f->ctx, fail(CKINV_ECUDA, "copy of B failed"));
  if (Cp && cudaMemcpyAsync(Cp, f->Cp, bytes, cudaMemcpyDeviceToDevice, st) != cudaSuccess)
    return finish(f->ctx, fail(CKINV_ECUDA, "copy of C' failed"));
  if (logdet) {
    double lp[2];
    if (cudaMemcpyAsync(lp, f->logdet_parts, sizeof(lp), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
        cudaStreamSynchronize(st) != cudaSuccess)
      return finish(f->ctx, fail(CKINV_ECUDA, "copy of log-determinants failed"));
    *logdet = (double)(f->n - f->d) * std::log(f->tau) + lp[1] - lp[0];
  }
  return CKINV_OK;
}

// ------------------------------------------------------------------ row shards
ckinv_status ckinv_sketch_rows(ckinv_ctx *ctx, const ckinv_plan_desc *plan, const ckinv_kernel *kern,
                               const float *points, const float *K, int64_t ldk, int64_t row0, int64_t m, float *Y,
                               int64_t ldy, ckinv_stream stream) {
  if (!ctx) return finish(nullptr, fail(CKINV_EINVAL, "null context"));
  DeviceGuard g(ctx->device);
  return finish(ctx, do_sketch(ctx, plan, kern, points, K, ldk, false, Y, ldy, (cudaStream_t)stream, row0, m));
}

ckinv_status ckinv_tsqr_shard(ckinv_ctx *ctx, const ckinv_plan_desc *plan, const ckinv_kernel *kern, float *Y,
                              int64_t ldy, int64_t row0, int64_t m, ckinv_factor **out, double *R_local,
                              ckinv_stream stream) {
  if (!ctx) return finish(nullptr, fail(CKINV_EINVAL, "null context"));
  DeviceGuard g(ctx->device);
  cudaStream_t st = (cudaStream_t)stream;
  Error e = check_plan(plan, kern, false);
  if (e.st == CKINV_OK && (!Y || !out || !R_local || row0 < 0 || m < plan->d || row0 + m > plan->n || ldy < m))
    e = fail(CKINV_EINVAL, "need Y, out, R_local, 0 <= row0, d <= m, row0 + m <= n, ldy >= m");
  if (e.st == CKINV_OK && plan->omega_kind != 0) e = fail(CKINV_EINVAL, "row shards take the Walsh-Hadamard Omega only");
  if (e.st) return finish(ctx, e);
  *out = nullptr;
  const int d = plan->d;
  ckinv_plan_desc local = *plan;
  local.n = m;
  int b = leaf_rows(ctx, &local);
  e = omega_draw(ctx, plan->n, d, plan->seed, st);
  if (e.st) return finish(ctx, e);
  ckinv_factor *f = new ckinv_factor();
  f->ctx = ctx;
  f->device = ctx->device;
  f->stream = st;
  f->n = m;
  f->d = d;
  f->tau = kern->nugget;
  f->refine_steps = 0;
  f->prec = plan->prec;
  f->omega_scale = 1.0 / std::sqrt((double)padded_order(plan->n));
  f->row0 = row0;
  f->n_total = plan->n;
  auto alloc = [&](void **p, size_t bytes) {
    if (e.st != CKINV_OK) return;
    cudaError_t ce = dev_alloc(p, bytes, st);
    if (ce != cudaSuccess) e = fail(CKINV_ENOMEM, std::string("factor allocation: ") + cudaGetErrorString(ce));
  };
  const size_t dd = (size_t)d * d;
  alloc((void **)&f->Q, sizeof(float) * (size_t)m * d);
  alloc((void **)&f->R, sizeof(double) * dd);
  alloc((void **)&f->B, sizeof(double) * dd);
  alloc((void **)&f->Cp, sizeof(double) * dd);
  alloc((void **)&f->luB, sizeof(double) * dd * 2);
  alloc((void **)&f->pivB, sizeof(int32_t) * d * 2);
  if (e.st == CKINV_OK) {
    f->luC = f->luB + dd;
    f->pivC = f->pivB + d;
  }
  alloc((void **)&f->logdet_parts, sizeof(double) * 2);
  alloc((void **)&f->bits, sizeof(uint32_t) * ceil_div(plan->n, 32));
  alloc((void **)&f->cols, sizeof(int32_t) * d);
  if (e.st == CKINV_OK &&
      (cudaMemcpyAsync(f->bits, ctx->om.bits, sizeof(uint32_t) * ceil_div(plan->n, 32), cudaMemcpyDeviceToDevice, st) !=
           cudaSuccess ||
       cudaMemcpyAsync(f->cols, ctx->om.cols, sizeof(int32_t) * d, cudaMemcpyDeviceToDevice, st) != cudaSuccess))
    e = fail(CKINV_ECUDA, "copy of Omega into the factor failed");
  if (e.st == CKINV_OK)
    e = tsqr_factor(ctx, m, d, b, plan->tree_fp64_levels, plan->leaf_fp64 != 0, tsqr_on_tensor_cores(plan), Y, ldy,
                    f->Q, f->R, st);
  if (e.st == CKINV_OK && cudaMemcpyAsync(R_local, f->R, sizeof(double) * dd, cudaMemcpyDeviceToDevice, st) !=
                              cudaSuccess)
    e = fail(CKINV_ECUDA, "copy of R failed");
  if (e.st != CKINV_OK) {
    factor_release(f);
    return finish(ctx, e);
  }
  *out = f;
  return CKINV_OK;
}

ckinv_status ckinv_shard_combine(ckinv_ctx *ctx, ckinv_factor *f, const double *R_all, int32_t G, int32_t g,
                                 double *B_partial, ckinv_stream stream) {
  if (!ctx || !f) return finish(ctx, fail(CKINV_EINVAL, "null context or factor"));
  if (!R_all || !B_partial || G < 1 || g < 0 || g >= G || f->n_total == 0)
    return finish(ctx, fail(CKINV_EINVAL, "need a shard factor, R_all, B_partial and 0 <= g < G"));
  DeviceGuard gd(ctx->device);
  cudaStream_t st = (cudaStream_t)stream;
  const int d = f->d;
  const size_t dd = (size_t)d * d;
  double *X = nullptr;
  float *X32 = nullptr, *Qn = nullptr;
  Error e = ok();
  do {
    if (dev_alloc(&X, sizeof(double) * G * dd, st) != cudaSuccess || dev_alloc(&X32, sizeof(float) * dd, st) != cudaSuccess ||
        dev_alloc(&Qn, sizeof(float) * (size_t)f->n * d, st) != cudaSuccess) {
      e = fail(CKINV_ENOMEM, "shard combine workspace");
      break;
    }
    // the top of the tree over all shards' R factors (every rank computes it redundantly)
    if ((e = tsqr_combine_r(ctx, G, d, R_all, f->R, X, st)).st) break;
    note_launch();
    k_narrow_f64<<<64, 256, 0, st>>>(X + (size_t)g * dd, (int64_t)dd, X32);
    cudaError_t ce = cudaGetLastError();
    if (ce != cudaSuccess) {
      e = fail(CKINV_ECUDA, cudaGetErrorString(ce));
      break;
    }
    // this shard's rows of Q_hat: its own Q_hat times its block of the top Q factor
    if ((e = gemm_batched<float>(ctx, false, (int)f->n, d, d, 1.0f, f->Q, f->n, 0, X32, d, 0, 0.0f, Qn, f->n, 0, 1,
                                 st)).st)
      break;
    std::swap(f->Q, Qn);
    // B_partial = Omega[row0 : row0 + n_local]^T Q_hat_local
    e = tsprod(ctx, f->n, d, d, nullptr, 0, f->bits, f->cols, f->omega_scale, f->Q, f->n, B_partial, st, f->row0);
  } while (0);
  for (void *p : {(void *)X, (void *)X32, (void *)Qn})
    if (p) cudaFreeAsync(p, st);
  return finish(ctx, e);
}

ckinv_status ckinv_shard_core(ckinv_ctx *ctx, ckinv_factor *f, const double *B, ckinv_stream stream) {
  if (!ctx || !f || !B) return finish(ctx, fail(CKINV_EINVAL, "null argument"));
  DeviceGuard g(ctx->device);
  cudaStream_t st = (cudaStream_t)stream;
  if (cudaMemcpyAsync(f->B, B, sizeof(double) * f->d * f->d, cudaMemcpyDeviceToDevice, st) != cudaSuccess)
    return finish(ctx, fail(CKINV_ECUDA, "copy of B failed"));
  return finish(ctx, core_from_b(ctx, f, st));
}

ckinv_status ckinv_shard_solve_begin(ckinv_ctx *ctx, const ckinv_factor *f, const float *A, int64_t lda, int32_t m,
                                     double *Z_partial, ckinv_stream stream) {
  if (!ctx || !f || !A || !Z_partial || lda < f->n || m < 1 || m > 256)
    return finish(ctx, fail(CKINV_EINVAL, "need A, Z_partial, lda >= rows, 1 <= m <= 256"));
  DeviceGuard g(ctx->device);
  cudaStream_t st = (cudaStream_t)stream;
  Error e = check_finite(ctx, A, f->n, m, lda, st);
  if (e.st == CKINV_OK) e = tsprod(ctx, f->n, f->d, m, f->Q, f->n, nullptr, nullptr, 0.0, A, lda, Z_partial, st);
  return finish(ctx, e);
}

ckinv_status ckinv_shard_solve_end(ckinv_ctx *ctx, const ckinv_factor *f, const double *Z, const float *A, int64_t lda,
                                   int32_t m, float *X, int64_t ldx, ckinv_stream stream) {
  if (!ctx || !f || !Z || !A || !X || lda < f->n || ldx < f->n || m < 1 || m > 256)
    return finish(ctx, fail(CKINV_EINVAL, "need Z, A, X, lda/ldx >= rows, 1 <= m <= 256"));
  DeviceGuard g(ctx->device);
  return finish(ctx, solve_from_z(ctx, f, Z, A, lda, m, X, ldx, (cudaStream_t)stream));
}

ckinv_status ckinv_factor_project(ckinv_ctx *ctx, ckinv_factor *f, const ckinv_plan_desc *plan,
                                  const ckinv_kernel *kern, const float *points, double *S, double *colspace_err,
                                  ckinv_stream stream) {
  if (!ctx || !f) return finish(ctx, fail(CKINV_EINVAL, "null context or factor"));
  DeviceGuard g(ctx->device);
  Error e = check_plan(plan, kern, true);
  if (e.st == CKINV_OK && (kern->kind == CKINV_DENSE || !points))
    e = fail(CKINV_EINVAL, "the second pass needs points and a kernel function");
  if (e.st == CKINV_OK && (plan->n != f->n || plan->d != f->d)) e = fail(CKINV_EINVAL, "plan does not match the factor");
  if (e.st == CKINV_OK && f->n_total != 0) e = fail(CKINV_EINVAL, "a shard factor has no second pass");
  cudaStream_t st = (cudaStream_t)stream;
  if (e.st == CKINV_OK) e = check_finite(ctx, points, plan->dim, plan->n, plan->dim, st);
  if (e.st == CKINV_OK) e = two_pass_core(ctx, f, plan->dim, make_params(plan, kern), points, colspace_err, st);
  if (e.st == CKINV_OK && S && cudaMemcpyAsync(S, f->S2, sizeof(double) * f->d * f->d, cudaMemcpyDeviceToDevice, st) !=
                                   cudaSuccess)
    e = fail(CKINV_ECUDA, "copy of S failed");
  return finish(ctx, e);
}

ckinv_status ckinv_predict_mean(ckinv_ctx *ctx, const ckinv_plan_desc *plan, const ckinv_kernel *kern,
                                const float *points, const float *alpha, const float *new_points, int64_t n_new,
                                double *mean, ckinv_stream stream) {
  if (!ctx) return finish(nullptr, fail(CKINV_EINVAL, "null context"));
  DeviceGuard g(ctx->device);
  Error e = check_plan(plan, kern, true);
  if (e.st == CKINV_OK && kern->kind == CKINV_DENSE) e = fail(CKINV_EINVAL, "the predictive mean needs a kernel function");
  if (e.st == CKINV_OK && (!points || !alpha || !new_points || !mean || n_new < 0))
    e = fail(CKINV_EINVAL, "null argument or n_new < 0");
  cudaStream_t st = (cudaStream_t)stream;
  if (e.st == CKINV_OK) e = check_finite(ctx, new_points, plan->dim, n_new, plan->dim, st);
  if (e.st == CKINV_OK && n_new > 0)
    e = predict_mean(ctx, plan->n, plan->dim, make_params(plan, kern), points, alpha, new_points, n_new, mean, st);
  return finish(ctx, e);
}

ckinv_status ckinv_solve(ckinv_ctx *ctx, const ckinv_factor *f, const float *A, int64_t lda, int32_t m, float *X,
                         int64_t ldx, ckinv_stream stream) {
  if (!ctx || !f) return finish(ctx, fail(CKINV_EINVAL, "null context or factor"));
  if (!A || !X || lda < f->n || ldx < f->n || m < 1 || m > 256)
    return finish(ctx, fail(CKINV_EINVAL, "need A, X non-null, lda/ldx >= n, 1 <= m <= 256"));
  DeviceGuard g(ctx->device);
  Error e = check_finite(ctx, A, f->n, m, lda, (cudaStream_t)stream);
  if (e.st == CKINV_OK) e = lowrank_solve(ctx, f, A, lda, m, X, ldx, f->refine_steps, (cudaStream_t)stream);
  return finish(ctx, e);
}

ckinv_status ckinv_kinv_a(ckinv_ctx *ctx, const ckinv_plan_desc *plan, const ckinv_kernel *kern, const float *points,
                          const float *A, int64_t lda, int32_t m, float *X, int64_t ldx, ckinv_stream stream) {
  if (!ctx) return finish(nullptr, fail(CKINV_EINVAL, "null context"));
  DeviceGuard g(ctx->device);
  cudaStream_t st = (cudaStream_t)stream;
  Error e = check_plan(plan, kern, true);
  if (e.st) return finish(ctx, e);
  if (kern->kind == CKINV_DENSE) return finish(ctx, fail(CKINV_EINVAL, "ckinv_kinv_a needs points"));
  if (!points || !A || !X || lda < plan->n || ldx < plan->n || m < 1 || m > 256)
    return finish(ctx, fail(CKINV_EINVAL, "bad points/A/X or leading dimensions"));
  const int64_t n = plan->n;
  const int d = plan->d;
  const bool hp = is_host_pointer(points), ha = is_host_pointer(A), hx = is_host_pointer(X);
  float *dp = nullptr, *dA = nullptr, *dX = nullptr, *Y = nullptr;
  ckinv_factor *f = nullptr;
  do {
    const float *P = points;
    const float *Ad = A;
    int64_t ldad = lda;
    float *Xd = X;
    int64_t ldxd = ldx;
    if (hp) {
      if (dev_alloc((void **)&dp, sizeof(float) * n * plan->dim, st) != cudaSuccess ||
          cudaMemcpyAsync(dp, points, sizeof(float) * n * plan->dim, cudaMemcpyHostToDevice, st) != cudaSuccess) {
        e = fail(CKINV_ECUDA, "staging of points failed");
        break;
      }
      P = dp;
    }
    if (ha) {
      if (dev_alloc((void **)&dA, sizeof(float) * n * m, st) != cudaSuccess ||
          cudaMemcpy2DAsync(dA, sizeof(float) * n, A, sizeof(float) * lda, sizeof(float) * n, m,
                            cudaMemcpyHostToDevice, st) != cudaSuccess) {
        e = fail(CKINV_ECUDA, "staging of A failed");
        break;
      }
      Ad = dA;
      ldad = n;
    }
    if (hx) {
      if (dev_alloc((void **)&dX, sizeof(float) * n * m, st) != cudaSuccess) {
        e = fail(CKINV_ENOMEM, "staging of X failed");
        break;
      }
      Xd = dX;
      ldxd = n;
    }
    if (dev_alloc((void **)&Y, sizeof(float) * n * d, st) != cudaSuccess) {
      e = fail(CKINV_ENOMEM, "sketch allocation failed");
      break;
    }
    if ((e = check_finite(ctx, Ad, n, m, ldad, st)).st) break;
    if ((e = do_sketch(ctx, plan, kern, P, nullptr, 0, false, Y, n, st)).st) break;
    if ((e = do_tsqr(ctx, plan, kern, Y, n, &f, st)).st) break;
    if ((e = lowrank_solve(ctx, f, Ad, ldad, m, Xd, ldxd, plan->refine_steps, st)).st) break;
    if (hx && cudaMemcpy2DAsync(X, sizeof(float) * ldx, dX, sizeof(float) * n, sizeof(float) * n, m,
                                cudaMemcpyDeviceToHost, st) != cudaSuccess) {
      e = fail(CKINV_ECUDA, "copy of X to the host failed");
      break;
    }
  } while (0);
  if (hp || ha || hx || e.st) cudaStreamSynchronize(st);
  if (f) {
    cudaStreamSynchronize(st);
    factor_release(f);
  }
  for (void *p : {(void *)dp, (void *)dA, (void *)dX, (void *)Y})
    if (p) cudaFreeAsync(p, st);
  if (e.st == CKINV_OK && (hp || ha || hx)) e = read_device_error(ctx, st);
  return finish(ctx, e);
}

ckinv_status ckinv_nll_grad(ckinv_ctx *ctx, const ckinv_plan_desc *plan, const ckinv_kernel *kern,
                            const float *points, const float *y, double *nll, double *grad, ckinv_stream stream) {
  if (!ctx) return finish(nullptr, fail(CKINV_EINVAL, "null context"));
  DeviceGuard g(ctx->device);
  return finish(ctx, do_nll_grad(ctx, plan, kern, points, y, nll, grad, (cudaStream_t)stream));
}

ckinv_status ckinv_autotune(ckinv_ctx *ctx, const ckinv_plan_desc *plan, int32_t *block_rows, ckinv_stream stream) {
  if (!ctx) return finish(nullptr, fail(CKINV_EINVAL, "null context"));
  if (!plan || !block_rows) return finish(ctx, fail(CKINV_EINVAL, "null argument"));
  if (plan->d < 16 || plan->d > 512 || plan->d % 16 != 0 || plan->n < plan->d || plan->n > ((int64_t)1 << 31))
    return finish(ctx, fail(CKINV_EINVAL, "need 16 <= d <= 512, d % 16 == 0, d <= n <= 2^31"));
  if (plan->tree_fp64_levels < -1 || (plan->leaf_fp64 != 0 && plan->leaf_fp64 != 1))
    return finish(ctx, fail(CKINV_EINVAL, "bad tree_fp64_levels or leaf_fp64"));
  DeviceGuard g(ctx->device);
  int b = 0;
  Error e = autotune_leaf_rows(ctx, plan, (cudaStream_t)stream, &b);
  if (e.st == CKINV_OK) *block_rows = b;
  return finish(ctx, e);
}

ckinv_status ckinv_nll_grad_batched(ckinv_ctx *ctx, int32_t nprob, const ckinv_plan_desc *plans,
                                    const ckinv_kernel *kerns, const float *const *points, const float *const *y,
                                    double *nll, double *grad, ckinv_stream stream) {
  if (!ctx) return finish(nullptr, fail(CKINV_EINVAL, "null context"));
  if (nprob < 1 || !plans || !kerns || !points || !y || !nll || !grad)
    return finish(ctx, fail(CKINV_EINVAL, "null argument or nprob < 1"));
  DeviceGuard g(ctx->device);
  return finish(ctx, do_nll_grad_batched(ctx, nprob, plans, kerns, points, y, nll, grad, (cudaStream_t)stream));
}

}  // extern "C"
