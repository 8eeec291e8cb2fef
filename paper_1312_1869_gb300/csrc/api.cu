// C ABI of the ckinv library: argument checking, workspace ownership and the order of the
// stages (sketch -> TSQR -> core -> solve -> likelihood and gradient).  All arithmetic of
// the method runs in the kernels of the other translation units.
#include <cmath>
#include <cstdio>
#include <cstring>

#include "internal.cuh"

using namespace ckinv;

Error ckinv::stage_upload(ckinv_ctx *ctx, const void *src, size_t bytes, void *dst, cudaStream_t st) {
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
  if (plan->prec < CKINV_FP32 || plan->prec > CKINV_BF16X3) return fail(CKINV_EINVAL, "unknown precision");
  if (plan->block_rows != 0 && plan->block_rows < plan->d) return fail(CKINV_EINVAL, "block_rows must be >= d");
  if (plan->refine_steps < 0 || plan->refine_steps > 4) return fail(CKINV_EINVAL, "refine_steps must be 0..4");
  if (plan->tree_fp64_levels < -1) return fail(CKINV_EINVAL, "tree_fp64_levels must be >= -1");
  if (plan->leaf_fp64 != 0 && plan->leaf_fp64 != 1) return fail(CKINV_EINVAL, "leaf_fp64 must be 0 or 1");
  return ok();
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
    if (h & DERR_SINGULAR) return fail(CKINV_ESINGULAR, "zero pivot in an LU factorisation");
    if (h & DERR_CAPACITY) return fail(CKINV_EUNSUPPORTED, "device list capacity exceeded (Omega draw)");
  }
  return ok();
}

Error do_sketch(ckinv_ctx *ctx, const ckinv_plan_desc *plan, const ckinv_kernel *kern, const float *points,
                const float *K, int64_t ldk, bool deriv, float *Y, int64_t ldy, cudaStream_t st) {
  CK_TRY(check_plan(plan, kern, true));
  if (!Y || ldy < plan->n) return fail(CKINV_EINVAL, "Y must be non-null with ldy >= n");
  if (kern->kind == CKINV_DENSE) {
    if (!K || ldk < plan->n) return fail(CKINV_EINVAL, "dense kernel needs K with ldk >= n");
    if (deriv) return fail(CKINV_EINVAL, "no derivative sketch for a materialised K");
  } else if (!points) {
    return fail(CKINV_EINVAL, "points must be non-null");
  }
  CK_TRY(omega_draw(ctx, plan->n, plan->d, plan->seed, st));
  KernelParams kp = make_params(plan, kern);
  if (kern->kind == CKINV_DENSE) {
    // K is symmetric: its column i is read as row i (16-byte rows for the tensor-core path)
    if (plan->prec != CKINV_FP32 && ldk % 4 == 0 && (reinterpret_cast<uintptr_t>(K) & 15) == 0)
      return dense_tc(ctx, plan->n, plan->n, plan->d, plan->prec, K, ldk, kp.scale, Y, ldy, nullptr, 0, 0, st);
    return sketch_simt(ctx, plan->n, plan->dim, plan->d, kp, nullptr, K, ldk, false, Y, ldy, st);
  }
  if (plan->prec == CKINV_FP32)
    return sketch_simt(ctx, plan->n, plan->dim, plan->d, kp, points, nullptr, 0, deriv, Y, ldy, st);
  return sketch_tc(ctx, plan->n, plan->dim, plan->d, plan->prec, kp, points, deriv, Y, ldy, st);
}

void factor_release(ckinv_factor *f) {
  if (!f) return;
  for (void *p : {(void *)f->Q, (void *)f->R, (void *)f->B, (void *)f->Cp, (void *)f->luB, (void *)f->pivB,
                  (void *)f->logdet_parts, (void *)f->bits, (void *)f->cols})
    if (p) cudaFreeAsync(p, f->stream);
  delete f;
}

Error do_tsqr(ckinv_ctx *ctx, const ckinv_plan_desc *plan, const ckinv_kernel *kern, float *Y, int64_t ldy,
              ckinv_factor **out, cudaStream_t st) {
  CK_TRY(check_plan(plan, kern, false));
  if (!Y || !out || ldy < plan->n) return fail(CKINV_EINVAL, "Y/out must be non-null, ldy >= n");
  *out = nullptr;
  const int64_t n = plan->n;
  const int d = plan->d;
  int b = plan->block_rows ? plan->block_rows : auto_block_rows(n, d, ctx->sm_count);
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
    cudaError_t ce = cudaMallocAsync(p, bytes, st);
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
  if (e.st == CKINV_OK) {
    e = tsqr_factor(ctx, n, d, b, plan->tree_fp64_levels, plan->leaf_fp64 != 0, Y, ldy, f->Q, f->R, st);
  }
  if (e.st == CKINV_OK) e = lowrank_core(ctx, f, st);
  if (e.st != CKINV_OK) {
    cudaStreamSynchronize(st);
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
__global__ void k_dot(int64_t n, const double *x, int64_t incx, const double *y, int64_t incy, double *out) {
  __shared__ double red[256];
  double s = 0.0;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    s = fma(x[i * incx], y[i * incy], s);
  red[threadIdx.x] = s;
  __syncthreads();
  for (int o = 128; o > 0; o >>= 1) {
    if ((int)threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x == 0) atomicAdd(out, red[0]);
}

__global__ void k_dot_f32(int64_t n, const float *x, const float *y, double *out) {
  __shared__ double red[256];
  double s = 0.0;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    s = fma((double)x[i], (double)y[i], s);
  red[threadIdx.x] = s;
  __syncthreads();
  for (int o = 128; o > 0; o >>= 1) {
    if ((int)threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x == 0) atomicAdd(out, red[0]);
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

Error do_nll_grad(ckinv_ctx *ctx, const ckinv_plan_desc *plan, const ckinv_kernel *kern, const float *points,
                  const float *y, double *nll, double *grad, cudaStream_t st) {
  CK_TRY(check_plan(plan, kern, true));
  if (kern->kind == CKINV_DENSE) return fail(CKINV_EINVAL, "nll_grad needs a kernel function, not a matrix");
  if (!points || !y || !nll || !grad) return fail(CKINV_EINVAL, "null argument");
  const int64_t n = plan->n;
  const int d = plan->d;
  const size_t dd = (size_t)d * d;
  float *Y = nullptr, *Yd = nullptr, *alpha = nullptr;
  double *ws = nullptr;
  CK_CUDA(cudaMallocAsync((void **)&Y, sizeof(float) * n * d, st));
  CK_CUDA(cudaMallocAsync((void **)&Yd, sizeof(float) * n * d, st));
  CK_CUDA(cudaMallocAsync((void **)&alpha, sizeof(float) * n, st));
  // ws: G1, G2, E, F, T1, T2 (d x d each), g3, beta, gamma, v1, v2 (d each), alpha64? no, s[16], out[4]
  const size_t ws_elems = 6 * dd + 5 * (size_t)d + 16 + 4;
  CK_CUDA(cudaMallocAsync((void **)&ws, sizeof(double) * ws_elems, st));
  double *G1 = ws, *G2 = G1 + dd, *E = G2 + dd, *F = E + dd, *T1 = F + dd, *T2 = T1 + dd;
  double *g3 = T2 + dd, *beta = g3 + d, *gamma = beta + d, *v1 = gamma + d, *v2 = v1 + d;
  double *s = v2 + d, *out = s + 16;
  CK_CUDA(cudaMemsetAsync(s, 0, sizeof(double) * 20, st));

  CK_TRY(do_sketch(ctx, plan, kern, points, nullptr, 0, false, Y, n, st));
  CK_TRY(do_sketch(ctx, plan, kern, points, nullptr, 0, true, Yd, n, st));
  ckinv_factor *f = nullptr;
  CK_TRY(do_tsqr(ctx, plan, kern, Y, n, &f, st));
  Error e = ok();
  do {
    e = lowrank_solve(ctx, f, y, n, 1, alpha, n, plan->refine_steps, st);
    if (e.st) break;
    // beta = Q^T alpha, g3 = Yd^T alpha, G1 = Q^T Yd, G2 = Omega^T Yd
    if ((e = tsprod(ctx, n, d, 1, f->Q, n, nullptr, nullptr, 0, alpha, n, beta, st)).st) break;
    if ((e = tsprod(ctx, n, d, 1, Yd, n, nullptr, nullptr, 0, alpha, n, g3, st)).st) break;
    if ((e = tsprod(ctx, n, d, d, f->Q, n, nullptr, nullptr, 0, Yd, n, G1, st)).st) break;
    if (n % 4 == 0 && plan->prec != CKINV_FP32) {
      // G2 = Omega^T Yd on the tensor cores (rows of A are the columns of Yd)
      if ((e = omega_draw(ctx, n, d, plan->seed, st)).st) break;
      if ((e = dense_tc(ctx, d, n, d, 3, Yd, n, f->omega_scale, nullptr, 0, G2, d, 1, st)).st) break;
    } else if ((e = tsprod(ctx, n, d, d, nullptr, 0, f->bits, f->cols, f->omega_scale, Yd, n, G2, st)).st) {
      break;
    }
    // gamma = B^-T beta;  E = C'^-1;  F = B^-T E
    cudaMemcpyAsync(gamma, beta, sizeof(double) * d, cudaMemcpyDeviceToDevice, st);
    if ((e = lu_solve_dev(d, 1, f->luB, f->pivB, gamma, 1, st)).st) break;
    ::ckinv::note_launch(), k_identity<<<64, 256, 0, st>>>(d, E);
    if ((e = lu_solve_dev(d, d, f->luC, f->pivC, E, 0, st)).st) break;
    cudaMemcpyAsync(F, E, sizeof(double) * dd, cudaMemcpyDeviceToDevice, st);
    if ((e = lu_solve_dev(d, d, f->luB, f->pivB, F, 1, st)).st) break;
    const int gb = 64;
    // s0 = y^T alpha
    ::ckinv::note_launch(), k_dot_f32<<<gb, 256, 0, st>>>(n, y, alpha, s + 0);
    // s1 = <E, G1>, s3 = <F, G2>
    ::ckinv::note_launch(), k_dot<<<gb, 256, 0, st>>>((int64_t)dd, E, 1, G1, 1, s + 1);
    ::ckinv::note_launch(), k_dot<<<gb, 256, 0, st>>>((int64_t)dd, F, 1, G2, 1, s + 3);
    // s2 = gamma^T g3
    ::ckinv::note_launch(), k_dot<<<1, 256, 0, st>>>(d, gamma, 1, g3, 1, s + 2);
    // s4 = gamma^T G2 gamma
    ::ckinv::note_launch(), k_gemv<<<(d + 127) / 128, 128, 0, st>>>(d, G2, gamma, v1, 0);
    ::ckinv::note_launch(), k_dot<<<1, 256, 0, st>>>(d, gamma, 1, v1, 1, s + 4);
    // s5 = <E, R>, s6 = gamma^T R^T beta
    ::ckinv::note_launch(), k_dot<<<gb, 256, 0, st>>>((int64_t)dd, E, 1, f->R, 1, s + 5);
    ::ckinv::note_launch(), k_gemv<<<(d + 127) / 128, 128, 0, st>>>(d, f->R, beta, v1, 1);
    ::ckinv::note_launch(), k_dot<<<1, 256, 0, st>>>(d, gamma, 1, v1, 1, s + 6);
    // T1 = B R;  s7 = <F, B R>;  s8 = gamma^T B R gamma
    if ((e = gemm_small_dev(d, d, f->B, f->R, T1, 0, st)).st) break;
    ::ckinv::note_launch(), k_dot<<<gb, 256, 0, st>>>((int64_t)dd, F, 1, T1, 1, s + 7);
    ::ckinv::note_launch(), k_gemv<<<(d + 127) / 128, 128, 0, st>>>(d, T1, gamma, v2, 0);
    ::ckinv::note_launch(), k_dot<<<1, 256, 0, st>>>(d, gamma, 1, v2, 1, s + 8);
    // s9 = tr(E B) = <E^T, B>;  s10 = alpha^T alpha
    ::ckinv::note_launch(), k_transpose<<<64, 256, 0, st>>>(d, E, T2);
    ::ckinv::note_launch(), k_dot<<<gb, 256, 0, st>>>((int64_t)dd, T2, 1, f->B, 1, s + 9);
    ::ckinv::note_launch(), k_dot_f32<<<gb, 256, 0, st>>>(n, alpha, alpha, s + 10);
    ::ckinv::note_launch(), k_finish_nll<<<1, 1, 0, st>>>(s, f->logdet_parts, n, d, f->tau, out);
    double hout[4];
    if (cudaMemcpyAsync(hout, out, sizeof(hout), cudaMemcpyDeviceToHost, st) != cudaSuccess) {
      e = fail(CKINV_ECUDA, "copy of the likelihood to the host failed");
      break;
    }
    if (cudaStreamSynchronize(st) != cudaSuccess) {
      e = fail(CKINV_ECUDA, cudaGetErrorString(cudaGetLastError()));
      break;
    }
    *nll = hout[0];
    grad[0] = hout[1];
    grad[1] = hout[2];
    grad[2] = hout[3];
  } while (0);
  cudaError_t le = cudaGetLastError();
  if (e.st == CKINV_OK && le != cudaSuccess) e = fail(CKINV_ECUDA, cudaGetErrorString(le));
  cudaStreamSynchronize(st);
  factor_release(f);
  cudaFreeAsync(Y, st);
  cudaFreeAsync(Yd, st);
  cudaFreeAsync(alpha, st);
  cudaFreeAsync(ws, st);
  if (e.st == CKINV_OK) e = read_device_error(ctx, st);
  return e;
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
  delete ctx;
  return CKINV_OK;
}

const char *ckinv_last_error(const ckinv_ctx *ctx) {
  return ctx ? ctx->err.c_str() : g_static_err.c_str();
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

ckinv_status ckinv_sketch(ckinv_ctx *ctx, const ckinv_plan_desc *plan, const ckinv_kernel *kern, const float *points,
                          const float *K, int64_t ldk, float *Y, int64_t ldy, ckinv_stream stream) {
  if (!ctx) return finish(nullptr, fail(CKINV_EINVAL, "null context"));
  DeviceGuard g(ctx->device);
  return finish(ctx, do_sketch(ctx, plan, kern, points, K, ldk, false, Y, ldy, (cudaStream_t)stream));
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

ckinv_status ckinv_solve(ckinv_ctx *ctx, const ckinv_factor *f, const float *A, int64_t lda, int32_t m, float *X,
                         int64_t ldx, ckinv_stream stream) {
  if (!ctx || !f) return finish(ctx, fail(CKINV_EINVAL, "null context or factor"));
  if (!A || !X || lda < f->n || ldx < f->n || m < 1 || m > 256)
    return finish(ctx, fail(CKINV_EINVAL, "need A, X non-null, lda/ldx >= n, 1 <= m <= 256"));
  DeviceGuard g(ctx->device);
  return finish(ctx, lowrank_solve(ctx, f, A, lda, m, X, ldx, f->refine_steps, (cudaStream_t)stream));
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
      if (cudaMallocAsync((void **)&dp, sizeof(float) * n * plan->dim, st) != cudaSuccess ||
          cudaMemcpyAsync(dp, points, sizeof(float) * n * plan->dim, cudaMemcpyHostToDevice, st) != cudaSuccess) {
        e = fail(CKINV_ECUDA, "staging of points failed");
        break;
      }
      P = dp;
    }
    if (ha) {
      if (cudaMallocAsync((void **)&dA, sizeof(float) * n * m, st) != cudaSuccess ||
          cudaMemcpy2DAsync(dA, sizeof(float) * n, A, sizeof(float) * lda, sizeof(float) * n, m,
                            cudaMemcpyHostToDevice, st) != cudaSuccess) {
        e = fail(CKINV_ECUDA, "staging of A failed");
        break;
      }
      Ad = dA;
      ldad = n;
    }
    if (hx) {
      if (cudaMallocAsync((void **)&dX, sizeof(float) * n * m, st) != cudaSuccess) {
        e = fail(CKINV_ENOMEM, "staging of X failed");
        break;
      }
      Xd = dX;
      ldxd = n;
    }
    if (cudaMallocAsync((void **)&Y, sizeof(float) * n * d, st) != cudaSuccess) {
      e = fail(CKINV_ENOMEM, "sketch allocation failed");
      break;
    }
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

ckinv_status ckinv_nll_grad_batched(ckinv_ctx *ctx, int32_t nprob, const ckinv_plan_desc *plans,
                                    const ckinv_kernel *kerns, const float *const *points, const float *const *y,
                                    double *nll, double *grad, ckinv_stream stream) {
  if (!ctx) return finish(nullptr, fail(CKINV_EINVAL, "null context"));
  if (nprob < 1 || !plans || !kerns || !points || !y || !nll || !grad)
    return finish(ctx, fail(CKINV_EINVAL, "null argument or nprob < 1"));
  DeviceGuard g(ctx->device);
  Error e = ok();
  for (int p = 0; p < nprob && e.st == CKINV_OK; ++p)
    e = do_nll_grad(ctx, &plans[p], &kerns[p], points[p], y[p], &nll[p], &grad[3 * p], (cudaStream_t)stream);
  return finish(ctx, e);
}

}  // extern "C"
