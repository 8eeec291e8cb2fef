"""Thin Python binding of the ckinv C ABI (include/ckinv.h).

Argument marshalling only: torch tensors provide device memory and the current CUDA
stream, and every step of the method runs in the library's CUDA kernels.  The functions
carry the C names without the prefix (ckinv_sketch -> sketch, ...).  There is no CPU
path: every call raises if the compiled library is missing or no GB300 is present.

Layouts: points (n, dim) float32 row-major; Y, A, X (n, m) float32 column-major, i.e. a
tensor whose stride(0) == 1 (for example torch.empty(m, n).t()).
"""
import ctypes
import os
from dataclasses import dataclass

import torch

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libckinv.so")

OK, EINVAL, ENOMEM, ECUDA, ESINGULAR, ETIMEOUT, EUNSUPPORTED = range(7)
STATUS_NAMES = ["CKINV_OK", "CKINV_EINVAL", "CKINV_ENOMEM", "CKINV_ECUDA", "CKINV_ESINGULAR",
                "CKINV_ETIMEOUT", "CKINV_EUNSUPPORTED"]
SE, MATERN52, DENSE = 0, 1, 2
FP32, BF16, BF16X2, BF16X3, FP32_WHT = 0, 1, 2, 3, 4
WHT, GAUSSIAN, HARTLEY, COSINE = 0, 1, 2, 3       # Omega kinds
PRECISIONS = {"fp32": FP32, "bf16": BF16, "bf16x2": BF16X2, "bf16x3": BF16X3, "fp32_wht": FP32_WHT}


class CKInvError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__("%s: %s" % (STATUS_NAMES[status] if 0 <= status < 7 else status, msg))
        self.status = status


class PlanDesc(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int64), ("dim", ctypes.c_int32), ("d", ctypes.c_int32),
                ("block_rows", ctypes.c_int32), ("prec", ctypes.c_int32), ("seed", ctypes.c_uint64),
                ("refine_steps", ctypes.c_int32), ("tree_fp64_levels", ctypes.c_int32),
                ("leaf_fp64", ctypes.c_int32), ("omega_kind", ctypes.c_int32)]


class KernelDesc(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int32), ("reserved", ctypes.c_int32), ("lengthscale", ctypes.c_double),
                ("variance", ctypes.c_double), ("nugget", ctypes.c_double)]


_VP = ctypes.c_void_p
_SIGS = {
    "ckinv_version": (ctypes.c_char_p, []),
    "ckinv_kernel_launches": (ctypes.c_ulonglong, []),
    "ckinv_create": (ctypes.c_int, [ctypes.POINTER(_VP), ctypes.c_int]),
    "ckinv_destroy": (ctypes.c_int, [_VP]),
    "ckinv_last_error": (ctypes.c_char_p, [_VP]),
    "ckinv_check": (ctypes.c_int, [_VP, _VP]),
    "ckinv_set_wait_limit": (ctypes.c_int, [_VP, ctypes.c_uint64]),
    "ckinv_omega": (ctypes.c_int, [_VP, ctypes.c_int64, ctypes.c_int32, ctypes.c_uint64, _VP, _VP, _VP]),
    "ckinv_omega_matrix": (ctypes.c_int, [_VP, ctypes.c_int64, ctypes.c_int32, ctypes.c_uint64, ctypes.c_int32, _VP,
                                          ctypes.c_int64, _VP]),
    "ckinv_omega_noalloc": (ctypes.c_int, [ctypes.c_int64, ctypes.c_int32, ctypes.c_uint64, _VP, _VP, _VP]),
    "ckinv_sketch": (ctypes.c_int, [_VP, ctypes.POINTER(PlanDesc), ctypes.POINTER(KernelDesc), _VP, _VP,
                                    ctypes.c_int64, _VP, ctypes.c_int64, _VP]),
    "ckinv_kernel_matrix": (ctypes.c_int, [_VP, ctypes.POINTER(PlanDesc), ctypes.POINTER(KernelDesc), _VP, _VP,
                                           ctypes.c_int64, _VP]),
    "ckinv_sketch_dlogl": (ctypes.c_int, [_VP, ctypes.POINTER(PlanDesc), ctypes.POINTER(KernelDesc), _VP, _VP,
                                          ctypes.c_int64, _VP]),
    "ckinv_tsqr": (ctypes.c_int, [_VP, ctypes.POINTER(PlanDesc), ctypes.POINTER(KernelDesc), _VP, ctypes.c_int64,
                                  ctypes.POINTER(_VP), _VP]),
    "ckinv_factor_free": (ctypes.c_int, [_VP]),
    "ckinv_factor_r": (ctypes.c_int, [_VP, _VP, _VP]),
    "ckinv_factor_q": (ctypes.c_int, [_VP, _VP, ctypes.c_int64, _VP]),
    "ckinv_factor_core": (ctypes.c_int, [_VP, _VP, _VP, ctypes.POINTER(ctypes.c_double), _VP]),
    "ckinv_sketch_rows": (ctypes.c_int, [_VP, ctypes.POINTER(PlanDesc), ctypes.POINTER(KernelDesc), _VP, _VP,
                                         ctypes.c_int64, ctypes.c_int64, ctypes.c_int64, _VP, ctypes.c_int64, _VP]),
    "ckinv_tsqr_shard": (ctypes.c_int, [_VP, ctypes.POINTER(PlanDesc), ctypes.POINTER(KernelDesc), _VP, ctypes.c_int64,
                                        ctypes.c_int64, ctypes.c_int64, ctypes.POINTER(_VP), _VP, _VP]),
    "ckinv_shard_combine": (ctypes.c_int, [_VP, _VP, _VP, ctypes.c_int32, ctypes.c_int32, _VP, _VP]),
    "ckinv_shard_core": (ctypes.c_int, [_VP, _VP, _VP, _VP]),
    "ckinv_shard_solve_begin": (ctypes.c_int, [_VP, _VP, _VP, ctypes.c_int64, ctypes.c_int32, _VP, _VP]),
    "ckinv_shard_solve_end": (ctypes.c_int, [_VP, _VP, _VP, _VP, ctypes.c_int64, ctypes.c_int32, _VP, ctypes.c_int64,
                                             _VP]),
    "ckinv_factor_project": (ctypes.c_int, [_VP, _VP, ctypes.POINTER(PlanDesc), ctypes.POINTER(KernelDesc), _VP, _VP,
                                            ctypes.POINTER(ctypes.c_double), _VP]),
    "ckinv_predict_mean": (ctypes.c_int, [_VP, ctypes.POINTER(PlanDesc), ctypes.POINTER(KernelDesc), _VP, _VP, _VP,
                                          ctypes.c_int64, _VP, _VP]),
    "ckinv_solve": (ctypes.c_int, [_VP, _VP, _VP, ctypes.c_int64, ctypes.c_int32, _VP, ctypes.c_int64, _VP]),
    "ckinv_kinv_a": (ctypes.c_int, [_VP, ctypes.POINTER(PlanDesc), ctypes.POINTER(KernelDesc), _VP, _VP,
                                    ctypes.c_int64, ctypes.c_int32, _VP, ctypes.c_int64, _VP]),
    "ckinv_nll_grad": (ctypes.c_int, [_VP, ctypes.POINTER(PlanDesc), ctypes.POINTER(KernelDesc), _VP, _VP,
                                      ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_double), _VP]),
    "ckinv_autotune": (ctypes.c_int, [_VP, ctypes.POINTER(PlanDesc), ctypes.POINTER(ctypes.c_int32), _VP]),
    "ckinv_nll_grad_batched": (ctypes.c_int, [_VP, ctypes.c_int32, ctypes.POINTER(PlanDesc),
                                              ctypes.POINTER(KernelDesc), ctypes.POINTER(_VP), ctypes.POINTER(_VP),
                                              ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_double), _VP]),
}

_lib = None


def load(path=LIB_PATH):
    """Load libckinv.so (raises if it has not been built)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise RuntimeError("libckinv.so is not built (run __graft_entry__.build()); there is no CPU fallback")
    lib = ctypes.CDLL(path)
    for name, (res, args) in _SIGS.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


def version():
    return load().ckinv_version().decode()


def kernel_launches():
    return int(load().ckinv_kernel_launches())


def _ptr(t):
    return None if t is None else ctypes.c_void_p(t.data_ptr())


def _stream(stream=None):
    s = torch.cuda.current_stream() if stream is None else stream
    return ctypes.c_void_p(s.cuda_stream)


def _colmajor_ld(t, rows):
    if t.dtype != torch.float32 or not t.is_cuda:
        raise ValueError("expected a CUDA float32 tensor")
    if t.dim() == 1:
        return max(rows, 1)
    if t.stride(0) != 1 or t.shape[0] != rows:
        raise ValueError("expected a column-major (stride(0) == 1) tensor with %d rows" % rows)
    return t.stride(1) if t.shape[1] > 1 else rows


def colmajor(rows, cols, device="cuda", dtype=torch.float32):
    """An uninitialised column-major (rows, cols) tensor."""
    return torch.empty((cols, rows), device=device, dtype=dtype).t()


@dataclass
class Plan:
    n: int
    d: int
    dim: int = 2
    block_rows: int = 0
    prec: int = FP32
    seed: int = 0
    refine_steps: int = 1
    tree_fp64_levels: int = -1          # every level of the R tree combined in FP64
    leaf_fp64: int = 0
    omega_kind: int = WHT

    def desc(self):
        return PlanDesc(self.n, self.dim, self.d, self.block_rows, self.prec, self.seed, self.refine_steps,
                        self.tree_fp64_levels, self.leaf_fp64, self.omega_kind)


@dataclass
class Kernel:
    kind: int = SE
    lengthscale: float = 1.0
    variance: float = 1.0
    nugget: float = 1e-6

    def desc(self):
        return KernelDesc(self.kind, 0, self.lengthscale, self.variance, self.nugget)


class Context:
    """Owns a ckinv_ctx on one CUDA device."""

    def __init__(self, device=0):
        lib = load()
        h = ctypes.c_void_p()
        st = lib.ckinv_create(ctypes.byref(h), int(device))
        if st != OK:
            raise CKInvError(st, lib.ckinv_last_error(None).decode())
        self.handle = h
        self.device = device

    def _raise(self, st):
        if st != OK:
            raise CKInvError(st, load().ckinv_last_error(self.handle).decode())

    def close(self):
        if getattr(self, "handle", None):
            load().ckinv_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def check(ctx, stream=None):
    ctx._raise(load().ckinv_check(ctx.handle, _stream(stream)))


def set_wait_limit(ctx, nanoseconds):
    """Limit of the device-side waits of the tensor-core kernels launched afterwards from
    this context (0 restores the default of one second)."""
    ctx._raise(load().ckinv_set_wait_limit(ctx.handle, int(nanoseconds)))


def omega(ctx, n, d, seed, stream=None):
    """(sign_bits uint32[ceil(n/32)], cols int32[d]) on the device."""
    bits = torch.empty(((n + 31) // 32,), dtype=torch.int32, device="cuda")
    cols = torch.empty((d,), dtype=torch.int32, device="cuda")
    ctx._raise(load().ckinv_omega(ctx.handle, n, d, seed, _ptr(bits), _ptr(cols), _stream(stream)))
    return bits, cols


def omega_matrix(ctx, n, d, seed, kind=WHT, stream=None):
    """Omega as a dense column-major n x d float32 tensor."""
    Om = colmajor(n, d)
    ctx._raise(load().ckinv_omega_matrix(ctx.handle, n, d, seed, kind, _ptr(Om), n, _stream(stream)))
    return Om


def omega_noalloc(n, d, seed, sign_bits=None, cols=None, stream=None):
    """The Omega draw without any library allocation (outputs are the caller's tensors)."""
    if sign_bits is None:
        sign_bits = torch.empty(((n + 31) // 32,), dtype=torch.int32, device="cuda")
    if cols is None:
        cols = torch.empty((d,), dtype=torch.int32, device="cuda")
    st = load().ckinv_omega_noalloc(n, d, seed, _ptr(sign_bits), _ptr(cols), _stream(stream))
    if st != OK:
        raise CKInvError(st, load().ckinv_last_error(None).decode())
    return sign_bits, cols


def sketch(ctx, plan, kern, points=None, K=None, Y=None, stream=None):
    """Y = K0 Omega (column-major n x d float32)."""
    if Y is None:
        Y = colmajor(plan.n, plan.d)
    ldy = _colmajor_ld(Y, plan.n)
    ldk = 0
    if K is not None:
        ldk = _colmajor_ld(K, plan.n)
    if points is not None and (points.dtype != torch.float32 or not points.is_contiguous()):
        raise ValueError("points must be a contiguous float32 (n, dim) tensor")
    pd, kd = plan.desc(), kern.desc()
    ctx._raise(load().ckinv_sketch(ctx.handle, ctypes.byref(pd), ctypes.byref(kd), _ptr(points), _ptr(K), ldk,
                                   _ptr(Y), ldy, _stream(stream)))
    return Y


def kernel_matrix(ctx, plan, kern, points, K=None, stream=None):
    """K0 (n x n float32, column-major) materialised on the device."""
    if K is None:
        K = colmajor(plan.n, plan.n)
    ldk = _colmajor_ld(K, plan.n)
    pd, kd = plan.desc(), kern.desc()
    ctx._raise(load().ckinv_kernel_matrix(ctx.handle, ctypes.byref(pd), ctypes.byref(kd), _ptr(points), _ptr(K),
                                          ldk, _stream(stream)))
    return K


def sketch_dlogl(ctx, plan, kern, points, Y=None, stream=None):
    if Y is None:
        Y = colmajor(plan.n, plan.d)
    ldy = _colmajor_ld(Y, plan.n)
    pd, kd = plan.desc(), kern.desc()
    ctx._raise(load().ckinv_sketch_dlogl(ctx.handle, ctypes.byref(pd), ctypes.byref(kd), _ptr(points), _ptr(Y),
                                         ldy, _stream(stream)))
    return Y


class Factor:
    """A ckinv_factor (Q_hat, R, B, C' and their LUs); frees itself."""

    def __init__(self, ctx, handle, plan):
        self.ctx, self.handle, self.plan = ctx, handle, plan

    def r(self, stream=None):
        R = torch.empty((self.plan.d, self.plan.d), dtype=torch.float64, device="cuda")
        self.ctx._raise(load().ckinv_factor_r(self.handle, _ptr(R), _stream(stream)))
        return R.t()            # column-major storage -> logical R

    def q(self, stream=None):
        Q = colmajor(self.plan.n, self.plan.d)
        self.ctx._raise(load().ckinv_factor_q(self.handle, _ptr(Q), Q.stride(1), _stream(stream)))
        return Q

    def core(self, stream=None):
        d = self.plan.d
        B = torch.empty((d, d), dtype=torch.float64, device="cuda")
        C = torch.empty((d, d), dtype=torch.float64, device="cuda")
        ld = ctypes.c_double()
        self.ctx._raise(load().ckinv_factor_core(self.handle, _ptr(B), _ptr(C), ctypes.byref(ld), _stream(stream)))
        return B.t(), C.t(), ld.value

    def free(self):
        if self.handle:
            load().ckinv_factor_free(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.free()
        except Exception:
            pass


# ---------------------------------------------------------------- row shards
def sketch_rows(ctx, plan, kern, row0, m, points=None, K=None, Y=None, stream=None):
    """Rows row0 .. row0 + m - 1 of Y = K0 Omega (column-major m x d float32)."""
    if Y is None:
        Y = colmajor(m, plan.d)
    ldy = _colmajor_ld(Y, m)
    ldk = _colmajor_ld(K, plan.n) if K is not None else 0
    pd, kd = plan.desc(), kern.desc()
    ctx._raise(load().ckinv_sketch_rows(ctx.handle, ctypes.byref(pd), ctypes.byref(kd), _ptr(points), _ptr(K), ldk,
                                        row0, m, _ptr(Y), ldy, _stream(stream)))
    return Y


def tsqr_shard(ctx, plan, kern, Y, row0, stream=None):
    """Local TSQR of a row shard: (shard Factor, its d x d R as a float64 tensor, column-major
    storage: R_storage[j, i] = R[i, j])."""
    m = Y.shape[0]
    ldy = _colmajor_ld(Y, m)
    R = torch.empty((plan.d, plan.d), dtype=torch.float64, device="cuda")
    h = ctypes.c_void_p()
    pd, kd = plan.desc(), kern.desc()
    ctx._raise(load().ckinv_tsqr_shard(ctx.handle, ctypes.byref(pd), ctypes.byref(kd), _ptr(Y), ldy, row0, m,
                                       ctypes.byref(h), _ptr(R), _stream(stream)))
    f = Factor(ctx, h, Plan(n=m, d=plan.d, dim=plan.dim))
    return f, R


def shard_combine(ctx, factor, R_all, G, g, stream=None):
    """R_all: (G, d, d) float64 device tensor of the shards' R storages.  Returns this shard's
    B_partial storage (d, d) float64."""
    d = factor.plan.d
    Bp = torch.empty((d, d), dtype=torch.float64, device="cuda")
    ctx._raise(load().ckinv_shard_combine(ctx.handle, factor.handle, _ptr(R_all.contiguous()), G, g, _ptr(Bp),
                                          _stream(stream)))
    return Bp


def shard_core(ctx, factor, B, stream=None):
    ctx._raise(load().ckinv_shard_core(ctx.handle, factor.handle, _ptr(B.contiguous()), _stream(stream)))


def shard_solve_begin(ctx, factor, A, stream=None):
    """Z_partial = Q_hat_shard^T A_shard as a (m, d) float64 storage (column-major d x m)."""
    rows = factor.plan.n
    m = 1 if A.dim() == 1 else A.shape[1]
    lda = _colmajor_ld(A, rows)
    Z = torch.empty((m, factor.plan.d), dtype=torch.float64, device="cuda")
    ctx._raise(load().ckinv_shard_solve_begin(ctx.handle, factor.handle, _ptr(A), lda, m, _ptr(Z), _stream(stream)))
    return Z


def shard_solve_end(ctx, factor, Z, A, X=None, stream=None):
    rows = factor.plan.n
    m = 1 if A.dim() == 1 else A.shape[1]
    lda = _colmajor_ld(A, rows)
    if X is None:
        X = colmajor(rows, m) if A.dim() == 2 else torch.empty_like(A)
    ldx = _colmajor_ld(X, rows)
    ctx._raise(load().ckinv_shard_solve_end(ctx.handle, factor.handle, _ptr(Z.contiguous()), _ptr(A), lda, m, _ptr(X),
                                            ldx, _stream(stream)))
    return X


def project(ctx, factor, plan, kern, points, stream=None, colspace=True):
    """Second pass: S = Q_hat^T K0 Q_hat; the factor's solves use the two-pass core afterwards.
    Returns (S as a (d, d) float64 tensor, column-space error or None)."""
    d = plan.d
    S = torch.empty((d, d), dtype=torch.float64, device="cuda")
    err = ctypes.c_double()
    pd, kd = plan.desc(), kern.desc()
    ctx._raise(load().ckinv_factor_project(ctx.handle, factor.handle, ctypes.byref(pd), ctypes.byref(kd),
                                           _ptr(points), _ptr(S), ctypes.byref(err) if colspace else None,
                                           _stream(stream)))
    return S.t(), (err.value if colspace else None)


def predict_mean(ctx, plan, kern, points, alpha, new_points, stream=None):
    """mu* = K0(X*, X) alpha at the rows of new_points (float64 tensor)."""
    n_new = new_points.shape[0]
    mean = torch.empty((n_new,), dtype=torch.float64, device="cuda")
    pd, kd = plan.desc(), kern.desc()
    ctx._raise(load().ckinv_predict_mean(ctx.handle, ctypes.byref(pd), ctypes.byref(kd), _ptr(points), _ptr(alpha),
                                         _ptr(new_points), n_new, _ptr(mean), _stream(stream)))
    return mean


def tsqr(ctx, plan, kern, Y, stream=None):
    """Factor Y in place; returns a Factor."""
    ldy = _colmajor_ld(Y, plan.n)
    h = ctypes.c_void_p()
    pd, kd = plan.desc(), kern.desc()
    ctx._raise(load().ckinv_tsqr(ctx.handle, ctypes.byref(pd), ctypes.byref(kd), _ptr(Y), ldy, ctypes.byref(h),
                                 _stream(stream)))
    return Factor(ctx, h, plan)


def solve(ctx, factor, A, X=None, stream=None):
    n = factor.plan.n
    m = 1 if A.dim() == 1 else A.shape[1]
    lda = _colmajor_ld(A, n)
    if X is None:
        X = colmajor(n, m) if A.dim() == 2 else torch.empty_like(A)
    ldx = _colmajor_ld(X, n)
    ctx._raise(load().ckinv_solve(ctx.handle, factor.handle, _ptr(A), lda, m, _ptr(X), ldx, _stream(stream)))
    return X


def kinv_a(ctx, plan, kern, points, A, X=None, stream=None):
    """The whole path in one call; points/A/X may be CPU (pinned or pageable) or CUDA tensors."""
    n = plan.n
    m = 1 if A.dim() == 1 else A.shape[1]
    if A.dim() == 2 and A.stride(0) != 1:
        raise ValueError("A must be column-major")
    # a single column may carry any stride along its (size-1) second dimension
    lda = n if (A.dim() == 1 or m == 1) else A.stride(1)
    if X is None:
        X = torch.empty((m, n), dtype=torch.float32, device=A.device).t()
    if X.dim() == 2 and X.stride(0) != 1:
        raise ValueError("X must be column-major")
    ldx = n if (X.dim() == 1 or m == 1) else X.stride(1)
    pd, kd = plan.desc(), kern.desc()
    ctx._raise(load().ckinv_kinv_a(ctx.handle, ctypes.byref(pd), ctypes.byref(kd), _ptr(points), _ptr(A), lda, m,
                                   _ptr(X), ldx, _stream(stream)))
    return X


def nll_grad(ctx, plan, kern, points, y, stream=None):
    """(nll, [d/dlog l, d/dlog var, d/dlog nugget]) as Python floats."""
    nll = ctypes.c_double()
    g = (ctypes.c_double * 3)()
    pd, kd = plan.desc(), kern.desc()
    ctx._raise(load().ckinv_nll_grad(ctx.handle, ctypes.byref(pd), ctypes.byref(kd), _ptr(points), _ptr(y),
                                     ctypes.byref(nll), g, _stream(stream)))
    return nll.value, [g[0], g[1], g[2]]


def autotune(ctx, plan, stream=None):
    """Leaf height (block_rows) the library's autotuner picks for this plan's shape class;
    later plans with block_rows = 0 in the same class use it."""
    b = ctypes.c_int32(0)
    pd = plan.desc()
    ctx._raise(load().ckinv_autotune(ctx.handle, ctypes.byref(pd), ctypes.byref(b), _stream(stream)))
    return b.value


def nll_grad_batched(ctx, plans, kerns, points, ys, stream=None):
    """NLL and gradient of many independent problems, run as one CUDA graph."""
    P = len(plans)
    pds = (PlanDesc * P)(*[p.desc() for p in plans])
    kds = (KernelDesc * P)(*[k.desc() for k in kerns])
    pp = (ctypes.c_void_p * P)(*[t.data_ptr() for t in points])
    yy = (ctypes.c_void_p * P)(*[t.data_ptr() for t in ys])
    nll = (ctypes.c_double * P)()
    g = (ctypes.c_double * (3 * P))()
    ctx._raise(load().ckinv_nll_grad_batched(ctx.handle, P, pds, kds, pp, yy, nll, g, _stream(stream)))
    return list(nll), [list(g[3 * i:3 * i + 3]) for i in range(P)]


class CKInvNLL(torch.autograd.Function):
    """Gaussian NLL under K_tilde as a differentiable function of
    (log lengthscale, log variance, log nugget); the gradient comes from the library's
    hand-written adjoint, computed in the same call as the forward value."""

    @staticmethod
    def forward(ctx_, log_params, points, y, plan, kind, ckctx):
        lp = log_params.detach().double().cpu().tolist()
        kern = Kernel(kind, float(torch.tensor(lp[0]).exp()), float(torch.tensor(lp[1]).exp()),
                      float(torch.tensor(lp[2]).exp()))
        val, g = nll_grad(ckctx, plan, kern, points, y)
        ctx_.save_for_backward(torch.tensor(g, dtype=torch.float64))
        return torch.tensor(val, dtype=torch.float64)

    @staticmethod
    def backward(ctx_, gout):
        (g,) = ctx_.saved_tensors
        return (gout * g).to(torch.float64), None, None, None, None, None
