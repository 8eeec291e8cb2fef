// A double-FP32 number: the unevaluated sum hi + lo of two floats with |lo| <= ulp(hi) / 2,
// about 48 significand bits with FP32's exponent range.  This part runs FP64 at a small
// fraction of its FP32 rate, so the R-tree combine, the one place the method needs more
// than FP32, computes in this type on the FP32 pipes instead (an operation costs 3 to 20
// FP32 instructions against one FP64 instruction at 1/64 of the rate).
//
// The arithmetic is the standard error-free-transformation scheme: Knuth's TwoSum and
// Dekker's Fast2Sum for additions, the FMA-based exact product for multiplications
// (Dekker; Hida, Li & Bailey, "Algorithms for quad-double precision floating point
// arithmetic", 2001, for the double-double operations built from them).  Addition of two
// dfloats is the accurate variant (both halves summed exactly before renormalising); the
// multiply-add that dot products and updates use sums the leading parts exactly and the
// small terms in FP32, whose rounding is ~2^-24 of terms already ~2^-24 below the result.  The translation unit must
// not be compiled with value-changing floating-point flags (reassociation, fast math), which
// would undo the error-free transformations.
#ifndef CKINV_DFLOAT_CUH
#define CKINV_DFLOAT_CUH

#include <cuda_runtime.h>

namespace ckinv {
// The type and its functions live in their own namespace: argument-dependent lookup finds
// sqrt and __shfl_xor_sync for dfloat, while the same unqualified calls on float and double
// in namespace ckinv still find the global ones.
namespace dd {

struct dfloat {
  float hi, lo;
  dfloat() = default;
  __host__ __device__ constexpr dfloat(float h, float l) : hi(h), lo(l) {}
  __host__ __device__ constexpr dfloat(int v) : hi((float)v), lo(0.f) {}
  __host__ __device__ dfloat(double v) : hi((float)v), lo((float)(v - (double)(float)v)) {}
  __host__ __device__ explicit operator double() const { return (double)hi + (double)lo; }
  __host__ __device__ explicit operator float() const { return hi + lo; }
};

// s + e = a + b exactly (any magnitudes)
__device__ __forceinline__ dfloat two_sum(float a, float b) {
  const float s = a + b;
  const float bb = s - a;
  const float e = (a - (s - bb)) + (b - bb);
  return dfloat(s, e);
}
// s + e = a + b exactly when |a| >= |b| (or a == 0)
__device__ __forceinline__ dfloat fast_two_sum(float a, float b) {
  const float s = a + b;
  return dfloat(s, b - (s - a));
}

__device__ __forceinline__ dfloat operator-(dfloat a) { return dfloat(-a.hi, -a.lo); }

__device__ __forceinline__ dfloat operator+(dfloat a, dfloat b) {
  const dfloat s = two_sum(a.hi, b.hi);
  const dfloat t = two_sum(a.lo, b.lo);
  dfloat u = fast_two_sum(s.hi, s.lo + t.hi);
  return fast_two_sum(u.hi, u.lo + t.lo);
}
__device__ __forceinline__ dfloat operator-(dfloat a, dfloat b) { return a + (-b); }

__device__ __forceinline__ dfloat mul(dfloat a, dfloat b) {
  const float p = a.hi * b.hi;
  float e = fmaf(a.hi, b.hi, -p);              // the exact product's rounding error
  e = fmaf(a.hi, b.lo, fmaf(a.lo, b.hi, e));
  return fast_two_sum(p, e);
}

// c + a b in one pass: the leading parts summed exactly (TwoSum of c.hi and the rounded
// product), the product's exact error and the cross terms and c.lo gathered in FP32, one
// renormalisation; 15 FP32 instructions against 27 for a product followed by an exact sum.
__device__ __forceinline__ dfloat fma_dd(dfloat a, dfloat b, dfloat c) {
  const float p = a.hi * b.hi;
  const float pe = fmaf(a.hi, b.hi, -p);
  const dfloat s = two_sum(c.hi, p);
  float t = s.lo + pe;
  t = fmaf(a.hi, b.lo, t);
  t = fmaf(a.lo, b.hi, t);
  t = t + c.lo;
  return fast_two_sum(s.hi, t);
}

// A product not yet rounded to a dfloat: added to or subtracted from a dfloat it fuses into
// one fma_dd; anywhere else it becomes its rounded value.  This lets the same source serve
// FP32, FP64 and dfloat (acc += x * y).
struct dprod {
  dfloat a, b;
  __device__ __forceinline__ operator dfloat() const { return mul(a, b); }
};
__device__ __forceinline__ dprod operator*(dfloat a, dfloat b) { return dprod{a, b}; }
__device__ __forceinline__ dprod operator*(dprod x, dfloat b) { return dprod{mul(x.a, x.b), b}; }
__device__ __forceinline__ dprod operator*(dfloat a, dprod y) { return dprod{a, mul(y.a, y.b)}; }
__device__ __forceinline__ dprod operator-(dprod x) { return dprod{-x.a, x.b}; }
__device__ __forceinline__ dfloat operator+(dfloat c, dprod x) { return fma_dd(x.a, x.b, c); }
__device__ __forceinline__ dfloat operator+(dprod x, dfloat c) { return fma_dd(x.a, x.b, c); }
__device__ __forceinline__ dfloat operator-(dfloat c, dprod x) { return fma_dd(-x.a, x.b, c); }
__device__ __forceinline__ dfloat operator-(dprod x, dfloat c) { return fma_dd(x.a, x.b, -c); }

// The hardware's approximate reciprocal and square root (relative error about 2^-22): the
// corrections below square the precision, so the IEEE-rounded FP32 sequences (longer, and
// branching for special operands) are not needed.
__device__ __forceinline__ float rcp_approx(float x) {
  float r;
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
  return r;
}
__device__ __forceinline__ float sqrt_approx(float x) {
  float r;
  asm("sqrt.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
  return r;
}

__device__ __forceinline__ dfloat operator/(dfloat a, dfloat b) {
  // long division by an approximate reciprocal: each remainder's quotient is a correction
  // about 2^-22 smaller than the previous one, three terms give the full precision
  const float rb = rcp_approx(b.hi);
  const float q1 = a.hi * rb;
  const dfloat r = a - mul(b, dfloat(q1, 0.f));
  const float q2 = r.hi * rb;
  const dfloat r2 = r - mul(b, dfloat(q2, 0.f));
  const float q3 = r2.hi * rb;
  const dfloat q = fast_two_sum(q1, q2);
  return q + dfloat(q3, 0.f);
}

__device__ __forceinline__ dfloat sqrt(dfloat a) {
  if (!(a.hi > 0.f)) return dfloat(0.f, 0.f);
  // two corrections of the approximate root: s + (a - s^2) / (2 s), twice
  float s = sqrt_approx(a.hi);
  dfloat r = a - mul(dfloat(s, 0.f), dfloat(s, 0.f));
  const float h = 0.5f * rcp_approx(s);
  const dfloat s1 = fast_two_sum(s, r.hi * h);
  r = a - mul(s1, s1);
  return s1 + dfloat(r.hi * h, 0.f);
}

__device__ __forceinline__ dfloat &operator+=(dfloat &a, dfloat b) { return a = a + b; }
__device__ __forceinline__ dfloat &operator-=(dfloat &a, dfloat b) { return a = a - b; }
__device__ __forceinline__ dfloat &operator+=(dfloat &a, dprod x) { return a = fma_dd(x.a, x.b, a); }
__device__ __forceinline__ dfloat &operator-=(dfloat &a, dprod x) { return a = fma_dd(-x.a, x.b, a); }
__device__ __forceinline__ dfloat &operator*=(dfloat &a, dfloat b) { return a = mul(a, b); }

// Comparisons of normalised values: the high halves decide unless equal.
__device__ __forceinline__ bool operator>(dfloat a, dfloat b) { return a.hi > b.hi || (a.hi == b.hi && a.lo > b.lo); }
__device__ __forceinline__ bool operator<(dfloat a, dfloat b) { return b > a; }
__device__ __forceinline__ bool operator>=(dfloat a, dfloat b) { return !(b > a); }
__device__ __forceinline__ bool operator<=(dfloat a, dfloat b) { return !(a > b); }

__device__ __forceinline__ dfloat __shfl_xor_sync(unsigned mask, dfloat v, int lane_mask) {
  return dfloat(::__shfl_xor_sync(mask, v.hi, lane_mask), ::__shfl_xor_sync(mask, v.lo, lane_mask));
}

}  // namespace dd
using dd::dfloat;
}  // namespace ckinv

#endif
