// Double-float arithmetic: a value held as the unevaluated sum hi + lo of two
// FP32 numbers with |lo| <= ulp(hi) / 2, about 48 significant bits.  Sums use
// Knuth's two-sum and products Dekker's two-product with a fused multiply-add
// (the error-free transformations of T. J. Dekker, "A floating-point
// technique for extending the available precision", 1971).  On this GPU FP32
// runs at 64 times the FP64 rate, so an operator evaluation in double-float
// is several times faster than in FP64 while its rounding (about 2^-47
// relative) stays far below the Newton tolerance of the residuals it serves.
#pragma once
#include <cuda_runtime.h>

namespace dnnmg {

struct dfloat {
  float hi, lo;
  __host__ __device__ constexpr dfloat() : hi(0.f), lo(0.f) {}
  __host__ __device__ constexpr dfloat(double d)
      : hi((float)d), lo((float)(d - (double)(float)d)) {}
  __host__ __device__ constexpr dfloat(float h, float l) : hi(h), lo(l) {}
  __host__ __device__ explicit operator double() const { return (double)hi + (double)lo; }
};

// s + e == a + b exactly (no precondition on |a|, |b|)
__device__ __forceinline__ void df_two_sum(float a, float b, float& s, float& e) {
  s = __fadd_rn(a, b);
  const float bb = __fsub_rn(s, a);
  e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
}
// s + e == a + b exactly when |a| >= |b|
__device__ __forceinline__ void df_fast_two_sum(float a, float b, float& s, float& e) {
  s = __fadd_rn(a, b);
  e = __fsub_rn(b, __fsub_rn(s, a));
}

__device__ __forceinline__ dfloat operator+(dfloat x, dfloat y) {
  float s, e;
  df_two_sum(x.hi, y.hi, s, e);
  e = __fadd_rn(e, __fadd_rn(x.lo, y.lo));
  dfloat r;
  df_fast_two_sum(s, e, r.hi, r.lo);
  return r;
}
__device__ __forceinline__ dfloat operator-(dfloat x) { return dfloat(-x.hi, -x.lo); }
__device__ __forceinline__ dfloat operator-(dfloat x, dfloat y) { return x + (-y); }
__device__ __forceinline__ dfloat operator*(dfloat x, dfloat y) {
  const float p = __fmul_rn(x.hi, y.hi);
  float e = __fmaf_rn(x.hi, y.hi, -p);  // exact error of the leading product
  e = __fmaf_rn(x.hi, y.lo, e);
  e = __fmaf_rn(x.lo, y.hi, e);
  dfloat r;
  df_fast_two_sum(p, e, r.hi, r.lo);
  return r;
}
__device__ __forceinline__ dfloat& operator+=(dfloat& x, dfloat y) { return x = x + y; }
__device__ __forceinline__ dfloat& operator-=(dfloat& x, dfloat y) { return x = x - y; }
__device__ __forceinline__ dfloat& operator*=(dfloat& x, dfloat y) { return x = x * y; }

}  // namespace dnnmg
