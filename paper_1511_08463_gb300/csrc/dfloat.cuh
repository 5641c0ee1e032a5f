// Double-float arithmetic: a value is the unevaluated sum hi + lo of two FP32 numbers with
// |lo| <= ulp(hi)/2, which carries 48 significand bits.  The operations are built on the classical
// error-free transformations: Knuth's TwoSum for the high parts of additions and the FMA form of
// Dekker's TwoProduct for products.  Each result is within a few units of 2^-48 of the exact one,
// relative to the operands' magnitudes, so sums and products of FP64 inputs keep ~14 significant
// digits while running on the FP32 units (FP64 arithmetic throughput is a small fraction of FP32
// on this GPU).  Conversions from and to double cost one FP64 subtraction or addition.
//
// The file must be compiled without floating-point reassociation (nvcc's default); products use
// explicit fmaf, and no expression here has a product that contraction could fuse.
#pragma once
#include <cuda_runtime.h>

namespace pf {

struct dfloat {
  float hi, lo;
  dfloat() = default;
  __host__ __device__ constexpr dfloat(float h, float l) : hi(h), lo(l) {}
  // exact for the small integers of the gradient tables
  __host__ __device__ explicit constexpr dfloat(int i) : hi(float(i)), lo(0.f) {}
  __host__ __device__ explicit dfloat(double d) : hi(float(d)), lo(float(d - double(float(d)))) {}
  __host__ __device__ explicit operator double() const { return double(hi) + double(lo); }
};

__device__ __forceinline__ void df_two_sum(float a, float b, float& s, float& e) {
  s = a + b;
  const float bb = s - a;
  e = (a - (s - bb)) + (b - bb);
}
__device__ __forceinline__ void df_quick_two_sum(float a, float b, float& s, float& e) {
  s = a + b;
  e = b - (s - a);
}

// Sum with the high parts added exactly (TwoSum) and the low parts added in FP32: the error is
// within a few units of 2^-48 of |a| + |b| (not of |a + b|), which is the accuracy the operator
// sums need: their tolerance is relative to the magnitudes of the terms.
__device__ __forceinline__ dfloat operator+(dfloat a, dfloat b) {
  float s, e;
  df_two_sum(a.hi, b.hi, s, e);
  e += a.lo + b.lo;
  df_quick_two_sum(s, e, s, e);
  return dfloat(s, e);
}
__device__ __forceinline__ dfloat operator-(dfloat a) { return dfloat(-a.hi, -a.lo); }
__device__ __forceinline__ dfloat operator-(dfloat a, dfloat b) { return a + (-b); }
__device__ __forceinline__ dfloat operator*(dfloat a, dfloat b) {
  const float p = a.hi * b.hi;
  float e = fmaf(a.hi, b.hi, -p);
  e = fmaf(a.hi, b.lo, e);
  e = fmaf(a.lo, b.hi, e);
  float s, r;
  df_quick_two_sum(p, e, s, r);
  return dfloat(s, r);
}
// square root of a non-negative value: the FP32 root of the high part, corrected by one Newton
// step whose residual x - s^2 is formed exactly (TwoProduct)
__device__ __forceinline__ dfloat df_sqrt(dfloat x) {
  if (!(x.hi > 0.f)) return dfloat(0.f, 0.f);
  const float s = sqrtf(x.hi);
  const float p = s * s;
  const float pe = fmaf(s, s, -p);
  const float r = ((x.hi - p) - pe) + x.lo;
  float h, l;
  df_quick_two_sum(s, r / (s + s), h, l);
  return dfloat(h, l);
}
__device__ __forceinline__ bool df_positive(dfloat a) { return a.hi > 0.f || (a.hi == 0.f && a.lo > 0.f); }
__device__ __forceinline__ bool df_negative(dfloat a) { return a.hi < 0.f || (a.hi == 0.f && a.lo < 0.f); }
__device__ __forceinline__ dfloat& operator+=(dfloat& a, dfloat b) { return a = a + b; }
__device__ __forceinline__ dfloat& operator-=(dfloat& a, dfloat b) { return a = a - b; }
__device__ __forceinline__ dfloat& operator*=(dfloat& a, dfloat b) { return a = a * b; }

}  // namespace pf
