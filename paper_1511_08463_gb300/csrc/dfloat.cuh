// Double-float arithmetic: a value is the unevaluated sum hi + lo of two FP32 numbers with
// |lo| <= ulp(hi)/2, which carries 48 significand bits.  The operations are built on the classical
// error-free transformations: Knuth's TwoSum for the high parts of additions and the FMA form of
// Dekker's TwoProduct for products.  Each result is within a few units of 2^-48 of the exact one,
// relative to the operands' magnitudes, so sums and products of FP64 inputs keep ~14 significant
// digits while running on the FP32 units (FP64 arithmetic throughput is a small fraction of FP32
// on this GPU).  A double is split into hi + lo with integer operations on its bit pattern (no
// FP64 instruction); the conversion back costs one FP64 addition.
//
// The file must be compiled without floating-point reassociation (nvcc's default); products use
// explicit fmaf, and no expression here has a product that contraction could fuse.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>
#include <string.h>

namespace pf {

struct dfloat;
__host__ __device__ inline dfloat df_from_double(double d);

struct dfloat {
  float hi, lo;
  dfloat() = default;
  __host__ __device__ constexpr dfloat(float h, float l) : hi(h), lo(l) {}
  // exact for the small integers of the gradient tables
  __host__ __device__ explicit constexpr dfloat(int i) : hi(float(i)), lo(0.f) {}
  __host__ __device__ explicit dfloat(double d);
  __host__ __device__ explicit operator double() const { return double(hi) + double(lo); }
};

__host__ __device__ inline uint64_t df_bits(double d) {
#ifdef __CUDA_ARCH__
  return (uint64_t)__double_as_longlong(d);
#else
  uint64_t b;
  memcpy(&b, &d, sizeof b);
  return b;
#endif
}
__host__ __device__ inline float df_float_of_bits(uint32_t b) {
#ifdef __CUDA_ARCH__
  return __uint_as_float(b);
#else
  float f;
  memcpy(&f, &b, sizeof f);
  return f;
#endif
}

// hi = d rounded to FP32 (to nearest, ties away from zero), lo = the rest rounded to FP32, both
// from the IEEE-754 fields of d: sign s, biased exponent E, 52-bit fraction F.  hi keeps the top
// 23 fraction bits (+1 in the last place when the 29 bits below are at least half of it); the
// remainder r, |r| <= 2^28, is worth r 2^(E-1075).  Normal doubles with 2^-126 <= |d| < 2^127
// take this path (lo is flushed to zero below 2^-74, an absolute error under 2^-98); zeros give
// (0, 0); anything else (subnormals, huge values, infinities, NaN) goes through FP64 conversions.
__host__ __device__ inline dfloat df_from_double(double d) {
  const uint64_t b = df_bits(d);
  const int E = int((b >> 52) & 0x7FF);
  if (E >= 897 && E <= 1149) {
    const uint32_t sign = uint32_t(b >> 32) & 0x80000000u;
    uint32_t hb = sign | (uint32_t(E - 896) << 23) | uint32_t((b >> 29) & 0x7FFFFFu);
    int32_t r = int32_t(b & 0x1FFFFFFFu);
    if (r >= (1 << 28)) {  // round hi up (a carry into the exponent is the right result)
      hb += 1u;
      r -= 1 << 29;
    }
    float lo = 0.f;
    if (E >= 949 && r != 0) {
      const float scale = df_float_of_bits(uint32_t(E - 948) << 23);  // 2^(E - 1075)
      lo = float(r) * scale;
      if (sign) lo = -lo;
    }
    return dfloat(df_float_of_bits(hb), lo);
  }
  if ((b << 1) == 0) return dfloat(0.f, 0.f);
  const float h = float(d);
  return dfloat(h, float(d - double(h)));
}
__host__ __device__ inline dfloat::dfloat(double d) : dfloat(df_from_double(d)) {}

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
