// Float-float arithmetic: a value is the unevaluated sum hi + lo of two FP32 numbers with
// |lo| <= ulp(hi) / 2, about 44 significant bits (Dekker, Numer. Math. 18, 1971).  Sums use
// Knuth's error-free two-sum, products the FMA two-product (the rounding error of a*b is
// fma(a, b, -round(a*b)) exactly).  GB300 runs FP64 at about 1/64 of the FP32 rate, so the
// grid transforms that need more than FP32 (the potential and the output density) run in
// float-float on the FP32 pipes; the operands stay FP64 in memory.
#pragma once

#include <cmath>

#include "sgo_internal.cuh"

namespace sgo {

// Rounded sum and product that the compiler never fuses into an FMA (a fused a*b + c would
// break the error-free transforms below).
__host__ __device__ __forceinline__ float add_rn(float a, float b) {
#ifdef __CUDA_ARCH__
  return __fadd_rn(a, b);
#else
  return a + b;
#endif
}
__host__ __device__ __forceinline__ float sub_rn(float a, float b) {
#ifdef __CUDA_ARCH__
  return __fsub_rn(a, b);
#else
  return a - b;
#endif
}
__host__ __device__ __forceinline__ float mul_rn(float a, float b) {
#ifdef __CUDA_ARCH__
  return __fmul_rn(a, b);
#else
  return a * b;
#endif
}

struct ff {
  float hi, lo;
  ff() = default;
  __host__ __device__ constexpr ff(float h, float l) : hi(h), lo(l) {}
  // nearest float-float to v (a compile-time constant folds to two float immediates)
  __host__ __device__ constexpr explicit ff(double v) : hi((float)v), lo((float)(v - (double)(float)v)) {}
};

// s + e = a + b exactly (no assumption on the magnitudes)
__host__ __device__ __forceinline__ ff two_sum(float a, float b) {
  const float s = add_rn(a, b);
  const float bb = sub_rn(s, a);
  const float e = add_rn(sub_rn(a, sub_rn(s, bb)), sub_rn(b, bb));
  return ff(s, e);
}
// s + e = a + b exactly, for |a| >= |b| or a = 0
__host__ __device__ __forceinline__ ff fast_two_sum(float a, float b) {
  const float s = add_rn(a, b);
  return ff(s, sub_rn(b, sub_rn(s, a)));
}

__host__ __device__ __forceinline__ ff operator+(ff a, ff b) {
  const ff s = two_sum(a.hi, b.hi);
  return fast_two_sum(s.hi, add_rn(s.lo, add_rn(a.lo, b.lo)));
}
__host__ __device__ __forceinline__ ff operator-(ff a) { return ff(-a.hi, -a.lo); }
__host__ __device__ __forceinline__ ff operator-(ff a, ff b) { return a + (-b); }
__host__ __device__ __forceinline__ ff operator*(ff a, ff b) {
  const float p = mul_rn(a.hi, b.hi);
  const float e = fmaf(a.hi, b.hi, -p);  // rounding error of the product, exact
  return fast_two_sum(p, fmaf(a.hi, b.lo, fmaf(a.lo, b.hi, e)));
}
__host__ __device__ __forceinline__ bool operator<(ff a, ff b) { return a.hi < b.hi || (a.hi == b.hi && a.lo < b.lo); }

__device__ __forceinline__ ff ff_from(double v) {
  const float h = __double2float_rn(v);
  return ff(h, __double2float_rn(v - (double)h));
}
__device__ __forceinline__ double ff_to(ff a) { return (double)a.hi + (double)a.lo; }

// multiply by i s for s = +-1: a sign and a swap, no arithmetic
template <>
__host__ __device__ __forceinline__ cplx<ff> mul_is(cplx<ff> a, ff s) {
  return s.hi < 0.f ? mk(a.y, -a.x) : mk(-a.y, a.x);
}

}  // namespace sgo
