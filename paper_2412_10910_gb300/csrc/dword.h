// Double-word arithmetic on the FP32 pipes: a value is the unevaluated sum
// h + l of two floats with |l| <= ulp(h)/2, about 48 significand bits.
//
// Building blocks (own implementation of published error-free transforms):
//   TwoSum (Knuth): s = fl(a+b) and the exact error e with a + b = s + e;
//   FastTwoSum (Dekker), valid when |a| >= |b|;
//   TwoProduct with FMA: p = fl(a*b), e = fma(a, b, -p), a*b = p + e exactly.
// The sum below is the "sloppy" double-word addition and the product the
// double-word times double-word product of Joldes, Muller and Popescu (ACM
// TOMS 44(2), 2017); the sum's absolute error is bounded by a small multiple
// of 2^-48 (|a| + |b|), the same form of bound as an FP64 sum's 2^-53 (|a| + |b|).
// Every operation uses explicit round-to-nearest intrinsics so that the
// compiler neither contracts nor reorders them.
#pragma once

#include <cuda_runtime.h>

namespace nnmg {

struct dw {
  float h, l;
  __host__ __device__ dw() : h(0.f), l(0.f) {}
  __host__ __device__ dw(float v) : h(v), l(0.f) {}
  __host__ __device__ dw(float hi, float lo) : h(hi), l(lo) {}
};

__device__ __forceinline__ dw dw_fast_two_sum(float a, float b) {
  const float s = __fadd_rn(a, b);
  const float e = __fsub_rn(b, __fsub_rn(s, a));
  return dw(s, e);
}

__device__ __forceinline__ dw operator+(dw a, dw b) {
  const float s = __fadd_rn(a.h, b.h);
  const float bb = __fsub_rn(s, a.h);
  float e = __fadd_rn(__fsub_rn(a.h, __fsub_rn(s, bb)), __fsub_rn(b.h, bb));
  e = __fadd_rn(e, __fadd_rn(a.l, b.l));
  return dw_fast_two_sum(s, e);
}

__device__ __forceinline__ dw operator-(dw a) { return dw(-a.h, -a.l); }
__device__ __forceinline__ dw operator-(dw a, dw b) { return a + (-b); }

__device__ __forceinline__ dw operator*(dw a, dw b) {
  const float p = __fmul_rn(a.h, b.h);
  float e = __fmaf_rn(a.h, b.h, -p);
  e = __fmaf_rn(a.h, b.l, e);
  e = __fmaf_rn(a.l, b.h, e);
  return dw_fast_two_sum(p, e);
}

__device__ __forceinline__ dw& operator+=(dw& a, dw b) {
  a = a + b;
  return a;
}

// Conversions at the boundary of a kernel (FP64 vectors in memory).
__device__ __forceinline__ dw dw_from_double(double x) {
  const float h = __double2float_rn(x);
  const float l = __double2float_rn(x - (double)h);
  return dw(h, l);
}
__device__ __forceinline__ double dw_to_double(dw a) { return (double)a.h + (double)a.l; }

// Host: split a double into a double-word.
inline dw dw_split_host(double x) {
  const float h = (float)x;
  return dw(h, (float)(x - (double)h));
}

}  // namespace nnmg
