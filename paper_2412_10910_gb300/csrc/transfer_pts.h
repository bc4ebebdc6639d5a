// Device helpers of the point-evaluation transfer kernels (k_prolong.cu,
// k_restrict.cu): 1D Lagrange bases at a reference coordinate, and channel
// vectors of CH values moved and combined as packed pairs.
//
// A transfer vector row holds nch = components x right-hand sides channels;
// a thread works on a group of CH consecutive channels of one row.  In FP32
// with even CH a group is CH/2 float pairs and every multiply-add is one
// packed Blackwell FP32 instruction (__ffma2_rn, rounded as two scalar FMAs);
// rows are read and written with 16-byte (CH >= 4) or 8-byte vector accesses.
// In FP64 a group is CH doubles, read and written as 16-byte pairs for even CH.
#pragma once

#include <type_traits>

#include "nnmg_internal.h"

namespace nnmg {
namespace pts {

template <int N, int D>
struct ipow {
  static constexpr int value = N * ipow<N, D - 1>::value;
};
template <int N>
struct ipow<N, 0> {
  static constexpr int value = 1;
};

// L[l] = prod_{m != l} (xi - t_m) / prod_{m != l} (t_l - t_m), t the
// Gauss-Lobatto nodes of [0,1] (the coarse cell's 1D Lagrange basis at xi).
template <int N, typename T>
__device__ __forceinline__ void lagrange(const Basis1D<T>& B, T xi, T* L) {
  T dl[N];
#pragma unroll
  for (int m = 0; m < N; ++m) dl[m] = xi - B.gl[m];
#pragma unroll
  for (int l = 0; l < N; ++l) {
    T v = B.gl_scale[l];
#pragma unroll
    for (int m = 0; m < N; ++m)
      if (m != l) v *= dl[m];
    L[l] = v;
  }
}

// Packed element type of a channel group and the number of them.
template <typename T, int CH>
struct Pack {
  static constexpr bool pair = std::is_same<T, float>::value && CH % 2 == 0;
  using type = std::conditional_t<pair, float2, T>;
  static constexpr int n = pair ? CH / 2 : CH;
};

__device__ __forceinline__ float2 pbcast(float c, float2) { return make_float2(c, c); }
__device__ __forceinline__ float pbcast(float c, float) { return c; }
__device__ __forceinline__ double pbcast(double c, double) { return c; }
__device__ __forceinline__ float2 pzero(float2) { return make_float2(0.f, 0.f); }
__device__ __forceinline__ float pzero(float) { return 0.f; }
__device__ __forceinline__ double pzero(double) { return 0.0; }
__device__ __forceinline__ float2 pfma(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }
__device__ __forceinline__ float pfma(float a, float b, float c) { return fmaf(a, b, c); }
__device__ __forceinline__ double pfma(double a, double b, double c) { return fma(a, b, c); }
__device__ __forceinline__ float2 pmul(float2 a, float2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ float pmul(float a, float b) { return a * b; }
__device__ __forceinline__ double pmul(double a, double b) { return a * b; }
__device__ __forceinline__ float2 psub(float2 a, float2 b) {
  return make_float2(a.x - b.x, a.y - b.y);
}
__device__ __forceinline__ float psub(float a, float b) { return a - b; }
__device__ __forceinline__ double psub(double a, double b) { return a - b; }
__device__ __forceinline__ float2 padd(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ float padd(float a, float b) { return a + b; }
__device__ __forceinline__ double padd(double a, double b) { return a + b; }
__device__ __forceinline__ float2 pshfl_down(float2 v, int d) {
  return make_float2(__shfl_down_sync(0xffffffffu, v.x, d), __shfl_down_sync(0xffffffffu, v.y, d));
}
__device__ __forceinline__ float pshfl_down(float v, int d) { return __shfl_down_sync(0xffffffffu, v, d); }
__device__ __forceinline__ double pshfl_down(double v, int d) { return __shfl_down_sync(0xffffffffu, v, d); }

// Load / store one channel group of CH values at p (global or shared memory).
// p must be aligned to min(16, CH * sizeof(T)) bytes (the launchers check).
template <typename T, int CH>
__device__ __forceinline__ void load_group(const T* p, typename Pack<T, CH>::type* v) {
  if constexpr (std::is_same<T, float>::value && CH % 4 == 0) {
#pragma unroll
    for (int q = 0; q < CH / 4; ++q) {
      const float4 a = reinterpret_cast<const float4*>(p)[q];
      v[2 * q] = make_float2(a.x, a.y);
      v[2 * q + 1] = make_float2(a.z, a.w);
    }
  } else if constexpr (std::is_same<T, float>::value && CH == 2) {
    v[0] = *reinterpret_cast<const float2*>(p);
  } else if constexpr (std::is_same<T, double>::value && CH % 2 == 0) {
#pragma unroll
    for (int q = 0; q < CH / 2; ++q) {
      const double2 a = reinterpret_cast<const double2*>(p)[q];
      v[2 * q] = a.x;
      v[2 * q + 1] = a.y;
    }
  } else {
#pragma unroll
    for (int q = 0; q < CH; ++q) v[q] = p[q];
  }
}

template <typename T, int CH>
__device__ __forceinline__ void store_group(T* p, const typename Pack<T, CH>::type* v) {
  if constexpr (std::is_same<T, float>::value && CH % 4 == 0) {
#pragma unroll
    for (int q = 0; q < CH / 4; ++q)
      reinterpret_cast<float4*>(p)[q] = make_float4(v[2 * q].x, v[2 * q].y, v[2 * q + 1].x,
                                                    v[2 * q + 1].y);
  } else if constexpr (std::is_same<T, float>::value && CH == 2) {
    *reinterpret_cast<float2*>(p) = v[0];
  } else if constexpr (std::is_same<T, double>::value && CH % 2 == 0) {
#pragma unroll
    for (int q = 0; q < CH / 2; ++q)
      reinterpret_cast<double2*>(p)[q] = make_double2(v[2 * q], v[2 * q + 1]);
  } else {
#pragma unroll
    for (int q = 0; q < CH; ++q) p[q] = v[q];
  }
}

// Channels per thread for nch channels per row: the largest of 8 (FP32) or 4
// (FP64), halving, that divides nch and whose vector accesses the row bases
// a and b are aligned for.
template <typename T>
inline int channel_group(int nch, const void* a, const void* b) {
  int ch = sizeof(T) == 4 ? 8 : 4;
  for (; ch > 1; ch /= 2) {
    const size_t al = std::min<size_t>(16, ch * sizeof(T));
    if (nch % ch == 0 && (uintptr_t)a % al == 0 && (uintptr_t)b % al == 0) break;
  }
  return ch;
}

}  // namespace pts
}  // namespace nnmg
