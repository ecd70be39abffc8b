// Complex helpers on CUDA's float2 / double2 (interleaved re, im).
#pragma once
#include <cuda_runtime.h>

template <typename R> struct CT;
template <> struct CT<double> { using T = double2; };
template <> struct CT<float> { using T = float2; };

__device__ __forceinline__ double2 mk(double a, double b) { return make_double2(a, b); }
__device__ __forceinline__ float2 mk(float a, float b) { return make_float2(a, b); }

#define LS_CPLX_OPS(T, R)                                                                          \
  __device__ __forceinline__ T cadd(T a, T b) { return mk(a.x + b.x, a.y + b.y); }                \
  __device__ __forceinline__ T csub(T a, T b) { return mk(a.x - b.x, a.y - b.y); }                \
  __device__ __forceinline__ T cmul(T a, T b) { return mk(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x); } \
  __device__ __forceinline__ T cmulc(T a, T b) { return mk(a.x * b.x + a.y * b.y, a.y * b.x - a.x * b.y); } \
  __device__ __forceinline__ T cfma(T a, T b, T c) {                                               \
    return mk(fma(a.x, b.x, fma(-a.y, b.y, c.x)), fma(a.x, b.y, fma(a.y, b.x, c.y)));            \
  }                                                                                                \
  __device__ __forceinline__ T cscale(T a, R s) { return mk(a.x * s, a.y * s); }                    \
  __device__ __forceinline__ T cconj(T a) { return mk(a.x, -a.y); }                                 \
  __device__ __forceinline__ T cmul_i(T a) { return mk(-a.y, a.x); }                                \
  __device__ __forceinline__ T cmul_mi(T a) { return mk(a.y, -a.x); }                               \
  __device__ __forceinline__ T czero(T) { return mk(R(0), R(0)); }

LS_CPLX_OPS(double2, double)
LS_CPLX_OPS(float2, float)
#undef LS_CPLX_OPS

__device__ __forceinline__ double2 shfl_down(double2 v, int d) {
  return make_double2(__shfl_down_sync(0xffffffffu, v.x, d), __shfl_down_sync(0xffffffffu, v.y, d));
}
__device__ __forceinline__ float2 shfl_down(float2 v, int d) {
  return make_float2(__shfl_down_sync(0xffffffffu, v.x, d), __shfl_down_sync(0xffffffffu, v.y, d));
}
template <typename T>
__device__ __forceinline__ T warp_sum(T v) {
#pragma unroll
  for (int d = 16; d > 0; d >>= 1) v = cadd(v, shfl_down(v, d));
  return v;
}
