// Complex arithmetic on interleaved float2/double2 values (re = .x, im = .y).
#pragma once
#include <cuda_runtime.h>

namespace hh {

__host__ __device__ __forceinline__ float2 cmk(float a, float b) {
  return make_float2(a, b);
}
__host__ __device__ __forceinline__ double2 cmk(double a, double b) {
  return make_double2(a, b);
}

template <typename C> __host__ __device__ __forceinline__ C czero() {
  C z;
  z.x = 0;
  z.y = 0;
  return z;
}

template <typename C> __device__ __forceinline__ C cadd(C a, C b) {
  return cmk(a.x + b.x, a.y + b.y);
}
template <typename C> __device__ __forceinline__ C csub(C a, C b) {
  return cmk(a.x - b.x, a.y - b.y);
}
template <typename C> __device__ __forceinline__ C cneg(C a) {
  return cmk(-a.x, -a.y);
}
template <typename C> __device__ __forceinline__ C cmul(C a, C b) {
  return cmk(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
// a * b + c
template <typename C> __device__ __forceinline__ C cfma(C a, C b, C c) {
  return cmk(c.x + a.x * b.x - a.y * b.y, c.y + a.x * b.y + a.y * b.x);
}
template <typename C, typename R> __device__ __forceinline__ C cscale(C a, R s) {
  return cmk(a.x * s, a.y * s);
}
template <typename C> __device__ __forceinline__ auto cabs2(C a) {
  return a.x * a.x + a.y * a.y;
}
// a / b = a conj(b) / |b|^2 (the operands here are O(1)..O(1e10) in
// modulus, far from overflow in either precision).
template <typename C> __device__ __forceinline__ C cdiv(C a, C b) {
  const auto d = b.x * b.x + b.y * b.y;
  return cmk((a.x * b.x + a.y * b.y) / d, (a.y * b.x - a.x * b.y) / d);
}
// fused multiply-add a * b + c in the operands' precision
__device__ __forceinline__ float fmaf_any(float a, float b, float c) { return fmaf(a, b, c); }
__device__ __forceinline__ double fmaf_any(double a, double b, double c) { return fma(a, b, c); }
// 1 / b (one real division)
template <typename C> __device__ __forceinline__ C crcp(C b) {
  const auto s = decltype(b.x)(1) / (b.x * b.x + b.y * b.y);
  return cmk(b.x * s, -b.y * s);
}

}  // namespace hh
