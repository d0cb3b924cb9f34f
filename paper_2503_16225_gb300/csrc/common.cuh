// Shared device helpers of libeacg: complex arithmetic on float2/double2 and
// launch-error plumbing.  Every kernel of the library is written for sm_103a.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include <type_traits>

namespace eacg {

template <typename T>
struct cx;
template <>
struct cx<double> {
  using t = double2;
};
template <>
struct cx<float> {
  using t = float2;
};
template <typename T>
using cplx = typename cx<T>::t;

template <typename V>
__host__ __device__ __forceinline__ V mk(decltype(V::x) a, decltype(V::x) b) {
  V r;
  r.x = a;
  r.y = b;
  return r;
}
__host__ __device__ __forceinline__ double2 operator+(double2 a, double2 b) { return make_double2(a.x + b.x, a.y + b.y); }
__host__ __device__ __forceinline__ double2 operator-(double2 a, double2 b) { return make_double2(a.x - b.x, a.y - b.y); }
__host__ __device__ __forceinline__ float2 operator+(float2 a, float2 b) { return make_float2(a.x + b.x, a.y + b.y); }
__host__ __device__ __forceinline__ float2 operator-(float2 a, float2 b) { return make_float2(a.x - b.x, a.y - b.y); }
__host__ __device__ __forceinline__ double2 cmul(double2 a, double2 b) {
  return make_double2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
__host__ __device__ __forceinline__ float2 cmul(float2 a, float2 b) {
  return make_float2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
// conj(a) * b
__host__ __device__ __forceinline__ double2 cmulc(double2 a, double2 b) {
  return make_double2(a.x * b.x + a.y * b.y, a.x * b.y - a.y * b.x);
}
__host__ __device__ __forceinline__ float2 cmulc(float2 a, float2 b) {
  return make_float2(a.x * b.x + a.y * b.y, a.x * b.y - a.y * b.x);
}
__host__ __device__ __forceinline__ double2 cscale(double2 a, double s) { return make_double2(a.x * s, a.y * s); }
__host__ __device__ __forceinline__ float2 cscale(float2 a, float s) { return make_float2(a.x * s, a.y * s); }
__host__ __device__ __forceinline__ double2 cconj(double2 a) { return make_double2(a.x, -a.y); }
__host__ __device__ __forceinline__ float2 cconj(float2 a) { return make_float2(a.x, -a.y); }
// multiply by -i (forward) or +i (inverse)
template <bool INV, typename V>
__host__ __device__ __forceinline__ V mul_mi(V a) {
  V r;
  if (INV) {
    r.x = -a.y;
    r.y = a.x;
  } else {
    r.x = a.y;
    r.y = -a.x;
  }
  return r;
}

template <typename T>
__device__ __forceinline__ cplx<T> to_c(double2 a) {
  cplx<T> r;
  r.x = (T)a.x;
  r.y = (T)a.y;
  return r;
}
template <typename V>
__device__ __forceinline__ double2 to_d(V a) {
  return make_double2((double)a.x, (double)a.y);
}
// complex conversion between any of float2 / double2
template <typename D, typename S>
__device__ __forceinline__ D cvt(S a) {
  D r;
  r.x = (decltype(r.x))a.x;
  r.y = (decltype(r.y))a.y;
  return r;
}

}  // namespace eacg
