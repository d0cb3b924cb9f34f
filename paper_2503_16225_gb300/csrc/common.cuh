// Shared device helpers of libeacg: complex arithmetic on float2/double2 and
// launch-error plumbing.  Every kernel of the library is written for sm_103a.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include <type_traits>

namespace eacg {

// ---------------------------------------------------------------- double-float arithmetic
// A dfloat is the unevaluated sum hi + lo of two FP32 numbers (|lo| <= ulp(hi) / 2), about
// 48 significant bits.  GB300 runs FP32 at 64 times its FP64 rate, so FP64-accurate work that
// is add-dominated (the line FFTs) is faster in these pairs than on the FP64 pipe.  The
// building blocks are the error-free transformations of the literature, written from their
// published definitions:
//   two_sum       Knuth, TAOCP Vol. 2, Sec. 4.2.2 (TwoSum, 6 operations, no ordering needed)
//   fast_two_sum  Dekker 1971 (|a| >= |b| or a = 0)
//   two_prod      the FMA form of Dekker's exact product: p = a b, e = fma(a, b, -p)
//   df_add        Joldes, Muller & Popescu, ACM TOMS 2017, accurate double-word addition
//                 (relative error below 3 u^2, u = 2^-24)
//   df_mul        the same paper's double-word product with FMA (error below 5 u^2)
// Every operation uses the round-to-nearest intrinsics, which the compiler never contracts
// or reassociates.
struct dfloat {
  float hi, lo;
  dfloat() = default;
  __host__ __device__ constexpr dfloat(float h, float l) : hi(h), lo(l) {}
  // nearest pair of a double (constants fold at compile time)
  __host__ __device__ constexpr explicit dfloat(double c) : hi((float)c), lo((float)(c - (double)(float)c)) {}
};
struct dcomplex {
  dfloat x, y;
};

__device__ __forceinline__ dfloat two_sum(float a, float b) {
  const float s = __fadd_rn(a, b);
  const float bb = __fsub_rn(s, a);
  const float e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
  return dfloat(s, e);
}
__device__ __forceinline__ dfloat fast_two_sum(float a, float b) {
  const float s = __fadd_rn(a, b);
  return dfloat(s, __fsub_rn(b, __fsub_rn(s, a)));
}
__device__ __forceinline__ dfloat two_prod(float a, float b) {
  const float p = __fmul_rn(a, b);
  return dfloat(p, __fmaf_rn(a, b, -p));
}
__device__ __forceinline__ dfloat df_add(dfloat x, dfloat y) {
  const dfloat s = two_sum(x.hi, y.hi);
  const dfloat t = two_sum(x.lo, y.lo);
  const dfloat v = fast_two_sum(s.hi, __fadd_rn(s.lo, t.hi));
  return fast_two_sum(v.hi, __fadd_rn(t.lo, v.lo));
}
__device__ __forceinline__ dfloat df_neg(dfloat x) { return dfloat(-x.hi, -x.lo); }
__device__ __forceinline__ dfloat df_mul(dfloat x, dfloat y) {
  const dfloat c = two_prod(x.hi, y.hi);
  const float tl = __fmul_rn(x.hi, y.lo);
  const float cl = __fmaf_rn(x.lo, y.hi, tl);
  return fast_two_sum(c.hi, __fadd_rn(c.lo, cl));
}
__device__ __forceinline__ dfloat operator+(dfloat a, dfloat b) { return df_add(a, b); }
__device__ __forceinline__ dfloat operator-(dfloat a, dfloat b) { return df_add(a, df_neg(b)); }
__device__ __forceinline__ dfloat operator-(dfloat a) { return df_neg(a); }
__device__ __forceinline__ dfloat operator*(dfloat a, dfloat b) { return df_mul(a, b); }
// runtime split of a double into its nearest pair (one FP64 subtraction)
__device__ __forceinline__ dfloat df_from(double v) {
  const float h = __double2float_rn(v);
  return dfloat(h, __double2float_rn(v - (double)h));
}
__device__ __forceinline__ double df_to(dfloat a) { return (double)a.hi + (double)a.lo; }

__device__ __forceinline__ dcomplex operator+(dcomplex a, dcomplex b) { return {a.x + b.x, a.y + b.y}; }
__device__ __forceinline__ dcomplex operator-(dcomplex a, dcomplex b) { return {a.x - b.x, a.y - b.y}; }
__device__ __forceinline__ dcomplex cmul(dcomplex a, dcomplex b) {
  return {a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x};
}
__device__ __forceinline__ dcomplex cscale(dcomplex a, dfloat s) { return {a.x * s, a.y * s}; }
template <bool INV>
__device__ __forceinline__ dcomplex mul_mi(dcomplex a) {  // -i a (forward) or +i a (inverse), exact
  return INV ? dcomplex{-a.y, a.x} : dcomplex{a.y, -a.x};
}

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
template <>
struct cx<dfloat> {
  using t = dcomplex;
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
template <typename V>
__device__ __forceinline__ V czero() {
  V r;
  r.x = 0;
  r.y = 0;
  return r;
}
template <>
__device__ __forceinline__ dcomplex czero<dcomplex>() {
  return {dfloat(0.0f, 0.0f), dfloat(0.0f, 0.0f)};
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
template <>
__device__ __forceinline__ double2 to_d<dcomplex>(dcomplex a) {
  return make_double2(df_to(a.x), df_to(a.y));
}
// complex conversion between any of float2 / double2 / dcomplex
template <typename D, typename S>
__device__ __forceinline__ D cvt(S a) {
  if constexpr (std::is_same<D, dcomplex>::value) {
    if constexpr (std::is_same<S, dcomplex>::value) {
      return a;
    } else {
      return {df_from((double)a.x), df_from((double)a.y)};
    }
  } else if constexpr (std::is_same<S, dcomplex>::value) {
    const double2 d = to_d(a);
    D r;
    r.x = (decltype(r.x))d.x;
    r.y = (decltype(r.y))d.y;
    return r;
  } else {
    D r;
    r.x = (decltype(r.x))a.x;
    r.y = (decltype(r.y))a.y;
    return r;
  }
}

}  // namespace eacg
