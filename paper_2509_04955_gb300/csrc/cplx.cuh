// Complex helpers on float2 / double2 (x = re, y = im), shared by the kernels.
#pragma once
#include <cuda_runtime.h>

namespace qs {

template <typename R> struct V2;
template <> struct V2<float> { using T = float2; };
template <> struct V2<double> { using T = double2; };

template <typename R> __device__ __forceinline__ typename V2<R>::T mk(R x, R y) {
  typename V2<R>::T v; v.x = x; v.y = y; return v;
}

// Scalar a*b + c for every scalar the kernels use (float, double, and the
// FP32-pair type of dfloat.cuh, found by argument-dependent lookup).
__device__ __forceinline__ float fmac(float a, float b, float c) { return fmaf(a, b, c); }
__device__ __forceinline__ double fmac(double a, double b, double c) { return ::fma(a, b, c); }

// a*b
template <typename C> __device__ __forceinline__ C cmul(C a, C b) {
  C r; r.x = a.x * b.x - a.y * b.y; r.y = a.x * b.y + a.y * b.x; return r;
}
// acc + a*b
template <typename C> __device__ __forceinline__ C cfma(C a, C b, C acc) {
  acc.x = fmac(a.x, b.x, acc.x); acc.x = fmac(-a.y, b.y, acc.x);
  acc.y = fmac(a.x, b.y, acc.y); acc.y = fmac(a.y, b.x, acc.y);
  return acc;
}
template <typename C> __device__ __forceinline__ C cconj(C a) { a.y = -a.y; return a; }

// p*a + q*b with real p, q
template <typename R> __device__ __forceinline__ typename V2<R>::T rmix(R p, typename V2<R>::T a, R q,
                                                                       typename V2<R>::T b) {
  typename V2<R>::T r;
  r.x = fmac(q, b.x, p * a.x);
  r.y = fmac(q, b.y, p * a.y);
  return r;
}
// p*a + (i q)*b with real p, q
template <typename R> __device__ __forceinline__ typename V2<R>::T ixmix(R p, typename V2<R>::T a, R q,
                                                                        typename V2<R>::T b) {
  typename V2<R>::T r;
  r.x = fmac(-q, b.y, p * a.x);
  r.y = fmac(q, b.x, p * a.y);
  return r;
}

template <typename R> __device__ __forceinline__ typename V2<R>::T from_d(double2 d) {
  return mk<R>((R)d.x, (R)d.y);
}

}  // namespace qs
