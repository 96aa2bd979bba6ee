// Complex128 arithmetic in FP32 pairs ("double-float").
//
// GB300 issues FP32 FMAs at about 64x its FP64 rate, and complex128 tile
// passes are bound by the FP64 pipe. Here a real number is held as h + l with
// two floats and combined with error-free transformations: Knuth's TwoSum,
// Dekker's FastTwoSum and the FMA-based TwoProduct (the product's rounding
// error is fma(a, b, -a*b)). Products and sums keep about 46-48 significant
// bits (relative error near 2^-46 per operation; a sum that cancels keeps its
// absolute error at that level of its inputs), against FP64's 53.
//
// Amplitudes stay complex128 in HBM: a tile is split into (h, l) pairs when it
// is loaded and joined back to FP64 when it is stored. The split works on the
// bit pattern (no FP64 instruction): h takes the sign, the exponent and the
// top 23 stored mantissa bits, l the next 23 bits of the remainder. Values
// below 2^-126 in magnitude become 0 (an absolute error below 1e-38), and the
// lowest 6 of the 52 mantissa bits are dropped (2^-46 relative). The join
// widens both floats to FP64 by their bit patterns and adds them once in FP64.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "cplx.cuh"

namespace qs {

struct dfl {
  float h, l;
  dfl() = default;
  __host__ __device__ constexpr dfl(float h_, float l_) : h(h_), l(l_) {}
  __device__ explicit dfl(double d);
  __device__ explicit operator double() const;
};

struct __align__(16) dfc {
  dfl x, y;
};

// s + e = a + b exactly (any magnitudes)
__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e) {
  s = a + b;
  const float bb = s - a;
  e = (a - (s - bb)) + (b - bb);
}
// s + e = a + b exactly when |a| >= |b| (or a = 0)
__device__ __forceinline__ dfl fast_two_sum(float a, float b) {
  const float s = a + b;
  return dfl(s, b - (s - a));
}

__device__ __forceinline__ dfl operator-(dfl a) { return dfl(-a.h, -a.l); }

__device__ __forceinline__ dfl operator+(dfl a, dfl b) {
  float s, e;
  two_sum(a.h, b.h, s, e);
  e += a.l + b.l;
  return fast_two_sum(s, e);
}
__device__ __forceinline__ dfl operator-(dfl a, dfl b) { return a + (-b); }
__device__ __forceinline__ dfl& operator+=(dfl& a, dfl b) { return a = a + b; }

__device__ __forceinline__ dfl operator*(dfl a, dfl b) {
  const float p = a.h * b.h;
  float e = fmaf(a.h, b.h, -p);
  e = fmaf(a.h, b.l, e);
  e = fmaf(a.l, b.h, e);
  return fast_two_sum(p, e);
}

// a * b + c
__device__ __forceinline__ dfl fmac(dfl a, dfl b, dfl c) {
  const float p = a.h * b.h;
  float e = fmaf(a.h, b.h, -p);
  e = fmaf(a.h, b.l, e);
  e = fmaf(a.l, b.h, e);
  float s, t;
  two_sum(p, c.h, s, t);
  t += e + c.l;
  return fast_two_sum(s, t);
}

__device__ __forceinline__ dfl::dfl(double d) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(d);
  const uint32_t hi = (uint32_t)(b >> 32), lo = (uint32_t)b;
  const uint32_t ex = (hi >> 20) & 0x7ffu;     // biased FP64 exponent
  const uint32_t sign = hi & 0x80000000u;
  if (ex <= 896u) {                            // |d| < 2^-126 (or zero): flushed
    h = 0.f;
    l = 0.f;
    return;
  }
  // ex >= 1151 would overflow a float; amplitudes and gate entries are <= 1 in magnitude
  h = __uint_as_float(sign | ((ex - 896u) << 23) | ((hi & 0xfffffu) << 3) | (lo >> 29));
  // remainder r = sign * (lo & 0x1fffffff) * 2^(ex - 1075): X - Y with X = sign * (1 + m 2^-23) * 2^(ex - 1046),
  // Y = sign * 2^(ex - 1046), m = the remainder's top 23 bits (exact subtraction)
  if (ex < 920u) {
    l = 0.f;
    return;
  }
  const uint32_t eb = (ex - 919u) << 23;
  l = __uint_as_float(sign | eb | ((lo & 0x1fffffffu) >> 6)) - __uint_as_float(sign | eb);
}

// float -> double by the bit pattern (normal floats; zero and subnormals -> +-0)
__device__ __forceinline__ double widen(float f) {
  const uint32_t u = __float_as_uint(f);
  const unsigned long long s = (unsigned long long)(u & 0x80000000u) << 32;
  if ((u & 0x7f800000u) == 0) return __longlong_as_double((long long)s);
  // exponent rebias 127 -> 1023 (+896) in 64-bit arithmetic: 896 << 23 does not fit 32 bits
  return __longlong_as_double((long long)(s | (((unsigned long long)(u & 0x7fffffffu) + (896ull << 23)) << 29)));
}

__device__ __forceinline__ dfl::operator double() const { return widen(h) + widen(l); }

template <> struct V2<dfl> { using T = dfc; };

__device__ __forceinline__ dfc to_dfc(double2 a) {
  dfc r;
  r.x = dfl(a.x);
  r.y = dfl(a.y);
  return r;
}
__device__ __forceinline__ double2 from_dfc(dfc a) { return make_double2((double)a.x, (double)a.y); }

}  // namespace qs
