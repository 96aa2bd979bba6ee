// Reductions and Pauli-sum kernels (not in the paper; textbook definitions).
//
// Norm sum_i |psi_i|^2, inner product <a|b>, expectation of Pauli strings
// P|i> = i^{#Y} (-1)^{popcount(i & z)} |i xor x>, and H|psi>.
//
// Every reduction runs on a fixed grid (reduce_blocks() CTAs) so the partial
// sums, and therefore the FP64 result, do not depend on timing. complex64
// states accumulate runs of kRun terms in FP32 and add each run into an FP64
// total; complex128 states accumulate in FP64. The runs are explicit inner
// loops, so the FP64 add happens once per run and not, predicated, once per
// term (GB300's FP64 pipe is about 1/60 of its FP32 rate). Partials are
// combined in FP64 by one CTA in a fixed order.
#include <cuda_runtime.h>

#include "cplx.cuh"
#include "qs_internal.h"

namespace qs {

constexpr int kRedThreads = 256;
// The reduction grid is a fixed constant, deliberately not the device's SM
// count: the CTA partition of the index range, hence every partial sum and the
// order in which they are combined, is the same on every device and every
// run, so the FP64 results are bit-for-bit reproducible. 608 CTAs = four per
// SM on a 152-SM GB300.
constexpr int kRedBlocks = 608;
constexpr int kRun = 32;
constexpr int kUnroll = 4;   // independent 16-byte loads per thread per iteration (bytes in flight)

// 16-byte vector of amplitudes: two complex64 or one complex128.
template <typename R> struct Vec16;
template <> struct Vec16<float> {
  using T = float4;
  static constexpr int amps = 2;
  __device__ __forceinline__ static float2 amp(const float4& v, int k) {
    return k == 0 ? make_float2(v.x, v.y) : make_float2(v.z, v.w);
  }
};
template <> struct Vec16<double> {
  using T = double2;
  static constexpr int amps = 1;
  __device__ __forceinline__ static double2 amp(const double2& v, int) { return v; }
};

__device__ __forceinline__ bool aligned16(const void* p) { return ((uintptr_t)p & 15) == 0; }

// Amplitudes 2v and 2v + 1 (16-byte aligned state): one float4 for complex64,
// two double2 for complex128.
template <typename R> struct AmpPair;
template <> struct AmpPair<float> {
  float4 v;
  __device__ __forceinline__ void load(const void* psi, uint64_t vi) { v = ((const float4*)psi)[vi]; }
  __device__ __forceinline__ void zero() { v = make_float4(0, 0, 0, 0); }
  __device__ __forceinline__ float2 a(int k) const { return k == 0 ? make_float2(v.x, v.y) : make_float2(v.z, v.w); }
};
template <> struct AmpPair<double> {
  double2 v0, v1;
  __device__ __forceinline__ void load(const void* psi, uint64_t vi) {
    v0 = ((const double2*)psi)[2 * vi];
    v1 = ((const double2*)psi)[2 * vi + 1];
  }
  __device__ __forceinline__ void zero() { v0 = v1 = make_double2(0, 0); }
  __device__ __forceinline__ double2 a(int k) const { return k == 0 ? v0 : v1; }
};

int reduce_blocks() { return kRedBlocks; }

// Sum of a per-thread double across the CTA; result valid in thread 0.
__device__ __forceinline__ double block_sum(double v) {
  __shared__ double ws[kRedThreads / 32];
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  __syncthreads();
  if (lane == 0) ws[w] = v;
  __syncthreads();
  double s = 0;
  if (threadIdx.x == 0)
    for (int k = 0; k < kRedThreads / 32; ++k) s += ws[k];
  return s;
}

constexpr int kRunIters = kRun / kUnroll;   // vector iterations per FP32 run

// ---------------------------------------------------------------- norm / inner

// Each thread walks its vectors in a fixed order, kUnroll loads at a time
// (grid stride), so the result is the same on every run.
template <typename R>
__global__ void __launch_bounds__(kRedThreads) k_norm(const typename V2<R>::T* __restrict__ psi, uint64_t dim,
                                                       double* __restrict__ partials) {
  using VT = typename Vec16<R>::T;
  constexpr int A = Vec16<R>::amps;
  double tot = 0;
  const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
  const uint64_t g = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (aligned16(psi) && dim % A == 0) {
    const VT* __restrict__ pv = (const VT*)psi;
    const uint64_t nv = dim / A;
    for (uint64_t b = g; b < nv;) {
      R run = 0;
#pragma unroll 1
      for (int it = 0; it < kRunIters && b < nv; ++it, b += stride * kUnroll) {
        VT v[kUnroll];
#pragma unroll
        for (int u = 0; u < kUnroll; ++u) {
          const uint64_t idx = b + u * stride;
          v[u] = idx < nv ? pv[idx] : VT{};
        }
#pragma unroll
        for (int u = 0; u < kUnroll; ++u)
#pragma unroll
          for (int k = 0; k < A; ++k) {
            const auto a = Vec16<R>::amp(v[u], k);
            run = fmac(a.y, a.y, fmac(a.x, a.x, run));   // two FMAs: the FP64 pipe bounds complex128
          }
      }
      tot += (double)run;
    }
  } else {
    for (uint64_t i = g; i < dim;) {
      R run = 0;
#pragma unroll 1
      for (int it = 0; it < kRun && i < dim; ++it, i += stride) {
        const auto v = psi[i];
        run = fmac(v.y, v.y, fmac(v.x, v.x, run));
      }
      tot += (double)run;
    }
  }
  const double s = block_sum(tot);
  if (threadIdx.x == 0) partials[blockIdx.x] = s;
}

template <typename R>
__global__ void __launch_bounds__(kRedThreads) k_inner(const typename V2<R>::T* __restrict__ a,
                                                        const typename V2<R>::T* __restrict__ b, uint64_t dim,
                                                        double* __restrict__ partials) {
  using VT = typename Vec16<R>::T;
  constexpr int A = Vec16<R>::amps;
  double tre = 0, tim = 0;
  const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
  const uint64_t g = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (aligned16(a) && aligned16(b) && dim % A == 0) {
    const VT* __restrict__ av = (const VT*)a;
    const VT* __restrict__ bv = (const VT*)b;
    const uint64_t nv = dim / A;
    for (uint64_t base = g; base < nv;) {
      R rr = 0, ri = 0;
#pragma unroll 1
      for (int it = 0; it < kRunIters && base < nv; ++it, base += stride * kUnroll) {
        VT va[kUnroll], vb[kUnroll];
#pragma unroll
        for (int u = 0; u < kUnroll; ++u) {
          const uint64_t idx = base + u * stride;
          va[u] = idx < nv ? av[idx] : VT{};
          vb[u] = idx < nv ? bv[idx] : VT{};
        }
#pragma unroll
        for (int u = 0; u < kUnroll; ++u)
#pragma unroll
          for (int k = 0; k < A; ++k) {
            const auto x = Vec16<R>::amp(va[u], k), y = Vec16<R>::amp(vb[u], k);
            rr += x.x * y.x + x.y * y.y;   // conj(x) * y
            ri += x.x * y.y - x.y * y.x;
          }
      }
      tre += (double)rr;
      tim += (double)ri;
    }
  } else {
    for (uint64_t i = g; i < dim;) {
      R rr = 0, ri = 0;
#pragma unroll 1
      for (int it = 0; it < kRun && i < dim; ++it, i += stride) {
        const auto x = a[i], y = b[i];
        rr += x.x * y.x + x.y * y.y;   // conj(x) * y
        ri += x.x * y.y - x.y * y.x;
      }
      tre += (double)rr;
      tim += (double)ri;
    }
  }
  const double sr = block_sum(tre);
  const double si = block_sum(tim);
  if (threadIdx.x == 0) { partials[blockIdx.x] = sr; partials[kRedBlocks + blockIdx.x] = si; }
}

// out[r] = sum_c partials[r * cols + c] in a fixed order (one CTA per row).
__global__ void __launch_bounds__(kRedThreads) k_sum_rows(const double* __restrict__ partials, int cols,
                                                           double* __restrict__ out) {
  const double* row = partials + (int64_t)blockIdx.x * cols;
  double v = 0;
  for (int c = threadIdx.x; c < cols; c += kRedThreads) v += row[c];
  const double s = block_sum(v);
  if (threadIdx.x == 0) out[blockIdx.x] = s;
}

cudaError_t launch_sum_rows(const double* partials, int rows, int cols, double* out, cudaStream_t st) {
  if (rows == 0) return cudaSuccess;
  k_sum_rows<<<rows, kRedThreads, 0, st>>>(partials, cols, out);
  note_launch();
  return cudaGetLastError();
}

cudaError_t launch_norm(const void* psi, int n, qs_dtype dt, double* partials, double* out, cudaStream_t st) {
  const uint64_t dim = 1ull << n;
  if (dt == QS_C64) k_norm<float><<<kRedBlocks, kRedThreads, 0, st>>>((const float2*)psi, dim, partials);
  else k_norm<double><<<kRedBlocks, kRedThreads, 0, st>>>((const double2*)psi, dim, partials);
  note_launch();
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  return launch_sum_rows(partials, 1, kRedBlocks, out, st);
}

cudaError_t launch_inner(const void* a, const void* b, int n, qs_dtype dt, double* partials, double* out2,
                         cudaStream_t st) {
  const uint64_t dim = 1ull << n;
  if (dt == QS_C64)
    k_inner<float><<<kRedBlocks, kRedThreads, 0, st>>>((const float2*)a, (const float2*)b, dim, partials);
  else
    k_inner<double><<<kRedBlocks, kRedThreads, 0, st>>>((const double2*)a, (const double2*)b, dim, partials);
  note_launch();
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  return launch_sum_rows(partials, 2, kRedBlocks, out2, st);
}

// ---------------------------------------------------------------- state difference

// Per-CTA max |a_i - b_i| and sum |a_i - b_i|^2 (FP64) of two states of any dtypes.
template <typename RA, typename RB>
__global__ void __launch_bounds__(kRedThreads) k_diff(const typename V2<RA>::T* __restrict__ a,
                                                       const typename V2<RB>::T* __restrict__ b, uint64_t dim,
                                                       double* __restrict__ partials) {
  double mx = 0, sq = 0;
  const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
  for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < dim; i += stride) {
    const double dx = (double)a[i].x - (double)b[i].x, dy = (double)a[i].y - (double)b[i].y;
    const double d2 = dx * dx + dy * dy;
    sq += d2;
    mx = fmax(mx, d2);
  }
  const double s = block_sum(sq);
  __shared__ double wm[kRedThreads / 32];
  for (int o = 16; o > 0; o >>= 1) mx = fmax(mx, __shfl_down_sync(0xffffffffu, mx, o));
  __syncthreads();
  if ((threadIdx.x & 31) == 0) wm[threadIdx.x >> 5] = mx;
  __syncthreads();
  if (threadIdx.x == 0) {
    double m = 0;
    for (int k = 0; k < kRedThreads / 32; ++k) m = fmax(m, wm[k]);
    partials[blockIdx.x] = sqrt(m);
    partials[kRedBlocks + blockIdx.x] = s;
  }
}

cudaError_t launch_diff(const void* a, qs_dtype da, const void* b, qs_dtype db, int n, double* partials,
                        cudaStream_t st) {
  const uint64_t dim = 1ull << n;
  if (da == QS_C64 && db == QS_C64)
    k_diff<float, float><<<kRedBlocks, kRedThreads, 0, st>>>((const float2*)a, (const float2*)b, dim, partials);
  else if (da == QS_C64)
    k_diff<float, double><<<kRedBlocks, kRedThreads, 0, st>>>((const float2*)a, (const double2*)b, dim, partials);
  else if (db == QS_C64)
    k_diff<double, float><<<kRedBlocks, kRedThreads, 0, st>>>((const double2*)a, (const float2*)b, dim, partials);
  else
    k_diff<double, double><<<kRedBlocks, kRedThreads, 0, st>>>((const double2*)a, (const double2*)b, dim, partials);
  note_launch();
  return cudaGetLastError();
}

// ---------------------------------------------------------------- Pauli expval

constexpr int kMaxZ = kExpvalMaxZ;

// One sweep for all strings sharing xmask x. Pairs (i, j = i xor x) are
// visited once (i has the highest bit of x clear). For w = conj(psi_j) psi_i:
//   <P> contribution = i^{ny} s_i (w + (-1)^{ny} conj(w)),  s_i = (-1)^{popcount(i & z)}
// which is s_i * 2 Re(w) * (-1)^{ny/2} for even ny and s_i * 2 Im(w) * (-1)^{(ny+1)/2}
// for odd ny (the sign and the re/im choice are folded into coef/odd below).
// x = 0: each index once, contribution s_i |psi_i|^2.
template <typename R>
__global__ void __launch_bounds__(kRedThreads) k_expval_x(const typename V2<R>::T* __restrict__ psi, int n,
                                                           uint64_t x, const uint64_t* __restrict__ zm,
                                                           int nz, double* __restrict__ partials) {
  __shared__ uint64_t z_s[kMaxZ];
  __shared__ int odd_s[kMaxZ];
  if (threadIdx.x < nz) {
    z_s[threadIdx.x] = zm[threadIdx.x];
    odd_s[threadIdx.x] = __popcll(x & zm[threadIdx.x]) & 1;
  }
  __syncthreads();
  double tot[kMaxZ];
  R run[kMaxZ];
#pragma unroll
  for (int k = 0; k < kMaxZ; ++k) tot[k] = 0;
  auto fold = [&]() {
#pragma unroll
    for (int k = 0; k < kMaxZ; ++k) {
      if (k < nz) tot[k] += (double)run[k];
      run[k] = 0;
    }
  };
  const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
  const uint64_t g = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (x == 0) {
    using VT = typename Vec16<R>::T;
    constexpr int A = Vec16<R>::amps;
    const uint64_t dim = 1ull << n;
    if (aligned16(psi) && dim % A == 0) {
      const VT* __restrict__ pv = (const VT*)psi;
      const uint64_t nv = dim / A;
      for (uint64_t b = g; b < nv;) {
#pragma unroll
        for (int k = 0; k < kMaxZ; ++k) run[k] = 0;
#pragma unroll 1
        for (int it = 0; it < kRunIters && b < nv; ++it, b += stride * kUnroll) {
          VT v[kUnroll];
#pragma unroll
          for (int u = 0; u < kUnroll; ++u) {
            const uint64_t idx = b + u * stride;
            v[u] = idx < nv ? pv[idx] : VT{};
          }
#pragma unroll
          for (int u = 0; u < kUnroll; ++u) {
            const uint64_t i0 = (b + u * stride) * A;
#pragma unroll
            for (int e = 0; e < A; ++e) {
              const auto a = Vec16<R>::amp(v[u], e);
              const R p = a.x * a.x + a.y * a.y;
#pragma unroll
              for (int k = 0; k < kMaxZ; ++k)
                if (k < nz) run[k] += (__popcll((i0 + e) & z_s[k]) & 1) ? -p : p;
            }
          }
        }
        fold();
      }
    } else {
      for (uint64_t i = g; i < dim;) {
#pragma unroll
        for (int k = 0; k < kMaxZ; ++k) run[k] = 0;
#pragma unroll 1
        for (int it = 0; it < kRun && i < dim; ++it, i += stride) {
          const auto a = psi[i];
          const R p = a.x * a.x + a.y * a.y;
#pragma unroll
          for (int k = 0; k < kMaxZ; ++k)
            if (k < nz) run[k] += (__popcll(i & z_s[k]) & 1) ? -p : p;
        }
        fold();
      }
    }
  } else {
    const int32_t hb = 63 - __clzll((long long)x);
    const uint64_t count = 1ull << (n - 1);
    for (uint64_t p0 = g; p0 < count;) {
#pragma unroll
      for (int k = 0; k < kMaxZ; ++k) run[k] = 0;
#pragma unroll 1
      for (int it = 0; it < kRunIters && p0 < count; ++it, p0 += stride * kUnroll) {
        typename V2<R>::T a[kUnroll], b[kUnroll];
#pragma unroll
        for (int u = 0; u < kUnroll; ++u) {
          const uint64_t p = p0 + u * stride;
          const uint64_t i = ((p >> hb) << (hb + 1)) | (p & ((1ull << hb) - 1));
          if (p < count) {
            a[u] = psi[i];
            b[u] = psi[i ^ x];
          } else {
            a[u] = mk<R>(0, 0);
            b[u] = mk<R>(0, 0);
          }
        }
#pragma unroll
        for (int u = 0; u < kUnroll; ++u) {
          const uint64_t p = p0 + u * stride;
          const uint64_t i = ((p >> hb) << (hb + 1)) | (p & ((1ull << hb) - 1));
          const R wr = b[u].x * a[u].x + b[u].y * a[u].y;   // Re(conj(b) a)
          const R wi = b[u].x * a[u].y - b[u].y * a[u].x;   // Im(conj(b) a)
#pragma unroll
          for (int k = 0; k < kMaxZ; ++k) {
            if (k < nz) {
              const R v = odd_s[k] ? wi : wr;
              run[k] += (__popcll(i & z_s[k]) & 1) ? -v : v;
            }
          }
        }
      }
      fold();
    }
  }
#pragma unroll
  for (int k = 0; k < kMaxZ; ++k) {
    if (k < nz) {
      const double s = block_sum(tot[k]);
      if (threadIdx.x == 0) partials[(int64_t)k * gridDim.x + blockIdx.x] = s;
    }
  }
}

cudaError_t launch_expval_x(const void* psi, int n, qs_dtype dt, uint64_t xmask, const uint64_t* zm,
                            const double* /*coeffs*/, int nz, double* partials, double* out, cudaStream_t st) {
  if (nz > kMaxZ) return cudaErrorInvalidValue;
  if (dt == QS_C64)
    k_expval_x<float><<<kRedBlocks, kRedThreads, 0, st>>>((const float2*)psi, n, xmask, zm, nz, partials);
  else
    k_expval_x<double><<<kRedBlocks, kRedThreads, 0, st>>>((const double2*)psi, n, xmask, zm, nz, partials);
  note_launch();
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  return launch_sum_rows(partials, nz, kRedBlocks, out, st);
}

// ---------------------------------------------------------------- batched, L2-resident waves

// All Pauli groups for the states [b0, b0 + gridDim.y) of a batch in one
// launch. A wave's states (a few MiB each) stay resident in L2 while every
// group sweeps them, so each state is read from HBM about once per wave
// instead of once per group. CTA (c, s) sweeps slice c of state b0 + s for
// every group in turn; partials[(b Z + zi) C + c] receives its FP64 sum for
// string zi (C = gridDim.x). Loads take amplitude pairs (2v, 2v + 1): for x
// with its highest bit hb >= 1, pairs 2q and 2q + 1 start at consecutive even
// indices i, i + 1 and their partners i ^ x, (i + 1) ^ x form one aligned
// pair (swapped when x is odd); x = 1 pairs the two halves of an item; x = 0
// takes two diagonal terms per item. NZ bounds the strings of a group; I is
// the index type (32-bit while 2^n fits). i is even, so the sign parity of
// i + 1 is that of i xor bit 0 of z: one popcount per item and string.
template <typename R, int NZ, typename I>
__global__ void __launch_bounds__(kRedThreads) k_expval_groups(const void* const* __restrict__ psis, int b0, int n,
                                                                const uint64_t* __restrict__ gx,
                                                                const int32_t* __restrict__ gz,
                                                                const int32_t* __restrict__ gc,
                                                                const int32_t* __restrict__ glist, int ngroups,
                                                                const uint64_t* __restrict__ zl, int Z,
                                                                double* __restrict__ partials) {
  using C2 = typename V2<R>::T;
  const int b = b0 + blockIdx.y;
  const void* __restrict__ psi = psis[b];
  const uint64_t cta = blockIdx.x, ncta = gridDim.x;
  for (int li = 0; li < ngroups; ++li) {
    const int l = glist[li];
    const uint64_t x = gx[l];
    const int zoff = gz[l], nz = gc[l];
    I zm[NZ];
    int odd[NZ];
#pragma unroll
    for (int k = 0; k < NZ; ++k) {
      const uint64_t z = k < nz ? zl[zoff + k] : 0;
      zm[k] = (I)z;
      odd[k] = __popcll(x & z) & 1;
    }
    const I xi = (I)x;
    double tot[NZ];
    R run[NZ];
#pragma unroll
    for (int k = 0; k < NZ; ++k) tot[k] = 0;
    const int32_t hb = x == 0 ? -1 : 63 - __clzll((long long)x);
    // vector items: x = 0 -> 2^(n-1) vectors of two amplitudes; x = 1 -> 2^(n-1) vectors
    // (one pair each); hb >= 1 -> 2^(n-2) pairs of pairs
    const I items = hb >= 1 ? ((I)1 << (n - 2)) : ((I)1 << (n - 1));
    const I lo = (I)((uint64_t)items * cta / ncta), hi = (I)((uint64_t)items * (cta + 1) / ncta);
    const I hmask = hb >= 1 ? (((I)1 << hb) - 1) : 0;
    // the two terms of an item: amplitudes i (even) and i + 1 against partners b0, b1
    auto accum2 = [&](const C2& a0, const C2& p0, const C2& a1, const C2& p1, I i0, bool two) {
      const R wr0 = p0.x * a0.x + p0.y * a0.y, wi0 = p0.x * a0.y - p0.y * a0.x;   // conj(b) a
      const R wr1 = p1.x * a1.x + p1.y * a1.y, wi1 = p1.x * a1.y - p1.y * a1.x;
#pragma unroll
      for (int k = 0; k < NZ; ++k) {
        if (k < nz) {
          const int par = __popc((uint32_t)(i0 & zm[k])) + (sizeof(I) > 4 ? __popc((uint32_t)((uint64_t)(i0 & zm[k]) >> 32)) : 0);
          const R v0 = odd[k] ? wi0 : wr0;
          run[k] += (par & 1) ? -v0 : v0;
          if (two) {
            const R v1 = odd[k] ? wi1 : wr1;
            run[k] += ((par ^ (int)zm[k]) & 1) ? -v1 : v1;
          }
        }
      }
    };
    for (I q0 = lo + threadIdx.x; q0 < hi;) {
#pragma unroll
      for (int k = 0; k < NZ; ++k) run[k] = 0;
#pragma unroll 1
      for (int it = 0; it < kRunIters && q0 < hi; ++it, q0 += (I)(kRedThreads * kUnroll)) {
        AmpPair<R> va[kUnroll], vb[kUnroll];
        I iu[kUnroll];
#pragma unroll
        for (int u = 0; u < kUnroll; ++u) {
          const I q2 = 2 * (q0 + (I)(u * kRedThreads));
          // first amplitude index of the item
          iu[u] = hb >= 1 ? (((q2 >> hb) << (hb + 1)) | (q2 & hmask)) : q2;
          if (q0 + (I)(u * kRedThreads) < hi) {
            va[u].load(psi, iu[u] >> 1);
            if (hb >= 1) vb[u].load(psi, (iu[u] ^ xi) >> 1);
            else vb[u] = va[u];
          } else {
            va[u].zero();
            vb[u].zero();
          }
        }
#pragma unroll
        for (int u = 0; u < kUnroll; ++u) {
          const C2 a0 = va[u].a(0), a1 = va[u].a(1);
          if (hb < 0) {            // diagonal: two indices per item
            accum2(a0, a0, a1, a1, iu[u], true);
          } else if (hb == 0) {    // x = 1: the item holds the pair
            accum2(a0, a1, a0, a1, iu[u], false);
          } else {
            const C2 p0 = vb[u].a(0), p1 = vb[u].a(1);
            const bool sw = (x & 1) != 0;
            accum2(a0, sw ? p1 : p0, a1, sw ? p0 : p1, iu[u], true);
          }
        }
      }
#pragma unroll
      for (int k = 0; k < NZ; ++k)
        if (k < nz) tot[k] += (double)run[k];
    }
#pragma unroll
    for (int k = 0; k < NZ; ++k) {
      if (k < nz) {
        const double s = block_sum(tot[k]);
        if (threadIdx.x == 0) partials[((int64_t)b * Z + zoff + k) * ncta + cta] = s;
      }
    }
  }
}

int expval_wave_states(int n, qs_dtype dt, int nstates) {
  const uint64_t bytes = (1ull << n) * (dt == QS_C64 ? 8 : 16);
  const uint64_t budget = 64ull << 20;   // about half of L2
  uint64_t s = bytes >= budget ? 1 : budget / bytes;
  if (s > (uint64_t)nstates) s = nstates;
  return (int)s;
}
int expval_wave_ctas(int wave_states) {
  const int c = kRedBlocks / wave_states;
  return c < 1 ? 1 : c;
}

template <typename R, typename I>
static void expval_groups_wave(dim3 grid, cudaStream_t st, const void* const* psis, int b0, int n, const uint64_t* gx,
                               const int32_t* gz, const int32_t* gc, const int32_t* glist, int ngroups1,
                               int ngroups, const uint64_t* zl, int Z, double* partials) {
  if (ngroups1)
    k_expval_groups<R, 1, I><<<grid, kRedThreads, 0, st>>>(psis, b0, n, gx, gz, gc, glist, ngroups1, zl, Z,
                                                           partials);
  if (ngroups > ngroups1)
    k_expval_groups<R, kMaxZ, I><<<grid, kRedThreads, 0, st>>>(psis, b0, n, gx, gz, gc, glist + ngroups1,
                                                               ngroups - ngroups1, zl, Z, partials);
}

cudaError_t launch_expval_groups_batched(const void* const* psis, int nstates, int n, qs_dtype dt,
                                         const uint64_t* gx, const int32_t* gz, const int32_t* gc,
                                         const int32_t* glist, int ngroups1, int ngroups, const uint64_t* zl, int Z,
                                         double* partials, double* out, cudaStream_t st) {
  // glist[0, ngroups1): groups with one string; glist[ngroups1, ngroups): the rest
  const int S = expval_wave_states(n, dt, nstates);
  const int C = expval_wave_ctas(S);
  const bool i32 = n <= 31;
  for (int b0 = 0; b0 < nstates; b0 += S) {
    const int nb = nstates - b0 < S ? nstates - b0 : S;
    const dim3 grid(C, nb);
    if (dt == QS_C64) {
      if (i32) expval_groups_wave<float, uint32_t>(grid, st, psis, b0, n, gx, gz, gc, glist, ngroups1, ngroups, zl, Z, partials);
      else expval_groups_wave<float, uint64_t>(grid, st, psis, b0, n, gx, gz, gc, glist, ngroups1, ngroups, zl, Z, partials);
    } else {
      if (i32) expval_groups_wave<double, uint32_t>(grid, st, psis, b0, n, gx, gz, gc, glist, ngroups1, ngroups, zl, Z, partials);
      else expval_groups_wave<double, uint64_t>(grid, st, psis, b0, n, gx, gz, gc, glist, ngroups1, ngroups, zl, Z, partials);
    }
    note_launch((ngroups1 ? 1 : 0) + (ngroups > ngroups1 ? 1 : 0));
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
  }
  return launch_sum_rows(partials, nstates * Z, C, out, st);
}

// ---------------------------------------------------------------- H |psi>

constexpr int kMaxTermsPerLaunch = 512;

// out[k] = sum_j c_j i^{ny_j} (-1)^{popcount((k xor x_j) & z_j)} psi[k xor x_j]
// (thread per output index; a warp's reads psi[k xor x] stay within one
// aligned 32-amplitude segment, so they coalesce).
template <typename R>
__global__ void __launch_bounds__(kRedThreads) k_apply_pauli(const typename V2<R>::T* __restrict__ psi,
                                                              typename V2<R>::T* __restrict__ out, uint64_t dim,
                                                              const uint64_t* __restrict__ xm,
                                                              const uint64_t* __restrict__ zm,
                                                              const double2* __restrict__ ph, int nt,
                                                              int accumulate) {
  using C = typename V2<R>::T;
  __shared__ uint64_t xs[kMaxTermsPerLaunch], zs[kMaxTermsPerLaunch];
  __shared__ C cs[kMaxTermsPerLaunch];
  for (int j = threadIdx.x; j < nt; j += blockDim.x) { xs[j] = xm[j]; zs[j] = zm[j]; cs[j] = from_d<R>(ph[j]); }
  __syncthreads();
  const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
  for (uint64_t k = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; k < dim; k += stride) {
    C acc = accumulate ? out[k] : mk<R>(0, 0);
    for (int j = 0; j < nt; ++j) {
      const uint64_t src = k ^ xs[j];
      C v = psi[src];
      if (__popcll(src & zs[j]) & 1) { v.x = -v.x; v.y = -v.y; }
      acc = cfma(cs[j], v, acc);
    }
    out[k] = acc;
  }
}

// ph[j] = c_j * i^{ny_j}, prepared on the host.
cudaError_t launch_apply_pauli(const void* psi, void* out, int n, qs_dtype dt, const uint64_t* xm,
                               const uint64_t* zm, const double* ph, int nt, cudaStream_t st) {
  const uint64_t dim = 1ull << n;
  int first = 1;
  for (int off = 0; off < nt || first; off += kMaxTermsPerLaunch) {
    const int cnt = nt - off < kMaxTermsPerLaunch ? nt - off : kMaxTermsPerLaunch;
    uint64_t g = (dim + kRedThreads - 1) / kRedThreads;
    const uint64_t cap = (uint64_t)device_sm_count() * 16;
    if (g > cap) g = cap;
    if (dt == QS_C64)
      k_apply_pauli<float><<<(unsigned)g, kRedThreads, 0, st>>>((const float2*)psi, (float2*)out, dim, xm + off,
                                                                 zm + off, (const double2*)ph + off, cnt, !first);
    else
      k_apply_pauli<double><<<(unsigned)g, kRedThreads, 0, st>>>((const double2*)psi, (double2*)out, dim, xm + off,
                                                                  zm + off, (const double2*)ph + off, cnt, !first);
    note_launch();
    first = 0;
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    if (off + kMaxTermsPerLaunch >= nt) break;
  }
  return cudaSuccess;
}

}  // namespace qs
