// Diagonal phase pass: one HBM sweep that multiplies amplitude x by
//   D(x) = prod_j exp(i alpha_j s_j(x)),   s_j(x) = (-1)^popcount(mask_j & x),
// the phase polynomial of a run of CNOTs and diagonal gates whose basis
// permutation composes to the identity (a QAOA cost layer, Section 4.1's third
// circuit class: every exp(-i gamma Z_u Z_v) is CNOT . RZ . CNOT).
//
// The index splits into lo = bits 0..11 and hi = bits 12..n-1. A term's sign
// is (-1)^(parity(mask_lo & lo) xor parity(mask_hi & hi)), so the terms fall
// into four classes (the host sorts them):
//   LOW   mask_hi = 0, >= 2 lo bits: a function of lo alone; multiplied into
//         the 4096-entry table E[lo] once per CTA;
//   LIN   one lo bit u: for a fixed hi, a factor w_u or conj(w_u) by bit u of
//         lo, where w_u is the product of the u-terms with their hi signs;
//   HIGH  mask_lo = 0: a constant for a fixed hi;
//   MIXED the rest (>= 2 lo bits and hi bits): a per-amplitude factor.
// A warp owns a chunk of 4096 consecutive amplitudes (one hi); it forms
// A[l1] = C prod_{u<6} w_u^{+-1} and B[l2] = prod_{u>=6} w_u^{+-1} over the
// 64 values of each half of lo in its own shared memory, then streams the
// chunk with 16-byte loads: D(x) = E[lo] B[lo >> 6] A[lo & 63] (x MIXED).
// Three complex products per amplitude: HBM-bound for complex64 (FP32),
// bound by GB300's FP64 pipe for complex128, unless the plan computes
// complex128 in FP32 pairs (dfloat.cuh): the amplitudes are then split into
// pairs as they are loaded and joined as they are stored.
#include <cuda_runtime.h>

#include <algorithm>

#include "cplx.cuh"
#include "dfloat.cuh"
#include "qs_internal.h"

namespace qs {

constexpr int kPhaseThreads = 256;
constexpr int kPhaseWarps = kPhaseThreads / 32;
constexpr int kPhaseChunk = 1 << kPhaseChunkBits;   // 4096 amplitudes

__device__ __forceinline__ int parity64(uint64_t v) { return __popcll(v) & 1; }

template <typename C> __device__ __forceinline__ C conj_if(C z, int flip) {
  if (flip) z.y = -z.y;
  return z;
}

__device__ __forceinline__ float shfl_r(float v, int src) { return __shfl_sync(0xffffffffu, v, src); }
__device__ __forceinline__ double shfl_r(double v, int src) { return __shfl_sync(0xffffffffu, v, src); }
__device__ __forceinline__ dfl shfl_r(dfl v, int src) {
  return dfl(__shfl_sync(0xffffffffu, v.h, src), __shfl_sync(0xffffffffu, v.l, src));
}
__device__ __forceinline__ float shfl_xor_r(float v, int m) { return __shfl_xor_sync(0xffffffffu, v, m); }
__device__ __forceinline__ double shfl_xor_r(double v, int m) { return __shfl_xor_sync(0xffffffffu, v, m); }
__device__ __forceinline__ dfl shfl_xor_r(dfl v, int m) {
  return dfl(__shfl_xor_sync(0xffffffffu, v.h, m), __shfl_xor_sync(0xffffffffu, v.l, m));
}

template <typename C> __device__ __forceinline__ C shfl_c(C v, int src) {
  v.x = shfl_r(v.x, src);
  v.y = shfl_r(v.y, src);
  return v;
}

// amplitude type in HBM; complex128 computed in FP32 pairs keeps complex128 there
template <typename R> struct PhaseG { using T = typename V2<R>::T; };
template <> struct PhaseG<dfl> { using T = double2; };
__device__ __forceinline__ double2 to_calc(double2 a, double) { return a; }
__device__ __forceinline__ dfc to_calc(double2 a, dfl) { return to_dfc(a); }
__device__ __forceinline__ double2 to_mem(double2 a) { return a; }
__device__ __forceinline__ double2 to_mem(dfc a) { return from_dfc(a); }

template <typename R> __device__ __forceinline__ typename V2<R>::T c_one() { return mk<R>(R(1.0), R(0.0)); }

// z_j and mask_j arrays are sized for an even count, which keeps the per-warp
// tables after them 16-byte aligned
__host__ __device__ __forceinline__ int phase_terms_padded(int nterms) { return (nterms + 1) & ~1; }

size_t phase_smem_bytes(int nterms, qs_dtype dt) {
  const size_t c = dt == QS_C64 ? 8 : 16;
  return c * kPhaseChunk                          // E
         + (c + 8) * (size_t)phase_terms_padded(nterms)   // z_j and mask_j
         + c * kPhaseWarps * (128 + kPhaseMaxMixed);   // per warp: A, B, MIXED factors
}

template <typename R>
__global__ void __launch_bounds__(kPhaseThreads) k_phase_pass(void* psi0, void* const* psis, int n,
                                                              const DevPhaseTerm* __restrict__ terms,
                                                              PhasePassDesc d, const double* __restrict__ theta,
                                                              int64_t ntheta) {
  using C = typename V2<R>::T;
  using G = typename PhaseG<R>::T;
  extern __shared__ __align__(16) unsigned char smem[];
  C* E = reinterpret_cast<C*>(smem);
  C* Z = E + kPhaseChunk;
  uint64_t* M = reinterpret_cast<uint64_t*>(Z + phase_terms_padded(d.nterms));
  C* AB = reinterpret_cast<C*>(M + phase_terms_padded(d.nterms));
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  C* ab = AB + warp * (128 + kPhaseMaxMixed);
  C* mx = ab + 128;

  const int row = blockIdx.y;
  G* psi = reinterpret_cast<G*>(psis ? psis[row] : psi0);
  const DevPhaseTerm* T = terms + d.term_off;

  // z_j = exp(i alpha_j): angles in FP64 from theta, rounded to the state's precision
  for (int j = threadIdx.x; j < d.nterms; j += kPhaseThreads) {
    const DevPhaseTerm t = T[j];
    double a = t.alpha0;
    if (t.pidx >= 0) a += t.coef * theta[(int64_t)row * ntheta + t.pidx];
    double s, c;
    sincos(a, &s, &c);
    Z[j] = mk<R>(R(c), R(s));
    M[j] = t.mask;
  }
  __syncthreads();
  for (int lo = threadIdx.x; lo < kPhaseChunk; lo += kPhaseThreads) {
    C e = c_one<R>();
    for (int j = 0; j < d.nlow; ++j) e = cmul(e, conj_if(Z[j], parity64(M[j] & (uint64_t)lo)));
    E[lo] = e;
  }
  __syncthreads();

  const int nmixed = d.nterms - d.mixed_begin;
  int u_lo = 0, u_hi = 0;   // (constant-index reads keep the descriptor out of local memory)
#pragma unroll
  for (int u = 0; u < kPhaseChunkBits; ++u)
    if (lane == u) {
      u_lo = d.lin_off[u];
      u_hi = d.lin_off[u + 1];
    }
  const uint64_t nchunks = 1ull << (n - kPhaseChunkBits);
  for (uint64_t ch = (uint64_t)blockIdx.x * kPhaseWarps + warp; ch < nchunks;
       ch += (uint64_t)gridDim.x * kPhaseWarps) {
    const uint64_t base = ch << kPhaseChunkBits;
    // C = product of the HIGH terms (spread over the lanes, then a butterfly product)
    C cst = c_one<R>();
    for (int j = d.high_begin + lane; j < d.mixed_begin; j += 32)
      cst = cmul(cst, conj_if(Z[j], parity64(M[j] & base)));
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      C other;
      other.x = shfl_xor_r(cst.x, o);
      other.y = shfl_xor_r(cst.y, o);
      cst = cmul(cst, other);
    }
    // lane u < 12: w_u = product of its LIN terms with their hi signs
    C wv = c_one<R>();
    for (int j = u_lo; j < u_hi; ++j) wv = cmul(wv, conj_if(Z[j], parity64(M[j] & base)));
    C w[kPhaseChunkBits];
#pragma unroll
    for (int u = 0; u < kPhaseChunkBits; ++u) w[u] = shfl_c(wv, u);
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const int e = lane + 32 * h;
      C a = cst, b = c_one<R>();
#pragma unroll
      for (int u = 0; u < 6; ++u) {
        a = cmul(a, conj_if(w[u], (e >> u) & 1));
        b = cmul(b, conj_if(w[6 + u], (e >> u) & 1));
      }
      ab[e] = a;
      ab[64 + e] = b;
    }
    if (lane < nmixed) mx[lane] = conj_if(Z[d.mixed_begin + lane], parity64(M[d.mixed_begin + lane] & base));
    __syncwarp();

    if constexpr (sizeof(R) == 4) {
      // lane l holds float4 f = l + 32 i (amplitudes 2f, 2f + 1): lo & 63 = 2l + b, lo >> 6 = i
      float4* p4 = reinterpret_cast<float4*>(psi + base);
      const float4* E4 = reinterpret_cast<const float4*>(E);
      const C a0 = ab[2 * lane], a1 = ab[2 * lane + 1];
#pragma unroll 1
      for (int i0 = 0; i0 < 64; i0 += 8) {
        float4 v[8];
#pragma unroll
        for (int k = 0; k < 8; ++k) v[k] = p4[lane + 32 * (i0 + k)];
#pragma unroll
        for (int k = 0; k < 8; ++k) {
          const int i = i0 + k;
          const C bi = ab[64 + i];
          const float4 e = E4[lane + 32 * i];
          C f0 = cmul(cmul(mk<R>(e.x, e.y), bi), a0);
          C f1 = cmul(cmul(mk<R>(e.z, e.w), bi), a1);
          if (nmixed) {
            const uint64_t lo = 2 * (uint64_t)(lane + 32 * i);
            for (int j = 0; j < nmixed; ++j) {
              const uint64_t m = M[d.mixed_begin + j];
              f0 = cmul(f0, conj_if(mx[j], parity64(m & lo)));
              f1 = cmul(f1, conj_if(mx[j], parity64(m & (lo + 1))));
            }
          }
          const C x0 = cmul(mk<R>(v[k].x, v[k].y), f0), x1 = cmul(mk<R>(v[k].z, v[k].w), f1);
          v[k] = make_float4(x0.x, x0.y, x1.x, x1.y);
        }
#pragma unroll
        for (int k = 0; k < 8; ++k) p4[lane + 32 * (i0 + k)] = v[k];
      }
    } else {
      // lane l holds amplitude l + 32 i: lo & 63 = l + 32 (i & 1), lo >> 6 = i >> 1
      G* p = psi + base;
      const C a0 = ab[lane], a1 = ab[lane + 32];
#pragma unroll 1
      for (int i0 = 0; i0 < 128; i0 += 4) {
        G v[4];
#pragma unroll
        for (int k = 0; k < 4; ++k) v[k] = p[lane + 32 * (i0 + k)];
#pragma unroll
        for (int k = 0; k < 4; ++k) {
          const int i = i0 + k;
          C f = cmul(cmul(E[lane + 32 * i], ab[64 + (i >> 1)]), (i & 1) ? a1 : a0);
          if (nmixed) {
            const uint64_t lo = (uint64_t)(lane + 32 * i);
            for (int j = 0; j < nmixed; ++j) f = cmul(f, conj_if(mx[j], parity64(M[d.mixed_begin + j] & lo)));
          }
          v[k] = to_mem(cmul(to_calc(v[k], R()), f));
        }
#pragma unroll
        for (int k = 0; k < 4; ++k) p[lane + 32 * (i0 + k)] = v[k];
      }
    }
    __syncwarp();   // the next chunk rewrites this warp's A, B and MIXED factors
  }
}

static int phase_sm_count() {
  static int sms = 0;
  if (!sms) {
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (sms <= 0) sms = 1;
  }
  return sms;
}

// Host side, outside any stream capture: shared-memory limit and residency.
cudaError_t prepare_phase_pass(PhasePassDesc& d, qs_dtype dt) {
  if (d.nterms > kPhaseMaxTerms || d.nterms - d.mixed_begin > kPhaseMaxMixed) return cudaErrorInvalidValue;
  const size_t smem = phase_smem_bytes(d.nterms, dt);
  const void* fn = dt == QS_C64 ? (const void*)k_phase_pass<float>
                   : d.df ? (const void*)k_phase_pass<dfl> : (const void*)k_phase_pass<double>;
  cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)phase_smem_bytes(kPhaseMaxTerms, dt));
  if (e != cudaSuccess) return e;
  int occ = 0;
  e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, fn, kPhaseThreads, smem);
  if (e != cudaSuccess) return e;
  d.occ = occ > 0 ? occ : 1;
  phase_sm_count();
  return cudaSuccess;
}

cudaError_t launch_phase_pass(void* psi, void* const* psis, int nstates, int n, qs_dtype dt,
                              const DevPhaseTerm* terms, const PhasePassDesc& d, const double* theta,
                              int64_t ntheta, cudaStream_t st) {
  if (n < kPhaseChunkBits || nstates < 1 || d.occ < 1 || d.nterms > kPhaseMaxTerms ||
      d.nterms - d.mixed_begin > kPhaseMaxMixed)
    return cudaErrorInvalidValue;
  const uint64_t chunks = 1ull << (n - kPhaseChunkBits);
  const uint64_t need = (chunks + kPhaseWarps - 1) / kPhaseWarps;
  const uint64_t fill = std::max<uint64_t>(1, (uint64_t)phase_sm_count() * d.occ / (uint64_t)nstates);
  const unsigned gx = (unsigned)std::min(need, fill);
  const size_t smem = phase_smem_bytes(d.nterms, dt);
  if (dt == QS_C64)
    k_phase_pass<float><<<dim3(gx, nstates), kPhaseThreads, smem, st>>>(psi, psis, n, terms, d, theta, ntheta);
  else if (d.df)
    k_phase_pass<dfl><<<dim3(gx, nstates), kPhaseThreads, smem, st>>>(psi, psis, n, terms, d, theta, ntheta);
  else
    k_phase_pass<double><<<dim3(gx, nstates), kPhaseThreads, smem, st>>>(psi, psis, n, terms, d, theta, ntheta);
  note_launch();
  return cudaGetLastError();
}

}  // namespace qs
