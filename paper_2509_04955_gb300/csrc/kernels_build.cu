// Device-side construction of contracted blocks that depend on theta.
//
// A block of Section 3.4 is the ordered product of its member gates (Eq. 7
// for distinct qubits, M2 M1 on one qubit). When members are parametric the
// product changes with every parameter vector, so it is rebuilt here from the
// gate table that k_resolve filled for each batch row: one CTA per (block,
// row); column c of the 2^k x 2^k matrix is e_c pushed through the member
// gates, in FP64. Dense blocks are written to the
// block table, diagonal blocks as their diagonal, tensor-core blocks as the
// 16-bit hi / lo W image (complex64 pass) or the five fp16 digit planes
// (complex128 pass) in the K-major 128-byte-swizzled layout the tensor-core
// pass loads (real embedding W[2c+a][2c'+b] of U[c'][c]).
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>

#include "qs_internal.h"

namespace qs {

constexpr int kBuildThreads = 256;

__device__ __forceinline__ double2 zmul(double2 a, double2 b) {
  return make_double2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
__device__ __forceinline__ double2 zadd(double2 a, double2 b) { return make_double2(a.x + b.x, a.y + b.y); }
// p a + q b with real p, q
__device__ __forceinline__ double2 rmix2(double p, double2 a, double q, double2 b) {
  return make_double2(p * a.x + q * b.x, p * a.y + q * b.y);
}
// p a + i q b with real p, q
__device__ __forceinline__ double2 imix2(double p, double2 a, double q, double2 b) {
  return make_double2(p * a.x - q * b.y, p * a.y + q * b.x);
}

// Work items of a gate: (pair or quad index, column), column fastest so a
// warp touches consecutive matrix entries. Each member's structure (its form:
// a permutation, a diagonal, real or RX-like entries) is fixed for every
// theta, so only the arithmetic the form needs is done; all of it in FP64.
__global__ void __launch_bounds__(kBuildThreads) k_build_blocks(const DevBlock* __restrict__ blocks,
                                                                 const DevMember* __restrict__ mem,
                                                                 const double2* __restrict__ gtab, int64_t gstride,
                                                                 double2* __restrict__ btab, int64_t bstride,
                                                                 uint16_t* __restrict__ wimg, int64_t wstride,
                                                                 int wmode, int64_t wpass) {
  extern __shared__ double2 M[];   // D x D, row-major: M[r * D + c]
  const DevBlock blk = blocks[blockIdx.x];
  const int row = blockIdx.y;
  const int k = blk.k, D = 1 << k;
  const double2* gt = gtab + (int64_t)row * gstride;
  for (int i = threadIdx.x; i < D * D; i += kBuildThreads)
    M[i] = make_double2((i >> k) == (i & (D - 1)) ? 1.0 : 0.0, 0.0);
  __syncthreads();
  for (int mi = blk.mem_begin; mi < blk.mem_end; ++mi) {
    const DevMember g = mem[mi];
    const double2* u = gt + (int64_t)g.gate * 16;
    if (g.nt == 1) {
      const int t0 = g.t0, tb = 1 << t0;
      const double2 u00 = u[0], u01 = u[1], u10 = u[2], u11 = u[3];
      const int items = D << (k - 1);   // D / 2 pairs x D columns
      for (int e = threadIdx.x; e < items; e += kBuildThreads) {
        const int c = e & (D - 1), pi = e >> k;
        const int i = ((pi >> t0) << (t0 + 1)) | (pi & (tb - 1));
        if ((i & (int)g.cmask) != (int)g.cmask) continue;
        double2* p0 = M + i * D + c;
        double2* p1 = M + (i | tb) * D + c;
        const double2 a0 = *p0, a1 = *p1;
        switch (g.form) {
          case FORM_X1: *p0 = a1; *p1 = a0; break;
          case FORM_PHASE1: *p1 = zmul(u11, a1); break;
          case FORM_DIAG1: *p0 = zmul(u00, a0); *p1 = zmul(u11, a1); break;
          case FORM_ANTI1: *p0 = zmul(u01, a1); *p1 = zmul(u10, a0); break;
          case FORM_REAL1: *p0 = rmix2(u00.x, a0, u01.x, a1); *p1 = rmix2(u10.x, a0, u11.x, a1); break;
          case FORM_RXLIKE1: *p0 = imix2(u00.x, a0, u01.y, a1); *p1 = imix2(u11.x, a1, u10.y, a0); break;
          default:
            *p0 = zadd(zmul(u00, a0), zmul(u01, a1));
            *p1 = zadd(zmul(u10, a0), zmul(u11, a1));
        }
      }
    } else {
      const int ta = 1 << g.t0, tb = 1 << g.t1;
      const int lo_t = g.t0 < g.t1 ? g.t0 : g.t1, hi_t = g.t0 < g.t1 ? g.t1 : g.t0;
      const int items = D << (k - 2);   // D / 4 quads x D columns
      for (int e = threadIdx.x; e < items; e += kBuildThreads) {
        const int c = e & (D - 1), qi = e >> k;
        int i = ((qi >> lo_t) << (lo_t + 1)) | (qi & ((1 << lo_t) - 1));
        i = ((i >> hi_t) << (hi_t + 1)) | (i & ((1 << hi_t) - 1));
        if ((i & (int)g.cmask) != (int)g.cmask) continue;
        const int idx[4] = {i, i | ta, i | tb, i | ta | tb};
        if (g.form == FORM_SWAP2) {
          const double2 x1 = M[idx[1] * D + c], x2 = M[idx[2] * D + c];
          M[idx[1] * D + c] = x2;
          M[idx[2] * D + c] = x1;
          continue;
        }
        double2 a[4];
#pragma unroll
        for (int j = 0; j < 4; ++j) a[j] = M[idx[j] * D + c];
#pragma unroll
        for (int r = 0; r < 4; ++r) {
          double2 acc = zmul(u[4 * r], a[0]);
#pragma unroll
          for (int j = 1; j < 4; ++j) acc = zadd(acc, zmul(u[4 * r + j], a[j]));
          M[idx[r] * D + c] = acc;
        }
      }
    }
    __syncthreads();
  }
  if (blk.kind == 0) {
    double2* out = btab + (int64_t)row * bstride + blk.out;
    for (int i = threadIdx.x; i < D * D; i += kBuildThreads) out[i] = M[i];
  } else if (blk.kind == 1) {
    double2* out = btab + (int64_t)row * bstride + blk.out;
    for (int i = threadIdx.x; i < D; i += kBuildThreads) out[i] = M[i * D + i];
  } else if (wmode == 2) {
    // complex128 pass (D = 32): digit planes of the real embedding, entry
    // (nn, k) = W[k][nn], w = 2^-8 sum_j g_j 2^(-9 j) with balanced digits of
    // X = rint(w 2^53) (the host's build_w_digits), fp16, K-major 128-byte
    // swizzle, planes g_0 .. g_5
    uint16_t* img = wimg + (int64_t)row * wstride + blk.out * wpass;
    for (int e = threadIdx.x; e < 64 * 64; e += kBuildThreads) {
      const int nn = e >> 6, kk = e & 63;
      const int co = nn >> 1, b = nn & 1, ci = kk >> 1, a = kk & 1;
      const double2 uv = M[co * 32 + ci];
      const double w = a == 0 ? (b == 0 ? uv.x : uv.y) : (b == 0 ? -uv.y : uv.x);
      long long X = __double2ll_rn(w * 9007199254740992.0);   // w 2^53 (exact scaling)
      int g[6];
#pragma unroll
      for (int j = 5; j >= 1; --j) {
        g[j] = (int)(((X + 256) & 511) - 256);
        X = (X - g[j]) / 512;
      }
      g[0] = (int)X;
      const int off = (nn * 128 + (((kk >> 3) ^ (nn & 7)) << 4) + (kk & 7) * 2) >> 1;
#pragma unroll
      for (int j = 0; j < 6; ++j) img[j * 4096 + off] = __half_as_ushort(__int2half_rn(g[j]));
    }
  } else {
    // W image: 16-byte chunks of 8 consecutive k (4 input columns) of output row nn,
    // K atom `atom`, 128-byte swizzle; hi / lo split in FP32 (the product is FP64),
    // fp16 parts when `whalf` (the pass splits the state into fp16), else bf16
    const bool whalf = wmode == 1;
    uint16_t* img = wimg + (int64_t)row * wstride + blk.out * wpass;
    for (int e = threadIdx.x; e < 2048; e += kBuildThreads) {
      const int atom = e >> 10, nn = (e >> 3) & 127, ch = e & 7;
      const int co = nn >> 1, b = nn & 1, ci0 = atom * 32 + ch * 4;
      uint32_t hi[4], lo[4];
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const double2 uv = M[co * 64 + ci0 + q];
        const float ur = (float)uv.x, ui = (float)uv.y;
        const float w0 = b == 0 ? ur : ui, w1 = b == 0 ? -ui : ur;   // W[nn][2 ci], W[nn][2 ci + 1]
        if (whalf) {
          const __half2 h = __floats2half2_rn(w0, w1);
          const float2 hf = __half22float2(h);
          const __half2 l = __floats2half2_rn(w0 - hf.x, w1 - hf.y);
          hi[q] = *(const uint32_t*)&h;
          lo[q] = *(const uint32_t*)&l;
        } else {
          const __nv_bfloat162 h = __floats2bfloat162_rn(w0, w1);
          const float2 hf = __bfloat1622float2(h);
          const __nv_bfloat162 l = __floats2bfloat162_rn(w0 - hf.x, w1 - hf.y);
          hi[q] = *(const uint32_t*)&h;
          lo[q] = *(const uint32_t*)&l;
        }
      }
      const int off = (atom * 16384 + nn * 128 + ((ch ^ (nn & 7)) << 4)) >> 1;   // uint16 units
      *(uint4*)(img + off) = make_uint4(hi[0], hi[1], hi[2], hi[3]);
      *(uint4*)(img + 16384 + off) = make_uint4(lo[0], lo[1], lo[2], lo[3]);
    }
  }
}

static bool g_build_ready = false;

// Host-side set-up (outside any stream capture): 64 KiB of dynamic shared memory.
cudaError_t prepare_build_blocks() {
  if (g_build_ready) return cudaSuccess;
  cudaError_t e = cudaFuncSetAttribute(k_build_blocks, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       64 * 64 * (int)sizeof(double2));
  if (e != cudaSuccess) return e;
  g_build_ready = true;
  return cudaSuccess;
}

cudaError_t launch_build_blocks(const DevBlock* blocks, int nblocks, const DevMember* mem, const double2* gtab,
                                int64_t gstride, int rows, double2* btab, int64_t bstride, uint16_t* wimg,
                                int64_t wstride, int wmode, int64_t wpass, cudaStream_t st) {
  if (nblocks == 0 || rows == 0) return cudaSuccess;
  if (!g_build_ready) return cudaErrorInvalidConfiguration;   // not prepared
  const int smem = 64 * 64 * (int)sizeof(double2);
  k_build_blocks<<<dim3(nblocks, rows), kBuildThreads, smem, st>>>(blocks, mem, gtab, gstride, btab, bstride, wimg,
                                                                   wstride, wmode, wpass);
  note_launch();
  return cudaGetLastError();
}

}  // namespace qs
