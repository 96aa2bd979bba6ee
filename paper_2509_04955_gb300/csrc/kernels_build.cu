// Device-side construction of contracted blocks that depend on theta.
//
// A block of Section 3.4 is the ordered product of its member gates (Eq. 7
// for distinct qubits, M2 M1 on one qubit). When members are parametric the
// product changes with every parameter vector, so it is rebuilt here from the
// gate table that k_resolve filled for each batch row: one CTA per (block,
// row); column c of the 2^k x 2^k matrix is e_c pushed through the member
// gates (thread c owns column c), in FP64. Dense blocks are written to the
// block table, diagonal blocks as their diagonal, tensor-core blocks as the
// bf16 hi / lo W image in the K-major 128-byte-swizzled layout the
// tensor-core pass loads (real embedding W[2c+a][2c'+b] of U[c'][c]).
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include "qs_internal.h"

namespace qs {

constexpr int kBuildThreads = 128;

__device__ __forceinline__ double2 zmul(double2 a, double2 b) {
  return make_double2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
__device__ __forceinline__ double2 zadd(double2 a, double2 b) { return make_double2(a.x + b.x, a.y + b.y); }

__global__ void __launch_bounds__(kBuildThreads) k_build_blocks(const DevBlock* __restrict__ blocks,
                                                                 const DevMember* __restrict__ mem,
                                                                 const double2* __restrict__ gtab, int64_t gstride,
                                                                 double2* __restrict__ btab, int64_t bstride,
                                                                 uint16_t* __restrict__ wimg, int64_t wstride) {
  extern __shared__ double2 M[];   // D x D, row-major
  const DevBlock blk = blocks[blockIdx.x];
  const int row = blockIdx.y;
  const int D = 1 << blk.k;
  const double2* gt = gtab + (int64_t)row * gstride;
  for (int i = threadIdx.x; i < D * D; i += kBuildThreads)
    M[i] = make_double2((i / D) == (i % D) ? 1.0 : 0.0, 0.0);
  __syncthreads();
  const int c = threadIdx.x;
  if (c < D) {
    for (int mi = blk.mem_begin; mi < blk.mem_end; ++mi) {
      const DevMember g = mem[mi];
      const double2* u = gt + (int64_t)g.gate * 16;
      if (g.nt == 1) {
        const double2 u00 = u[0], u01 = u[1], u10 = u[2], u11 = u[3];
        const int tb = 1 << g.t0;
        for (int i = 0; i < D; ++i) {
          if ((i & tb) || (i & g.cmask) != g.cmask) continue;
          const double2 a0 = M[i * D + c], a1 = M[(i | tb) * D + c];
          M[i * D + c] = zadd(zmul(u00, a0), zmul(u01, a1));
          M[(i | tb) * D + c] = zadd(zmul(u10, a0), zmul(u11, a1));
        }
      } else {
        const int ta = 1 << g.t0, tb = 1 << g.t1;
        for (int i = 0; i < D; ++i) {
          if ((i & (ta | tb)) || (i & g.cmask) != g.cmask) continue;
          const int idx[4] = {i, i | ta, i | tb, i | ta | tb};
          double2 a[4];
          for (int j = 0; j < 4; ++j) a[j] = M[idx[j] * D + c];
          for (int r = 0; r < 4; ++r) {
            double2 acc = make_double2(0, 0);
            for (int j = 0; j < 4; ++j) acc = zadd(acc, zmul(u[4 * r + j], a[j]));
            M[idx[r] * D + c] = acc;
          }
        }
      }
    }
  }
  __syncthreads();
  if (blk.kind == 0) {
    double2* out = btab + (int64_t)row * bstride + blk.out;
    for (int i = threadIdx.x; i < D * D; i += kBuildThreads) out[i] = M[i];
  } else if (blk.kind == 1) {
    double2* out = btab + (int64_t)row * bstride + blk.out;
    for (int i = threadIdx.x; i < D; i += kBuildThreads) out[i] = M[i * D + i];
  } else {
    uint16_t* img = wimg + (int64_t)row * wstride + blk.out * 32768;
    for (int e = threadIdx.x; e < 128 * 128; e += kBuildThreads) {
      const int nn = e >> 7, k = e & 127;
      const int co = nn >> 1, b = nn & 1, ci = k >> 1, a = k & 1;
      const double2 uv = M[co * 64 + ci];
      const double w = (a == 0) ? (b == 0 ? uv.x : uv.y) : (b == 0 ? -uv.y : uv.x);
      const __nv_bfloat16 hi = __double2bfloat16(w);
      const __nv_bfloat16 lo = __double2bfloat16(w - (double)__bfloat162float(hi));
      const int kk = k & 63;
      const int off = ((k >> 6) * 16384 + nn * 128 + (((kk >> 3) ^ (nn & 7)) << 4) + (kk & 7) * 2) >> 1;
      img[off] = *(const uint16_t*)&hi;
      img[16384 + off] = *(const uint16_t*)&lo;
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
                                int64_t wstride, cudaStream_t st) {
  if (nblocks == 0 || rows == 0) return cudaSuccess;
  if (!g_build_ready) return cudaErrorInvalidConfiguration;   // not prepared
  const int smem = 64 * 64 * (int)sizeof(double2);
  k_build_blocks<<<dim3(nblocks, rows), kBuildThreads, smem, st>>>(blocks, mem, gtab, gstride, btab, bstride, wimg,
                                                                   wstride);
  note_launch();
  return cudaGetLastError();
}

}  // namespace qs
