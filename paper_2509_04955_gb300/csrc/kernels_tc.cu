// Tensor-core pass: one dense 6-qubit block (64 x 64 complex) applied to a
// complex64 state with tcgen05 MMAs, FP32 accumulation in tensor memory.
//
// A fused block of Section 3.4 acting on qubits Q (|Q| = 6) is the complex
// matrix product psi'[r, :] = U psi[r, :] over the 2^(n-6) "rows" r (the other
// bits). Written over reals with interleaved (re, im) columns it is a real GEMM
//   D[r][2c'+b] = sum_{c,a} A[r][2c+a] * W[2c+a][2c'+b],   K = N = 128,
// with W[2c][2c'] = Re U[c'][c], W[2c+1][2c'] = -Im U[c'][c],
//      W[2c][2c'+1] = Im U[c'][c], W[2c+1][2c'+1] = Re U[c'][c].
// One persistent CTA per SM (256 threads, two per row) walks a contiguous
// range of tiles of 128 rows: the 7 lowest qubits outside Q are the row bits (a warp's 32 rows are
// consecutive amplitudes when Q holds no low qubit, so its loads coalesce),
// Q the column bits. Software pipeline per tile i: the loads of tile i+1 are
// issued into registers, tile i's accumulator is read back from tensor memory
// and stored, then tile i+1 is converted into the other A buffer and its MMAs
// are issued into the other accumulator (A operands and accumulators are
// double-buffered, 256 TMEM columns).
// Precision: A and W are split into bf16 hi + lo parts; bf16x3 accumulates
// lo*hi + hi*lo + hi*hi (about 16 significant bits per product), bf16 takes
// hi*hi only. Operands sit in shared memory in the K-major 128-byte-swizzled
// layout; the W image (hi and lo, 64 KiB) is prepared on the host and stays
// resident in shared memory for all tiles of the CTA.
//
// Every wait on an mbarrier is bounded: on timeout the kernel sets *err,
// stops taking tiles, frees its tensor memory and returns.
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include "qs_internal.h"

namespace qs {

constexpr int kTcAtomBytes = 16384;            // 128 rows x 128 B (64 bf16 of K)
constexpr int kTcOperandBytes = 2 * kTcAtomBytes;   // K = 128 bf16 per row
constexpr uint32_t kTcSpinLimit = 1u << 26;

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}

// Shared-memory matrix descriptor: K-major, 128-byte swizzle, 8-row groups
// 1024 B apart (stride byte offset), version 1 (bits 46-48).
__device__ __forceinline__ uint64_t smem_desc(uint32_t addr) {
  uint64_t d = 0;
  d |= (uint64_t)((addr >> 4) & 0x3FFF);
  d |= (uint64_t)1 << 16;                 // leading byte offset (unused with 128B swizzle)
  d |= (uint64_t)(1024 >> 4) << 32;       // stride byte offset
  d |= (uint64_t)1 << 46;                 // descriptor version
  d |= (uint64_t)2 << 61;                 // SWIZZLE_128B
  return d;
}

// Instruction descriptor: kind::f16 with BF16 A/B, FP32 D, both K-major, M = 128, N = 128.
constexpr uint32_t kIdesc = (1u << 4) | (1u << 7) | (1u << 10) | ((128u >> 3) << 17) | ((128u >> 4) << 24);

__device__ __forceinline__ void mma_bf16(uint32_t tmem, uint64_t a, uint64_t b, uint32_t acc) {
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "setp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(tmem),
      "l"(a), "l"(b), "r"(kIdesc), "r"(acc));
}

__device__ __forceinline__ void mma_commit(uint32_t mbar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(mbar)
               : "memory");
}

__device__ __forceinline__ bool mbar_wait(uint32_t mbar, uint32_t phase) {
  for (uint32_t it = 0; it < kTcSpinLimit; ++it) {
    uint32_t done;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}\n"
        : "=r"(done)
        : "r"(mbar), "r"(phase)
        : "memory");
    if (done) return true;
  }
  return false;
}

__device__ __forceinline__ void tmem_ld32(uint32_t taddr, float* v) {
  uint32_t r[32];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
      "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
        "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]),
        "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]),
        "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int i = 0; i < 32; ++i) v[i] = __uint_as_float(r[i]);
}

// Byte offset of bf16 element (row, k) in a K-major SW128 operand of 128 rows.
__device__ __forceinline__ uint32_t sw128_offset(uint32_t row, uint32_t k) {
  const uint32_t atom = k >> 6, kk = k & 63;
  const uint32_t chunk = (kk >> 3) ^ (row & 7);
  return atom * kTcAtomBytes + row * 128 + chunk * 16 + (kk & 7) * 2;
}

// Issues the 24 (bf16x3) or 8 (bf16) MMAs of one tile: D = A * W^T over K = 128.
template <int PREC>
__device__ __forceinline__ void issue_tile_mmas(uint32_t tmem_d, uint32_t ah, uint32_t al, uint32_t wh, uint32_t wl) {
  uint32_t acc = 0;
  if (PREC == 3) {
#pragma unroll
    for (int ks = 0; ks < 8; ++ks) {     // lo * hi
      const uint32_t o = (ks >> 2) * kTcAtomBytes + (ks & 3) * 32;
      mma_bf16(tmem_d, smem_desc(al + o), smem_desc(wh + o), acc);
      acc = 1;
    }
#pragma unroll
    for (int ks = 0; ks < 8; ++ks) {     // hi * lo
      const uint32_t o = (ks >> 2) * kTcAtomBytes + (ks & 3) * 32;
      mma_bf16(tmem_d, smem_desc(ah + o), smem_desc(wl + o), 1);
    }
  }
#pragma unroll
  for (int ks = 0; ks < 8; ++ks) {       // hi * hi
    const uint32_t o = (ks >> 2) * kTcAtomBytes + (ks & 3) * 32;
    mma_bf16(tmem_d, smem_desc(ah + o), smem_desc(wh + o), acc);
    acc = 1;
  }
}

// 256 threads: thread (warp w, lane) owns row r = 32 (w % 4) + lane and
// column half h = w / 4 (complex columns 32h .. 32h + 31 = K atom h).
constexpr int kTc2Threads = 256;

template <int PREC, bool MULTI>
__global__ void __launch_bounds__(kTc2Threads, 1)
    k_tc_block(float2* __restrict__ psi0, void* const* __restrict__ psis, TcPassDesc p,
               const uint4* __restrict__ wimg, int64_t wstride16, int lg_tiles1, uint64_t ntiles,
               int* __restrict__ err) {
  // ntiles = 2^lg_tiles1 x states; tile index t covers state t >> lg_tiles1 (batched execution).
  // Each CTA takes a contiguous range of tiles; with per-state W images
  // (wstride16 = uint4 stride, non-zero for parametric blocks) the image is
  // reloaded when the range crosses into the next state.
  const uint64_t tmask1 = (1ull << lg_tiles1) - 1;
  // tile order: strided over the grid (t = blockIdx.x + i * gridDim.x) when one
  // W image serves every tile; contiguous per CTA when W is per state
  const uint64_t chunk = (ntiles + gridDim.x - 1) / gridDim.x;
  const bool contig = MULTI && wstride16 != 0;
  const uint64_t ts = contig ? 1 : gridDim.x;
  const uint64_t t_begin = contig ? (uint64_t)blockIdx.x * chunk : blockIdx.x;
  const uint64_t t_end = contig ? (t_begin + chunk < ntiles ? t_begin + chunk : ntiles) : ntiles;
  extern __shared__ __align__(1024) unsigned char tc_smem_raw[];
  unsigned char* smem = (unsigned char*)(((uintptr_t)tc_smem_raw + 1023) & ~(uintptr_t)1023);
  // A operands double-buffered: buffer b at smem + b * 2 * kTcOperandBytes (hi, then lo)
  unsigned char* W_hi = smem + 4 * kTcOperandBytes;
  unsigned char* W_lo = W_hi + kTcOperandBytes;
  uint64_t* coff = (uint64_t*)(W_lo + kTcOperandBytes);   // 64 global column offsets
  uint64_t* mbar = coff + 64;                             // two barriers
  uint32_t* tmem_slot = (uint32_t*)(mbar + 2);
  __shared__ int s_abort;

  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int row = (warp & 3) * 32 + lane, half = warp >> 2;
  uint64_t wstate = t_begin >> lg_tiles1;   // state whose W image is resident
  auto load_w = [&](uint64_t state) {
    const uint4* src = wimg + (int64_t)state * wstride16;
    for (int i = tid; i < 2 * kTcOperandBytes / 16; i += kTc2Threads) ((uint4*)W_hi)[i] = src[i];
  };
  load_w(contig ? wstate : 0);
  if (tid < 64) {
    uint64_t o = 0;
    for (int b = 0; b < 6; ++b) o |= (uint64_t)((tid >> b) & 1) << p.col[b];
    coff[tid] = o;
  }
  if (tid == 0) {
    s_abort = 0;
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(mbar)) : "memory");
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(mbar + 1)) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], 256;" ::"r"(smem_u32(tmem_slot))
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = *tmem_slot;
  const uint32_t smem_a = smem_u32(smem), wh = smem_u32(W_hi), wl = smem_u32(W_lo);
  uint64_t roff = 0;
  for (int b = 0; b < 7; ++b) roff |= (uint64_t)((row >> b) & 1) << p.row[b];
  const uint64_t* hcoff = coff + half * 32;   // this thread's 32 column offsets (shared memory)
  uint32_t phase[2] = {0, 0};
  float2 va[32], vb[32];   // two tiles in flight: register double buffer

  auto state_of = [&](uint64_t t) -> float2* {
    if constexpr (MULTI) return (float2*)psis[t >> lg_tiles1];
    else return psi0;
  };
  auto load = [&](float2 (&v)[32], uint64_t t) {
    const float2* __restrict__ psi = state_of(t);
    const uint64_t rb = insert_zero_bits(t & tmask1, p.tile, 13) | roff;
#pragma unroll
    for (int c = 0; c < 32; ++c) v[c] = psi[rb | hcoff[c]];
  };
  // v -> bf16 hi / lo, swizzled K-major, K atom `half` of A buffer b
  auto convert = [&](const float2 (&v)[32], int b) {
    unsigned char* a_hi = smem + b * 2 * kTcOperandBytes + half * kTcAtomBytes;
    unsigned char* a_lo = a_hi + kTcOperandBytes;
#pragma unroll
    for (int j = 0; j < 8; ++j) {
      uint32_t hi[4], lo[4];
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const float2 a = v[4 * j + q];
        const __nv_bfloat162 h = __floats2bfloat162_rn(a.x, a.y);
        const float2 hf = __bfloat1622float2(h);
        const __nv_bfloat162 l = __floats2bfloat162_rn(a.x - hf.x, a.y - hf.y);
        hi[q] = *(const uint32_t*)&h;
        lo[q] = *(const uint32_t*)&l;
      }
      const uint32_t off = row * 128 + ((j ^ (row & 7)) << 4);
      *(uint4*)(a_hi + off) = make_uint4(hi[0], hi[1], hi[2], hi[3]);
      if (PREC == 3) *(uint4*)(a_lo + off) = make_uint4(lo[0], lo[1], lo[2], lo[3]);
    }
  };
  auto issue = [&](int b) {
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    if (tid == 0) {
      const uint32_t ah = smem_a + b * 2 * kTcOperandBytes;
      issue_tile_mmas<PREC>(tmem + b * 128, ah, ah + kTcOperandBytes, wh, wl);
      mma_commit(smem_u32(mbar + b));
    }
  };
  // one pipeline step for tile t (MMAs issued into accumulator b): `nxt`
  // holds tile t + g (in flight), `nn` receives tile t + 2g.
  auto step = [&](uint64_t t, int b, float2 (&nxt)[32], float2 (&nn)[32]) -> bool {
    if (t + 2 * ts < t_end) load(nn, t + 2 * ts);
    if (tid == 0 && !mbar_wait(smem_u32(mbar + b), phase[b])) {
      atomicExch(err, 1);
      s_abort = 1;
    }
    phase[b] ^= 1;
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    if (s_abort) return false;
    {   // epilogue: TMEM lane `row`, columns 64 half .. 64 half + 63 of accumulator b
      float2* __restrict__ psi = state_of(t);
      const uint64_t rb = insert_zero_bits(t & tmask1, p.tile, 13) | roff;
      const uint32_t taddr = tmem + b * 128 + half * 64 + ((uint32_t)((warp & 3) * 32) << 16);
#pragma unroll
      for (int chunk = 0; chunk < 2; ++chunk) {
        float o[32];
        tmem_ld32(taddr + chunk * 32, o);
#pragma unroll
        for (int q = 0; q < 16; ++q) psi[rb | hcoff[chunk * 16 + q]] = make_float2(o[2 * q], o[2 * q + 1]);
      }
    }
    if (t + ts < t_end) {
      if (contig && ((t + ts) >> lg_tiles1) != wstate) {   // previous MMAs are complete
        wstate = (t + ts) >> lg_tiles1;
        load_w(wstate);
      }
      convert(nxt, b ^ 1);
      issue(b ^ 1);
    }
    return true;
  };

  uint64_t t = t_begin;
  int b = 0;
  if (t < t_end) {
    load(va, t);
    convert(va, 0);
    issue(0);
    if (t + ts < t_end) load(va, t + ts);
  }
  while (t < t_end) {
    if (!step(t, b, va, vb)) break;
    t += ts;
    b ^= 1;
    if (t >= t_end) break;
    if (!step(t, b, vb, va)) break;
    t += ts;
    b ^= 1;
  }
  // after a timeout, give outstanding MMAs a second bounded wait before
  // their tensor memory is released
  if (tid == 0 && s_abort) mbar_wait(smem_u32(mbar + b), phase[b] ^ 1);   // the MMAs that timed out
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (warp == 0)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, 256;" ::"r"(tmem) : "memory");
}

size_t tc_smem_bytes() { return 6 * (size_t)kTcOperandBytes + 64 * 8 + 32 + 1024; }

static bool g_tc_ready = false;
static int g_tc_sms = 0;

// Host-side set-up (outside any stream capture): shared-memory attribute of
// both precision instances and the SM count.
cudaError_t prepare_tc_pass() {
  if (g_tc_ready) return cudaSuccess;
  const int smem = (int)tc_smem_bytes();
  cudaError_t e = cudaFuncSetAttribute(k_tc_block<3, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
  if (e == cudaSuccess) e = cudaFuncSetAttribute(k_tc_block<1, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
  if (e == cudaSuccess) e = cudaFuncSetAttribute(k_tc_block<3, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
  if (e == cudaSuccess) e = cudaFuncSetAttribute(k_tc_block<1, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
  if (e != cudaSuccess) return e;
  int dev = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&g_tc_sms, cudaDevAttrMultiProcessorCount, dev);
  g_tc_ready = true;
  return cudaSuccess;
}

cudaError_t launch_tc_pass_batched(void* psi, void* const* psis, int nstates, int64_t wstride, int n,
                                   const TcPassDesc& p, const void* wimg, int prec, int* err, cudaStream_t st) {
  if (!g_tc_ready) return cudaErrorInvalidConfiguration;   // not prepared
  const size_t smem = tc_smem_bytes();
  const int sms = g_tc_sms;
  const uint64_t ntiles1 = 1ull << (n - 13), ntiles = ntiles1 * (uint64_t)nstates;
  const uint64_t grid = ntiles < (uint64_t)sms ? ntiles : (uint64_t)sms;
#define QS_TC_ARGS (float2*)psi, psis, p, (const uint4*)wimg, wstride / 8, n - 13, ntiles, err
  if (psis) {
    if (prec == 3) k_tc_block<3, true><<<(unsigned)grid, kTc2Threads, smem, st>>>(QS_TC_ARGS);
    else k_tc_block<1, true><<<(unsigned)grid, kTc2Threads, smem, st>>>(QS_TC_ARGS);
  } else {
    if (prec == 3) k_tc_block<3, false><<<(unsigned)grid, kTc2Threads, smem, st>>>(QS_TC_ARGS);
    else k_tc_block<1, false><<<(unsigned)grid, kTc2Threads, smem, st>>>(QS_TC_ARGS);
  }
#undef QS_TC_ARGS
  note_launch();
  return cudaGetLastError();
}

cudaError_t launch_tc_pass(void* psi, int n, const TcPassDesc& p, const void* wimg, int prec, int* err,
                           cudaStream_t st) {
  return launch_tc_pass_batched(psi, nullptr, 1, 0, n, p, wimg, prec, err, st);
}

}  // namespace qs
