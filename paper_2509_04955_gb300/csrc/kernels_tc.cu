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
// Precision (PREC): A and W are split into hi + lo parts and the MMAs
// accumulate lo*hi + hi*lo + hi*hi. PREC 4 (default) splits into fp16: 11 + 11
// significant bits, about 2^-22 relative per product; the amplitudes are first
// multiplied by 2^s, s = min(floor(n / 2), 15) (exact), so that typical
// amplitudes of a 2^n state (about 2^(-n/2)) are not fp16 subnormals while the
// largest possible one (1) stays far below the fp16 maximum, and the outputs
// are multiplied by 2^-s. PREC 3 splits into bf16 (8 + 8 bits, about 2^-16),
// PREC 1 takes bf16 hi*hi only. Operands sit in shared memory in the K-major 128-byte-swizzled
// layout; the W image (hi and lo, 64 KiB) is prepared on the host and stays
// resident in shared memory for all tiles of the CTA.
//
// Every wait on an mbarrier is bounded: on timeout the kernel sets *err,
// stops taking tiles, frees its tensor memory and returns.
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>

#include "qs_internal.h"
#include "tcgen05.cuh"

namespace qs {

constexpr int kTcAtomBytes = 16384;            // 128 rows x 128 B (64 bf16 of K)
constexpr int kTcOperandBytes = 2 * kTcAtomBytes;   // K = 128 bf16 per row

// Instruction descriptor: kind::f16, FP32 D, both operands K-major, M = 128,
// N = 128; A and B both BF16 (PREC 1, 3) or both FP16 (PREC 4).
template <int PREC>
constexpr uint32_t idesc_for() {
  return (1u << 4) | (PREC == 4 ? 0u : ((1u << 7) | (1u << 10))) | ((128u >> 3) << 17) | ((128u >> 4) << 24);
}

template <int PREC>
__device__ __forceinline__ void mma_bf16(uint32_t tmem, uint64_t a, uint64_t b, uint32_t acc) {
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "setp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(tmem),
      "l"(a), "l"(b), "r"(idesc_for<PREC>()), "r"(acc));
}

// hi / lo split of one complex amplitude (scaled by `scale` first for PREC 4),
// packed as two 16-bit values (re low, im high) each.
template <int PREC>
__device__ __forceinline__ void split_amp(float2 a, float scale, uint32_t& hi, uint32_t& lo) {
  if constexpr (PREC == 4) {
    const float x = a.x * scale, y = a.y * scale;
    const __half2 h = __floats2half2_rn(x, y);
    const float2 hf = __half22float2(h);
    const __half2 l = __floats2half2_rn(x - hf.x, y - hf.y);
    hi = *(const uint32_t*)&h;
    lo = *(const uint32_t*)&l;
  } else {
    const __nv_bfloat162 h = __floats2bfloat162_rn(a.x, a.y);
    const float2 hf = __bfloat1622float2(h);
    const __nv_bfloat162 l = __floats2bfloat162_rn(a.x - hf.x, a.y - hf.y);
    hi = *(const uint32_t*)&h;
    lo = *(const uint32_t*)&l;
  }
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
  if (PREC >= 3) {
#pragma unroll
    for (int ks = 0; ks < 8; ++ks) {     // lo * hi
      const uint32_t o = (ks >> 2) * kTcAtomBytes + (ks & 3) * 32;
      mma_bf16<PREC>(tmem_d, smem_desc(al + o), smem_desc(wh + o), acc);
      acc = 1;
    }
#pragma unroll
    for (int ks = 0; ks < 8; ++ks) {     // hi * lo
      const uint32_t o = (ks >> 2) * kTcAtomBytes + (ks & 3) * 32;
      mma_bf16<PREC>(tmem_d, smem_desc(ah + o), smem_desc(wl + o), 1);
    }
  }
#pragma unroll
  for (int ks = 0; ks < 8; ++ks) {       // hi * hi
    const uint32_t o = (ks >> 2) * kTcAtomBytes + (ks & 3) * 32;
    mma_bf16<PREC>(tmem_d, smem_desc(ah + o), smem_desc(wh + o), acc);
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
               float ascale, int* __restrict__ err) {
  // ascale: factor applied to the amplitudes before the fp16 split (PREC 4), undone on output
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
  // a trailing CTA can get an empty range that starts past the last state
  if (t_begin < t_end) load_w(contig ? wstate : 0);
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
      for (int q = 0; q < 4; ++q) split_amp<PREC>(v[4 * j + q], ascale, hi[q], lo[q]);
      const uint32_t off = row * 128 + ((j ^ (row & 7)) << 4);
      *(uint4*)(a_hi + off) = make_uint4(hi[0], hi[1], hi[2], hi[3]);
      if (PREC >= 3) *(uint4*)(a_lo + off) = make_uint4(lo[0], lo[1], lo[2], lo[3]);
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
        const float inv = 1.0f / ascale;   // a power of two: exact
#pragma unroll
        for (int q = 0; q < 16; ++q)
          psi[rb | hcoff[chunk * 16 + q]] = make_float2(o[2 * q] * inv, o[2 * q + 1] * inv);
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

// ---------------------------------------------------------------------------
// Bulk-copy pipeline (single state). The register-staged kernel above reads
// and writes the state with 8-byte accesses spread over the 128 rows of a
// tile; its loads then reach about 0.8 of the copy bandwidth. Here a producer
// warp moves each tile into shared memory with cp.async.bulk: the tile is a
// set of 2^(13-p) runs of 2^p contiguous amplitudes (p >= 7: every qubit
// below the 7th row qubit belongs to the tile), so every copy is at least
// 1 KiB long and contiguous. Two landing slots of 64 KiB keep one tile in
// flight while the previous one is converted.
//   smem:  slot 0 | slot 1 | W hi | W lo | run/column tables | barriers
//   TMEM:  A buffers 2 x (hi 64 + lo 64 columns), accumulators 2 x 128
// The A operand (bf16 hi/lo of the tile, rows in lanes, K packed two per
// column) lives in tensor memory and is written with tcgen05.st, which frees
// the shared memory for the landing slots; W stays the smem B operand.
// Warps 0-7 convert (slot -> TMEM A), warps 8-15 drain (TMEM D -> HBM), one
// thread per (row, column half) in each group; warp 16 issues the bulk
// copies, warp 17 the MMAs. Converting and draining run concurrently: a
// tile's slot is released as soon as it is converted, its accumulator as
// soon as it is read, and the epilogue stores straight from registers. The
// global offset of a tile is looked up byte by byte in tables built once per
// CTA.
//
// Slot reads: element (row, c) sits at tile-local index lambda = the
// row and column bits deposited at their positions among the 13 tile qubits
// (ascending). A warp's 32 rows read one column at a time (16-column chunks:
// bits 0-3 of c vary inside the thread); when block qubits
// lie on qubits 0-3 (the low lambda bits, i.e. the shared-memory bank bits of
// an 8-byte element) all lanes would hit the same banks, so each lane reads its
// columns in an order XORed with phi(lane), built from lane bits whose row
// qubits are >= 4, and restores the natural order in registers afterwards.

constexpr int kTcbComputeWarps = 16;                     // 4 per TMEM lane quadrant
constexpr int kTcbThreads = (kTcbComputeWarps + 2) * 32;  // + producer warp + MMA warp
constexpr int kTcbSlotBytes = 65536;
constexpr uint32_t kTcbTmemCols = 512;

template <int PREC>
__device__ __forceinline__ void mma_bf16_tmem_a(uint32_t tmem_d, uint32_t tmem_a, uint64_t b, uint32_t acc) {
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "setp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], [%1], %2, %3, p;\n\t}\n" ::"r"(tmem_d),
      "r"(tmem_a), "l"(b), "r"(idesc_for<PREC>()), "r"(acc));
}

// Issues the MMAs of one tile with A in tensor memory: D = A * W^T, K = 128.
template <int PREC>
__device__ __forceinline__ void issue_tile_mmas_ta(uint32_t tmem_d, uint32_t a_hi, uint32_t wh, uint32_t wl) {
  const uint32_t a_lo = a_hi + 64;
  uint32_t acc = 0;
  if (PREC >= 3) {
#pragma unroll
    for (int ks = 0; ks < 8; ++ks) {     // lo * hi
      const uint32_t o = (ks >> 2) * kTcAtomBytes + (ks & 3) * 32;
      mma_bf16_tmem_a<PREC>(tmem_d, a_lo + ks * 8, smem_desc(wh + o), acc);
      acc = 1;
    }
#pragma unroll
    for (int ks = 0; ks < 8; ++ks) {     // hi * lo
      const uint32_t o = (ks >> 2) * kTcAtomBytes + (ks & 3) * 32;
      mma_bf16_tmem_a<PREC>(tmem_d, a_hi + ks * 8, smem_desc(wl + o), 1);
    }
  }
#pragma unroll
  for (int ks = 0; ks < 8; ++ks) {       // hi * hi
    const uint32_t o = (ks >> 2) * kTcAtomBytes + (ks & 3) * 32;
    mma_bf16_tmem_a<PREC>(tmem_d, a_hi + ks * 8, smem_desc(wh + o), acc);
    acc = 1;
  }
}

// Conditional swap of v[j] and v[j ^ (1 << B)] for every j with bit B clear.
template <int B>
__device__ __forceinline__ void xor_stage(float2 (&v)[16], bool on) {
#pragma unroll
  for (int j = 0; j < 16; ++j) {
    if (j & (1 << B)) continue;
    const float2 a = v[j], b = v[j | (1 << B)];
    v[j] = on ? b : a;
    v[j | (1 << B)] = on ? a : b;
  }
}

// Batched execution (MULTI): tile index tt covers state tt >> lg_tiles1 of
// `psis`; with per-state W images (wstride16 != 0, blocks rebuilt from each
// state's theta) every CTA takes a contiguous range of tiles and the producer
// reloads W by bulk copy when the range crosses into the next state, once the
// MMAs of the previous tile have completed.
// Exchange of in-thread bit J (slot index) with lane bit M: the lane with
// bit M clear keeps its slots with bit J clear and receives, into the slots
// with bit J set, its partner's slots with bit J clear; the partner the reverse.
template <int J, int M>
__device__ __forceinline__ void xchg_stage(float2 (&v)[16], bool up) {
#pragma unroll
  for (int q = 0; q < 16; ++q) {
    if (q & (1 << J)) continue;
    const int q1 = q | (1 << J);
    const float2 send = up ? v[q] : v[q1];
    float2 recv;
    recv.x = __shfl_xor_sync(0xffffffffu, send.x, 1 << M);
    recv.y = __shfl_xor_sync(0xffffffffu, send.y, 1 << M);
    if (up) v[q] = recv;
    else v[q1] = recv;
  }
}

template <int PREC, bool MULTI>
__global__ void __launch_bounds__(kTcbThreads, 1)
    k_tc_bulk(float2* __restrict__ psi0, void* const* __restrict__ psis, TcPassDesc p,
              const uint4* __restrict__ wimg, int64_t wstride16, int lg_tiles1, uint64_t ntiles,
              float ascale, int* __restrict__ err, uint32_t spin) {
  // ascale: factor applied to the amplitudes before the fp16 split (PREC 4), undone on output.
  // spin: polls allowed per pipeline wait; when one runs out the CTA records the
  // error and stops, and the waits for its copies and MMAs already in flight
  // use the default bound (kTcSpinLimit), so it never exits with them pending.
  extern __shared__ __align__(1024) unsigned char tcb_smem_raw[];
  unsigned char* smem = (unsigned char*)(((uintptr_t)tcb_smem_raw + 1023) & ~(uintptr_t)1023);
  unsigned char* slots = smem;                                   // 2 x 64 KiB
  unsigned char* W_hi = smem + 2 * kTcbSlotBytes;
  unsigned char* W_lo = W_hi + kTcOperandBytes;
  uint64_t* tbase = (uint64_t*)(W_lo + kTcOperandBytes);        // 4 x 256: tile number byte k -> offset
  uint64_t* runoff = tbase + 4 * 256;                            // 64: global offset of run j
  uint64_t* coff = runoff + 64;                                  // 64: global offset of column c
  uint32_t* lamcol = (uint32_t*)(coff + 64);                     // 64: tile-local index of column c
  int32_t* qpos = (int32_t*)(lamcol + 64);                       // tile[13], row[7], col[6], p, pad
  uint64_t* bar = (uint64_t*)(qpos + 28);   // full[2] empty[2] afull[2] mdone[2] dfree[2] wfull wfree
  uint32_t* tmem_slot = (uint32_t*)(bar + 12);
  __shared__ int s_abort;

  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  int32_t* s_tile = qpos;
  int32_t* s_row = qpos + 13;
  int32_t* s_col = qpos + 20;
  if (tid == 0) {
    for (int k = 0; k < 13; ++k) s_tile[k] = p.tile[k];
    for (int k = 0; k < 7; ++k) s_row[k] = p.row[k];
    for (int k = 0; k < 6; ++k) s_col[k] = p.col[k];
    int pp = 0;
    while (pp < 13 && p.tile[pp] == pp) ++pp;
    qpos[26] = pp;
    s_abort = 0;
    for (int i = 0; i < 12; ++i)   // full/mdone/wfull/wfree: 1 arrival; empty/afull/dfree: one per warp of a group
      asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar + i)),
                   "r"((i >= 2 && i != 6 && i != 7 && i < 10) ? kTcbComputeWarps / 2 : 1));
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  // tile sequence of this CTA: tt = t_begin + i * tstep, i < my
  const uint64_t tmask1 = (1ull << lg_tiles1) - 1;
  const bool contig = MULTI && wstride16 != 0;
  const uint64_t chunk_t = (ntiles + gridDim.x - 1) / gridDim.x;
  const uint64_t t_begin = contig ? (uint64_t)blockIdx.x * chunk_t : blockIdx.x;
  const uint64_t tstep = contig ? 1 : gridDim.x;
  const uint64_t t_end = contig ? (t_begin + chunk_t < ntiles ? t_begin + chunk_t : ntiles) : ntiles;
  const uint64_t my = t_begin < t_end ? (t_end - t_begin + tstep - 1) / tstep : 0;
  if (my > 0) {   // a trailing CTA can get an empty range that starts past the last state
    const uint4* w0 = wimg + (contig ? (int64_t)(t_begin >> lg_tiles1) * wstride16 : 0);
    for (int i = tid; i < 2 * kTcOperandBytes / 16; i += kTcbThreads) ((uint4*)W_hi)[i] = w0[i];
  }
  __syncthreads();
  const int pr = qpos[26];            // log2 of the run length in amplitudes (7..13)
  const int nruns = 1 << (13 - pr);
  // lambda(q) = position of qubit q among the 13 tile qubits (ascending)
  auto lam_of = [&](int q) {
    int l = 0;
    while (l < 12 && s_tile[l] != q) ++l;
    return l;
  };
  for (int e = tid; e < 4 * 256; e += kTcbThreads) {
    uint64_t x = (uint64_t)(e & 255) << (8 * (e >> 8));
    for (int k = 0; k < 13; ++k) {
      const int q = s_tile[k];
      x = ((x >> q) << (q + 1)) | (x & ((1ull << q) - 1));
    }
    tbase[e] = x;
  }
  if (tid < 64) {
    uint64_t o = 0;
    uint32_t lc = 0;
    for (int b = 0; b < 6; ++b) {
      o |= (uint64_t)((tid >> b) & 1) << s_col[b];
      lc |= (uint32_t)((tid >> b) & 1) << lam_of(s_col[b]);
    }
    coff[tid] = o;
    lamcol[tid] = lc;
    if (tid < nruns) {
      uint64_t r = 0;
      for (int b = 0; b < 13 - pr; ++b) r |= (uint64_t)((tid >> b) & 1) << s_tile[pr + b];
      runoff[tid] = r;
    }
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                 "r"(kTcbTmemCols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");   // W is read by the MMA (async proxy)
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = *tmem_slot;
  uint64_t* full = bar;
  uint64_t* empty = bar + 2;
  uint64_t* afull = bar + 4;
  uint64_t* mdone = bar + 6;
  uint64_t* dfree = bar + 8;
  uint64_t* wfull = bar + 10;
  uint64_t* wfree = bar + 11;   // completes when the MMAs on a state's W image are done
  auto tile_of = [&](uint64_t i) -> uint64_t { return t_begin + i * tstep; };
  auto state_ptr = [&](uint64_t tt) -> float2* {
    if constexpr (MULTI) return (float2*)psis[tt >> lg_tiles1];
    else return psi0;
  };
  // does tile i start a new state (W image reload)?
  auto new_state = [&](uint64_t i) -> bool {
    return contig && i > 0 && (tile_of(i) >> lg_tiles1) != (tile_of(i - 1) >> lg_tiles1);
  };
  auto fail = [&](int code) {
    atomicExch(err, code);
    *(volatile int*)&s_abort = 1;
  };
  // global offset of tile t's amplitude with tile-local bits all zero
  auto tile_base = [&](uint64_t t) -> uint64_t {
    return tbase[t & 255] | tbase[256 + ((t >> 8) & 255)] | tbase[512 + ((t >> 16) & 255)] |
           tbase[768 + ((t >> 24) & 255)];
  };

  if (warp == kTcbComputeWarps) {
    // ---------------- producer: bulk copies of tile runs into the slots
    const uint32_t runb = 8u << pr;
    uint64_t i = 0, w_issued = 0;
    for (; i < my; ++i) {
      if (__any_sync(0xffffffffu, *(volatile int*)&s_abort)) break;
      const int s = (int)(i & 1);
      if (i >= 2 && !mbar_wait_warp(smem_u32(empty + s), (uint32_t)(((i >> 1) - 1) & 1), spin)) {
        if (lane == 0) fail(1);
        break;
      }
      if (lane == 0)
        asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(full + s)),
                     "r"((uint32_t)kTcbSlotBytes)
                     : "memory");
      __syncwarp();
      const uint64_t tt = tile_of(i);
      const float2* src = state_ptr(tt) + tile_base(tt & tmask1);
      for (int j = lane; j < nruns; j += 32)
        asm volatile(
            "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                smem_u32(slots + s * kTcbSlotBytes + j * runb)),
            "l"(src + runoff[j]), "r"(runb), "r"(smem_u32(full + s))
            : "memory");
      if (new_state(i)) {
        // W of the next state, once the MMAs of tile i - 1 (the last on the old W) are
        // done: the MMA thread commits `wfree` after them. (The accumulator barriers
        // cannot tell: the producer may be up to three tiles ahead of the MMAs, and a
        // parity wait is exact only within one phase.) wfree completes once per state
        // boundary and its next completion needs this reload, so phase w_issued is
        // the one to wait for.
        if (!mbar_wait_warp(smem_u32(wfree), (uint32_t)(w_issued & 1), spin)) {
          if (lane == 0) fail(1);
          ++i;   // tile i's copies are in flight
          break;
        }
        if (lane == 0) {
          asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(wfull)),
                       "r"((uint32_t)(2 * kTcOperandBytes))
                       : "memory");
          asm volatile(
              "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                  smem_u32(W_hi)),
              "l"(wimg + (int64_t)(tt >> lg_tiles1) * wstride16), "r"((uint32_t)(2 * kTcOperandBytes)),
              "r"(smem_u32(wfull))
              : "memory");
        }
        ++w_issued;
        __syncwarp();
      }
    }
    // after an abort, the copies already issued land before the CTA exits
    if (*(volatile int*)&s_abort) {
      for (uint64_t k = i > 2 ? i - 2 : 0; k < i; ++k) mbar_wait(smem_u32(full + (k & 1)), (uint32_t)((k >> 1) & 1));
      if (w_issued > 0) mbar_wait(smem_u32(wfull), (uint32_t)((w_issued - 1) & 1));
    }
  } else if (warp == kTcbComputeWarps + 1) {
    // ---------------- MMA issue (one thread)
    if (lane == 0) {
      const uint32_t wh = smem_u32(W_hi), wl = smem_u32(W_lo);
      uint64_t i = 0, w_seen = 0;
      for (; i < my; ++i) {
        if (*(volatile int*)&s_abort) break;
        const int a = (int)(i & 1);
        if (new_state(i)) {
          if (!mbar_wait(smem_u32(wfull), (uint32_t)(w_seen & 1), spin)) { fail(1); break; }
          ++w_seen;
        }
        if (!mbar_wait(smem_u32(afull + a), (uint32_t)((i >> 1) & 1), spin)) { fail(1); break; }
        if (i >= 2 && !mbar_wait(smem_u32(dfree + a), (uint32_t)(((i >> 1) - 1) & 1), spin)) { fail(1); break; }
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        issue_tile_mmas_ta<PREC>(tmem + 256 + a * 128, tmem + a * 128, wh, wl);
        mma_commit(smem_u32(mdone + a));
        if (i + 1 < my && new_state(i + 1)) mma_commit(smem_u32(wfree));   // last tile on this W
      }
      // MMAs still in flight after an abort complete before the memory is released
      if (i > 0 && *(volatile int*)&s_abort) mbar_wait(smem_u32(mdone + ((i - 1) & 1)), (uint32_t)(((i - 1) >> 1) & 1));
    }
  } else {
    // ---------------- warps 0-15: thread = (row, column half)
    //   warps 0-7 convert (slot -> TMEM A), warps 8-15 drain (TMEM D -> HBM)
    const bool converter = warp < kTcbComputeWarps / 2;
    const int w8 = converter ? warp : warp - kTcbComputeWarps / 2;
    const int row = (w8 & 3) * 32 + lane, half = w8 >> 2;
    const uint32_t tq = (uint32_t)((w8 & 3) * 32) << 16;
    bool ok = true;
    if (converter) {
      uint32_t lrow = 0;
      for (int b = 0; b < 7; ++b) lrow |= (uint32_t)((row >> b) & 1) << lam_of(s_row[b]);
      // phi: column bits on qubits 0-3 take lane bits whose row qubits are >= 4
      uint32_t phi = 0, xbits = 0;
      {
        int k = 0;
        for (int b = 0; b < 4; ++b) {
          if (s_col[b] > 3) break;
          while (k < 5 && s_row[k] < 4) ++k;
          if (k >= 5) break;
          phi |= (uint32_t)((lane >> k) & 1) << b;
          xbits |= 1u << b;
          ++k;
        }
      }
      const float2* slot_f = (const float2*)slots;
      for (uint64_t i = 0; i < my; ++i) {
        if (__any_sync(0xffffffffu, *(volatile int*)&s_abort)) break;
        const int s = (int)(i & 1);
        // A buffer s was last read by the MMAs of tile i - 2
        if (i >= 2 && !mbar_wait_warp(smem_u32(mdone + s), (uint32_t)(((i >> 1) - 1) & 1), spin)) { ok = false; break; }
        if (!mbar_wait_warp(smem_u32(full + s), (uint32_t)((i >> 1) & 1), spin)) { ok = false; break; }
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        const float2* sl = slot_f + s * (kTcbSlotBytes / 8);
#pragma unroll 1
        for (int chunk = 0; chunk < 2; ++chunk) {
          const int c0 = half * 32 + chunk * 16;
          const uint32_t tb = lrow | lamcol[c0] | lamcol[phi];
          float2 v[16];
#pragma unroll
          for (int j = 0; j < 16; ++j) v[j] = sl[tb ^ lamcol[j]];
          if (xbits & 1) xor_stage<0>(v, phi & 1);
          if (xbits & 2) xor_stage<1>(v, (phi >> 1) & 1);
          if (xbits & 4) xor_stage<2>(v, (phi >> 2) & 1);
          if (xbits & 8) xor_stage<3>(v, (phi >> 3) & 1);
          uint32_t hi[16], lo[16];
#pragma unroll
          for (int j = 0; j < 16; ++j) split_amp<PREC>(v[j], ascale, hi[j], lo[j]);
          const uint32_t a_hi = tmem + tq + (uint32_t)s * 128 + c0;
          tmem_st16(a_hi, hi);
          if (PREC >= 3) tmem_st16(a_hi + 64, lo);
        }
        asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory");
        asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
        __syncwarp();
        if (lane == 0) {
          mbar_arrive(smem_u32(empty + s));
          mbar_arrive(smem_u32(afull + s));
        }
      }
    } else {
      // Store coalescing: a 32-byte sector is 4 amplitudes (qubits 0 and 1). When
      // column bit 0 (and bit 1) of the block sit on qubits 0 / 1, they are
      // exchanged with lane bits 4 (and 3), whose row qubits are >= 3, through
      // shuffles, so every warp store covers whole sectors. Slot q of lane l
      // then holds (row: l with bit 4 := q bit 0 [bit 3 := q bit 1],
      // column: q with bit 0 := l bit 4 [bit 1 := l bit 3]).
      const bool s0 = s_col[0] <= 1, s1 = s_col[0] == 0 && s_col[1] == 1;
      const bool l4 = (lane >> 4) & 1, l3 = (lane >> 3) & 1;
      const uint64_t rbit4 = 1ull << s_row[4], rbit3 = 1ull << s_row[3];
      uint64_t roff = 0;
      for (int b = 0; b < 7; ++b) roff |= (uint64_t)((row >> b) & 1) << s_row[b];
      if (s0) roff &= ~rbit4;
      if (s1) roff &= ~rbit3;
      const uint64_t* hc = coff + half * 32;
      const float inv = 1.0f / ascale;   // a power of two: exact
      for (uint64_t i = 0; i < my; ++i) {
        if (__any_sync(0xffffffffu, *(volatile int*)&s_abort)) break;
        const int d = (int)(i & 1);
        if (!mbar_wait_warp(smem_u32(mdone + d), (uint32_t)((i >> 1) & 1), spin)) { ok = false; break; }
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        const uint64_t tt = tile_of(i);
        float2* __restrict__ psi = state_ptr(tt);
        const uint64_t rb = tile_base(tt & tmask1) | roff;
#pragma unroll 1
        for (int chunk = 0; chunk < 2; ++chunk) {
          float o[32];
          tmem_ld32(tmem + tq + 256 + d * 128 + half * 64 + chunk * 32, o);
          if (chunk == 1) {   // accumulator read; the last stores follow
            asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
            __syncwarp();
            if (lane == 0) mbar_arrive(smem_u32(dfree + d));
          }
          float2 v[16];
#pragma unroll
          for (int q = 0; q < 16; ++q) v[q] = make_float2(o[2 * q] * inv, o[2 * q + 1] * inv);
          if (s0) xchg_stage<0, 4>(v, l4);
          if (s1) xchg_stage<1, 3>(v, l3);
#pragma unroll
          for (int q = 0; q < 16; ++q) {
            uint64_t a = rb;
            int qq = q;
            if (s0) {
              if (q & 1) a |= rbit4;
              qq = (qq & ~1) | (int)l4;
            }
            if (s1) {
              if (q & 2) a |= rbit3;
              qq = (qq & ~2) | ((int)l3 << 1);
            }
            psi[a | hc[chunk * 16 + qq]] = v[q];
          }
        }
      }
    }
    if (!ok && lane == 0) fail(1);
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (warp == 0)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kTcbTmemCols) : "memory");
}

size_t tc_bulk_smem_bytes() {
  return 2 * (size_t)kTcbSlotBytes + 2 * (size_t)kTcOperandBytes + 4 * 256 * 8 + 64 * 8 * 2 + 64 * 4 + 28 * 4 +
         12 * 8 + 16 + 1024;
}

size_t tc_smem_bytes() { return 6 * (size_t)kTcOperandBytes + 64 * 8 + 32 + 1024; }

static bool g_tc_ready = false;
static int g_tc_sms = 0;

// Host-side set-up (outside any stream capture): shared-memory attribute of
// every instance and the SM count.
template <int PREC>
static cudaError_t set_tc_attributes(int smem, int smem_bulk) {
  cudaError_t e = cudaFuncSetAttribute(k_tc_block<PREC, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
  if (e == cudaSuccess) e = cudaFuncSetAttribute(k_tc_block<PREC, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(k_tc_bulk<PREC, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem_bulk);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(k_tc_bulk<PREC, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem_bulk);
  return e;
}

cudaError_t prepare_tc_pass() {
  if (g_tc_ready) return cudaSuccess;
  const int smem = (int)tc_smem_bytes(), smem_bulk = (int)tc_bulk_smem_bytes();
  cudaError_t e = set_tc_attributes<1>(smem, smem_bulk);
  if (e == cudaSuccess) e = set_tc_attributes<3>(smem, smem_bulk);
  if (e == cudaSuccess) e = set_tc_attributes<4>(smem, smem_bulk);
  if (e != cudaSuccess) return e;
  int dev = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&g_tc_sms, cudaDevAttrMultiProcessorCount, dev);
  g_tc_ready = true;
  return cudaSuccess;
}

// 2^s with s = min(floor(n / 2), 15): the fp16 pre-scale of PREC 4 (|amp| <= 1,
// so scaled values stay <= 32768 < 65504, the largest fp16).
float tc_amp_scale(int n, int prec) {
  if (prec != 4) return 1.0f;
  const int s = n / 2 < 15 ? n / 2 : 15;
  return (float)(1u << s);
}

template <int PREC>
static void launch_tc_instance(int pipeline, bool multi, unsigned grid, size_t smem, cudaStream_t st, float2* psi,
                               void* const* psis, const TcPassDesc& p, const uint4* w, int64_t ws16, int lg,
                               uint64_t ntiles, float sc, int* err, uint32_t spin) {
  if (pipeline == 0) {
    if (multi) k_tc_bulk<PREC, true><<<grid, kTcbThreads, smem, st>>>(psi, psis, p, w, ws16, lg, ntiles, sc, err, spin);
    else k_tc_bulk<PREC, false><<<grid, kTcbThreads, smem, st>>>(psi, psis, p, w, ws16, lg, ntiles, sc, err, spin);
  } else {
    if (multi) k_tc_block<PREC, true><<<grid, kTc2Threads, smem, st>>>(psi, psis, p, w, ws16, lg, ntiles, sc, err);
    else k_tc_block<PREC, false><<<grid, kTc2Threads, smem, st>>>(psi, psis, p, w, ws16, lg, ntiles, sc, err);
  }
}

cudaError_t launch_tc_pass_batched(void* psi, void* const* psis, int nstates, int64_t wstride, int n,
                                   const TcPassDesc& p, const void* wimg, int prec, int pipeline, int* err,
                                   cudaStream_t st, uint32_t spin) {
  if (spin == 0) spin = kTcSpinLimit;
  if (!g_tc_ready) return cudaErrorInvalidConfiguration;   // not prepared
  if (prec != 1 && prec != 3 && prec != 4) return cudaErrorInvalidValue;
  const uint64_t ntiles = (1ull << (n - 13)) * (uint64_t)nstates;
  const unsigned grid = (unsigned)(ntiles < (uint64_t)g_tc_sms ? ntiles : (uint64_t)g_tc_sms);
  const size_t smem = pipeline == 0 ? tc_bulk_smem_bytes() : tc_smem_bytes();
  const float sc = tc_amp_scale(n, prec);
  const bool multi = psis != nullptr;
  const uint4* w = (const uint4*)wimg;
  if (prec == 4)
    launch_tc_instance<4>(pipeline, multi, grid, smem, st, (float2*)psi, psis, p, w, wstride / 8, n - 13, ntiles, sc, err, spin);
  else if (prec == 3)
    launch_tc_instance<3>(pipeline, multi, grid, smem, st, (float2*)psi, psis, p, w, wstride / 8, n - 13, ntiles, sc, err, spin);
  else
    launch_tc_instance<1>(pipeline, multi, grid, smem, st, (float2*)psi, psis, p, w, wstride / 8, n - 13, ntiles, sc, err, spin);
  note_launch();
  return cudaGetLastError();
}

cudaError_t launch_tc_pass(void* psi, int n, const TcPassDesc& p, const void* wimg, int prec, int pipeline,
                           int* err, cudaStream_t st, uint32_t spin) {
  return launch_tc_pass_batched(psi, nullptr, 1, 0, n, p, wimg, prec, pipeline, err, st, spin);
}

}  // namespace qs
