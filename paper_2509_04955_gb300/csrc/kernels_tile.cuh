#pragma once
// Tile-pass kernel: one HBM sweep applies a whole run of fused blocks.
//
// Section 3.4 contracts gates to cut operation counts, and Section 3.3 runs
// several gates per kernel to raise memory throughput. On GB300 both goals are
// met by staging a tile of 2^m amplitudes in shared memory and applying, in
// order, every op of a pass whose qubits lie in the tile's qubit set T:
//   T = {0 .. L-1} (contiguous runs of 2^L amplitudes: coalesced 16-byte
//       loads) plus up to m - L arbitrary higher qubits.
// A tile is the set of amplitudes whose bits outside T equal the tile number;
// the high tile qubits select 2^(m-L) runs of 2^L contiguous amplitudes.
// Tile-local index j: bits 0..L-1 = qubits 0..L-1, bits L.. = T's high qubits
// in ascending order. Ops carry tile-local bit positions.
//
// Each CTA walks tiles with a grid stride; the run offsets of the high qubits
// are computed once per CTA. Ops:
//   OP_GATE  one original gate (forms of the per-gate kernels, Eq. 3/4/6),
//            matrix from the gate table;
//   OP_DENSE dense 2^k x 2^k block (Eq. 6 generalised, Eq. 7 products),
//            matrix staged once per op in shared memory, one group of 2^k
//            amplitudes per thread held in registers;
//   OP_DIAG  diagonal block, 2^k phases.
#include <cuda_runtime.h>

#include <type_traits>

#include "cplx.cuh"
#include "dfloat.cuh"
#include "qs_internal.h"
#include "tcgen05.cuh"

namespace qs {

constexpr int kTileThreads = 256;

// Amplitude type in HBM for each arithmetic type of the tile (complex128 tiles
// computed in FP32 pairs keep complex128 in HBM).
template <typename R> struct GAmp { using T = typename V2<R>::T; };
template <> struct GAmp<dfl> { using T = double2; };

// The same transfer for FP32-pair tiles: one complex128 amplitude per 16-byte
// access, split into (h, l) pairs on the way in and joined on the way out.
template <bool LOAD, int BATCH = 4>
__device__ __forceinline__ void tile_io_df(double2* __restrict__ psi, dfc* tile, uint64_t base, const uint64_t* segoff,
                                           uint32_t size, int L, uint32_t lmask) {
  for (uint32_t e0 = threadIdx.x; e0 < size; e0 += kTileThreads * BATCH) {
    double2 buf[BATCH];
#pragma unroll
    for (int u = 0; u < BATCH; ++u) {
      const uint32_t e = e0 + (uint32_t)u * kTileThreads;
      if (e < size) {
        if (LOAD) buf[u] = psi[base | segoff[e >> L] | (e & lmask)];
        else buf[u] = from_dfc(tile[e]);
      }
    }
#pragma unroll
    for (int u = 0; u < BATCH; ++u) {
      const uint32_t e = e0 + (uint32_t)u * kTileThreads;
      if (e < size) {
        if (LOAD) tile[e] = to_dfc(buf[u]);
        else psi[base | segoff[e >> L] | (e & lmask)] = buf[u];
      }
    }
  }
}

// HBM <-> shared-memory transfer of one tile: 16-byte vectors, BATCH
// independent loads issued before their shared-memory stores (and the reverse
// on the way out), so a CTA keeps kTileThreads x BATCH x 16 bytes in flight.
template <typename C, typename C2, int VPT, bool LOAD, int BATCH = (VPT == 2 ? 8 : 4)>
__device__ __forceinline__ void tile_io(C* __restrict__ psi, C* tile, uint64_t base, const uint64_t* segoff,
                                        uint32_t size, int L, uint32_t lmask) {
  for (uint32_t e0 = threadIdx.x * VPT; e0 < size; e0 += kTileThreads * VPT * BATCH) {
    C2 buf[BATCH];
#pragma unroll
    for (int u = 0; u < BATCH; ++u) {
      const uint32_t e = e0 + (uint32_t)u * kTileThreads * VPT;
      if (e < size) {
        if (LOAD) buf[u] = *(const C2*)(psi + (base | segoff[e >> L] | (e & lmask)));
        else buf[u] = *(const C2*)(tile + e);
      }
    }
#pragma unroll
    for (int u = 0; u < BATCH; ++u) {
      const uint32_t e = e0 + (uint32_t)u * kTileThreads * VPT;
      if (e < size) {
        if (LOAD) *(C2*)(tile + e) = buf[u];
        else *(C2*)(psi + (base | segoff[e >> L] | (e & lmask))) = buf[u];
      }
    }
  }
}

__device__ __forceinline__ uint32_t ins0(uint32_t x, const int32_t* pos, int npos) {
  return insert_zero_bits_u<4, uint32_t>(x, pos, npos);
}

template <int K>
__device__ __forceinline__ uint32_t ins0k(uint32_t x, const int32_t* pos) {
#pragma unroll
  for (int k = 0; k < K; ++k) {
    const uint32_t lo = x & ((1u << pos[k]) - 1);
    x = ((x >> pos[k]) << (pos[k] + 1)) | lo;
  }
  return x;
}

// One-target gate over the tile: each thread takes kPairBatch independent
// pairs per iteration (all loads, then the arithmetic, then the stores), so
// the dependent chains of one pair overlap with the others'. A slot past the
// end recomputes the iteration's first pair and does not store.
constexpr int kPairBatch = 4;

// ONE: the op inserts a single zero bit (an uncontrolled one-target gate), so
// the pair index is ((p & ~lo) << 1) | (p & lo) with lo the bits below it.
template <bool ONE, typename C, typename F>
__device__ __forceinline__ void pairs_apply_t(C* tile, uint32_t count, const int32_t* ins, int nins, uint32_t cmask,
                                              uint32_t ta, F f) {
  const uint32_t lo = (1u << ins[0]) - 1;
  for (uint32_t p0 = threadIdx.x; p0 < count; p0 += kTileThreads * kPairBatch) {
    uint32_t idx[kPairBatch];
    C a0[kPairBatch], a1[kPairBatch];
#pragma unroll
    for (int u = 0; u < kPairBatch; ++u) {
      const uint32_t p = p0 + (uint32_t)u * kTileThreads;
      const uint32_t q = p < count ? p : p0;
      if constexpr (ONE) idx[u] = ((q & ~lo) << 1) | (q & lo);
      else idx[u] = ins0(q, ins, nins) | cmask;
      a0[u] = tile[idx[u]];
      a1[u] = tile[idx[u] | ta];
    }
#pragma unroll
    for (int u = 0; u < kPairBatch; ++u) f(a0[u], a1[u]);
#pragma unroll
    for (int u = 0; u < kPairBatch; ++u)
      if (p0 + (uint32_t)u * kTileThreads < count) {
        tile[idx[u]] = a0[u];
        tile[idx[u] | ta] = a1[u];
      }
  }
}

template <typename C, typename F>
__device__ __forceinline__ void pairs_apply(C* tile, uint32_t count, const int32_t* ins, int nins, uint32_t cmask,
                                            uint32_t ta, F f) {
  if (nins == 1 && cmask == 0) pairs_apply_t<true>(tile, count, ins, nins, cmask, ta, f);
  else pairs_apply_t<false>(tile, count, ins, nins, cmask, ta, f);
}

template <typename R>
__device__ __forceinline__ void apply_gate_op(typename V2<R>::T* tile, int m, const DevOp& op,
                                              const double2* __restrict__ gtab, typename V2<R>::T* mbuf) {
  using C = typename V2<R>::T;
  const double2* mat = gtab + (int64_t)op.mat * 16;
  const uint32_t count = 1u << (m - op.nins);
  const uint32_t ta = 1u << op.t0;
  if (op.form == FORM_DENSE2) {
    if (threadIdx.x < 16) mbuf[threadIdx.x] = from_d<R>(mat[threadIdx.x]);
    __syncthreads();
    const uint32_t tb = 1u << op.t1;
    for (uint32_t p = threadIdx.x; p < count; p += kTileThreads) {
      const uint32_t b = ins0(p, op.ins, op.nins) | op.cmask;
      const uint32_t idx[4] = {b, b | ta, b | tb, b | ta | tb};
      C a[4];
#pragma unroll
      for (int j = 0; j < 4; ++j) a[j] = tile[idx[j]];
#pragma unroll
      for (int r = 0; r < 4; ++r) {
        C acc = cmul(mbuf[4 * r], a[0]);
#pragma unroll
        for (int j = 1; j < 4; ++j) acc = cfma(mbuf[4 * r + j], a[j], acc);
        tile[idx[r]] = acc;
      }
    }
    return;
  }
  if (op.form == FORM_SWAP2) {
    const uint32_t tb = 1u << op.t1;
    for (uint32_t p = threadIdx.x; p < count; p += kTileThreads) {
      const uint32_t b = ins0(p, op.ins, op.nins) | op.cmask;
      const C x = tile[b | ta], y = tile[b | tb];
      tile[b | ta] = y;
      tile[b | tb] = x;
    }
    return;
  }
  const C m00 = from_d<R>(mat[0]), m01 = from_d<R>(mat[1]), m10 = from_d<R>(mat[2]), m11 = from_d<R>(mat[3]);
  switch (op.form) {
    case FORM_DENSE1:
      pairs_apply(tile, count, op.ins, op.nins, op.cmask, ta, [&](C& a0, C& a1) {
        const C r0 = cfma(m01, a1, cmul(m00, a0));
        a1 = cfma(m11, a1, cmul(m10, a0));
        a0 = r0;
      });
      break;
    case FORM_REAL1:
      pairs_apply(tile, count, op.ins, op.nins, op.cmask, ta, [&](C& a0, C& a1) {
        const C r0 = rmix<R>(m00.x, a0, m01.x, a1);
        a1 = rmix<R>(m10.x, a0, m11.x, a1);
        a0 = r0;
      });
      break;
    case FORM_RXLIKE1:
      pairs_apply(tile, count, op.ins, op.nins, op.cmask, ta, [&](C& a0, C& a1) {
        const C r0 = ixmix<R>(m00.x, a0, m01.y, a1);
        a1 = ixmix<R>(m11.x, a1, m10.y, a0);
        a0 = r0;
      });
      break;
    case FORM_X1:
      pairs_apply(tile, count, op.ins, op.nins, op.cmask, ta, [&](C& a0, C& a1) {
        const C r0 = a1;
        a1 = a0;
        a0 = r0;
      });
      break;
    case FORM_ANTI1:
      pairs_apply(tile, count, op.ins, op.nins, op.cmask, ta, [&](C& a0, C& a1) {
        const C r0 = cmul(m01, a1);
        a1 = cmul(m10, a0);
        a0 = r0;
      });
      break;
    case FORM_PHASE1:
      for (uint32_t p = threadIdx.x; p < count; p += kTileThreads) {
        const uint32_t b = ins0(p, op.ins, op.nins) | op.cmask;
        tile[b | ta] = cmul(m11, tile[b | ta]);
      }
      break;
    default:  // DIAG1
      for (uint32_t p = threadIdx.x; p < count; p += kTileThreads) {
        const uint32_t b = ins0(p, op.ins, op.nins) | op.cmask;
        tile[b] = cmul((b & ta) ? m11 : m00, tile[b]);
      }
  }
}

// Groups per thread of a dense op: each staged matrix entry is loaded once
// and used for G groups (register budget about 64 values for the inputs).
template <typename R, int K> struct DenseG {
  static constexpr int v = sizeof(R) == 4 ? (K <= 3 ? 4 : K == 4 ? 2 : 1) : (K <= 2 ? 2 : 1);
};

template <typename R, int K>
__device__ __forceinline__ void apply_dense_op(typename V2<R>::T* tile, int m, const DevOp& op,
                                               const double2* __restrict__ btab, typename V2<R>::T* mbuf) {
  using C = typename V2<R>::T;
  constexpr int D = 1 << K;
  constexpr int G = DenseG<R, K>::v;
  for (int i = threadIdx.x; i < D * D; i += kTileThreads) mbuf[i] = from_d<R>(btab[op.mat + i]);
  __syncthreads();
  uint32_t off[D];
#pragma unroll
  for (int j = 0; j < D; ++j) {
    uint32_t o = 0;
#pragma unroll
    for (int b = 0; b < K; ++b) o |= ((j >> b) & 1u) << op.ins[b];
    off[j] = o;
  }
  const uint32_t groups = 1u << (m - K);
  for (uint32_t g0 = threadIdx.x; g0 < groups; g0 += kTileThreads * G) {
    uint32_t i0[G];
    C v[G][D];
#pragma unroll
    for (int i = 0; i < G; ++i) {
      const uint32_t gi = g0 + i * kTileThreads;
      i0[i] = ins0k<K>(gi < groups ? gi : 0, op.ins);
#pragma unroll
      for (int j = 0; j < D; ++j) v[i][j] = tile[i0[i] | off[j]];
    }
#pragma unroll
    for (int r = 0; r < D; ++r) {
      C acc[G];
      {
        const C mm = mbuf[r * D];
#pragma unroll
        for (int i = 0; i < G; ++i) acc[i] = cmul(mm, v[i][0]);
      }
#pragma unroll
      for (int j = 1; j < D; ++j) {
        const C mm = mbuf[r * D + j];
#pragma unroll
        for (int i = 0; i < G; ++i) acc[i] = cfma(mm, v[i][j], acc[i]);
      }
#pragma unroll
      for (int i = 0; i < G; ++i)
        if (g0 + i * kTileThreads < groups) tile[i0[i] | off[r]] = acc[i];
    }
  }
}

template <typename R>
__device__ __forceinline__ void apply_diag_op(typename V2<R>::T* tile, int m, const DevOp& op,
                                              const double2* __restrict__ btab, typename V2<R>::T* mbuf) {
  const int D = 1 << op.k;
  for (int i = threadIdx.x; i < D; i += kTileThreads) mbuf[i] = from_d<R>(btab[op.mat + i]);
  __syncthreads();
  const uint32_t size = 1u << m;
  for (uint32_t e = threadIdx.x; e < size; e += kTileThreads) {
    uint32_t loc = 0;
#pragma unroll
    for (int b = 0; b < 6; ++b)
      if (b < op.k) loc |= ((e >> op.ins[b]) & 1u) << b;
    tile[e] = cmul(mbuf[loc], tile[e]);
  }
}

// The ops of a pass applied, in order, to the tile in shared memory (a barrier
// after each op).
template <typename R, int KMAX>
__device__ __forceinline__ void tile_apply_ops(typename V2<R>::T* tile, const PassDesc& p, const DevOp* __restrict__ ops,
                                               const double2* __restrict__ gtab, const double2* __restrict__ btab,
                                               int64_t brow0, int64_t bstride, uint64_t sb,
                                               typename V2<R>::T* mbuf) {
  const int m = p.m;
  for (int o = p.op_begin; o < p.op_end; ++o) {
    const DevOp op = ops[o];
    if (op.type == OP_GATE) {
      apply_gate_op<R>(tile, m, op, gtab, mbuf);
    } else {
      const double2* __restrict__ bt = op.per_row ? btab + (brow0 + (int64_t)sb) * bstride : btab;
      if (op.type == OP_DIAG) {
        apply_diag_op<R>(tile, m, op, bt, mbuf);
      } else {
        if (op.k == 1) apply_dense_op<R, 1>(tile, m, op, bt, mbuf);
        else if (op.k == 2) apply_dense_op<R, 2>(tile, m, op, bt, mbuf);
        if constexpr (KMAX >= 3) { if (op.k == 3) apply_dense_op<R, 3>(tile, m, op, bt, mbuf); }
        if constexpr (KMAX >= 4) { if (op.k == 4) apply_dense_op<R, 4>(tile, m, op, bt, mbuf); }
        if constexpr (KMAX >= 5) { if (op.k == 5) apply_dense_op<R, 5>(tile, m, op, bt, mbuf); }
      }
    }
    __syncthreads();
  }
}

// Gate-only passes (KMAX <= 2) keep two CTAs per SM (load of one tile overlaps
// the ops of the other); wider dense ops need more registers.
template <typename R, int KMAX>
__global__ void __launch_bounds__(kTileThreads, KMAX <= 2 ? 2 : 1) k_tile(typename GAmp<R>::T* __restrict__ psi0,
                                                        void* const* __restrict__ psis, int64_t gstride,
                                                        int64_t bstride, PassDesc p, const DevOp* __restrict__ ops,
                                                        const double2* __restrict__ gtab0,
                                                        const double2* __restrict__ btab, int64_t brow0, int lg_tiles,
                                                        uint64_t total) {
  using C = typename V2<R>::T;
  using G = typename GAmp<R>::T;
  using C2 = typename std::conditional<sizeof(R) == 4, float4, double2>::type;  // 16-byte vector
  constexpr int VPT = 16 / sizeof(C);                                           // amplitudes per vector
  constexpr bool kDF = std::is_same<R, dfl>::value;
  extern __shared__ __align__(16) unsigned char smem[];
  const int m = p.m, L = p.L, nh = p.nhigh;
  C* tile = (C*)smem;
  uint64_t* segoff = (uint64_t*)(tile + (1u << m));
  C* mbuf = (C*)(segoff + ((1u << nh) < 2 ? 2 : (1u << nh)));   // keeps mbuf 16-byte aligned

  for (uint32_t s = threadIdx.x; s < (1u << nh); s += kTileThreads) {
    uint64_t o = 0;
    for (int k = 0; k < nh; ++k) o |= (uint64_t)((s >> k) & 1u) << p.high[k];
    segoff[s] = o;
  }
  __syncthreads();
  const uint32_t size = 1u << m, lmask = (1u << L) - 1;
  // `total` = 2^lg_tiles x states: with a state list (batched execution) tile
  // index tt covers state tt >> lg_tiles, whose gate table row is gstride apart.
  for (uint64_t tt = blockIdx.x; tt < total; tt += gridDim.x) {
    const uint64_t sb = tt >> lg_tiles, t = tt & ((1ull << lg_tiles) - 1);
    G* __restrict__ psi = psis ? (G*)psis[sb] : psi0;
    const double2* __restrict__ gtab = gtab0 + sb * gstride;
    const uint64_t base = insert_zero_bits(t << L, p.high, nh);
    if constexpr (kDF) tile_io_df<true>(psi, tile, base, segoff, size, L, lmask);
    else tile_io<C, C2, VPT, true>(psi, tile, base, segoff, size, L, lmask);
    __syncthreads();
    tile_apply_ops<R, KMAX>(tile, p, ops, gtab, btab, brow0, bstride, sb, mbuf);
    if constexpr (kDF) tile_io_df<false>(psi, tile, base, segoff, size, L, lmask);
    else tile_io<C, C2, VPT, false>(psi, tile, base, segoff, size, L, lmask);
    __syncthreads();
  }
}

// The same pass with the tile moved by the bulk-copy (TMA) engine: each run
// of 2^L contiguous amplitudes is one cp.async.bulk of at least 16 bytes, into
// one of two shared-memory tile buffers, so the next tile streams in while the
// ops run on this one, and the tile goes back to HBM by bulk stores from the
// same buffer. Warp 0 issues the copies (its lane j takes runs j, j + 32, ...);
// a tile buffer is loaded again only after the stores from it have been read
// out (cp.async.bulk.wait_group.read). Waits for a tile are bounded by p.spin
// polls: when one runs out the CTA records *p.err = 1, waits for the copies it
// issued and returns. Complex64 and FP64 tiles only (FP32-pair tiles are
// converted on the way in).
template <typename R, int KMAX>
__global__ void __launch_bounds__(kTileThreads, KMAX <= 2 ? 2 : 1) k_tile_bulk(typename V2<R>::T* __restrict__ psi0,
                                                           void* const* __restrict__ psis, int64_t gstride,
                                                           int64_t bstride, PassDesc p, const DevOp* __restrict__ ops,
                                                           const double2* __restrict__ gtab0,
                                                           const double2* __restrict__ btab, int64_t brow0,
                                                           int lg_tiles, uint64_t total) {
  using C = typename V2<R>::T;
  extern __shared__ __align__(16) unsigned char smem[];
  const int m = p.m, L = p.L, nh = p.nhigh;
  const uint32_t size = 1u << m;
  C* tiles = (C*)smem;                                            // two buffers of 2^m amplitudes
  uint64_t* segoff = (uint64_t*)(tiles + 2 * size);
  C* mbuf = (C*)(segoff + ((1u << nh) < 2 ? 2 : (1u << nh)));
  uint64_t* full = (uint64_t*)(mbuf + (p.mbuf_elems < 16 ? 16 : p.mbuf_elems));   // [2]
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const uint32_t spin = p.spin ? p.spin : kTcSpinLimit;
  const uint32_t nruns = 1u << nh, runb = (uint32_t)sizeof(C) << L;
  for (uint32_t s = threadIdx.x; s < nruns; s += kTileThreads) {
    uint64_t o = 0;
    for (int k = 0; k < nh; ++k) o |= (uint64_t)((s >> k) & 1u) << p.high[k];
    segoff[s] = o;
  }
  if (threadIdx.x == 0) {
    for (int b = 0; b < 2; ++b) asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(full + b)), "r"(1));
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncthreads();
  const uint64_t my = blockIdx.x < total ? (total - blockIdx.x + gridDim.x - 1) / gridDim.x : 0;
  auto tile_at = [&](uint64_t i, C*& psi, uint64_t& base, uint64_t& sb) {
    const uint64_t tt = blockIdx.x + i * gridDim.x;
    sb = tt >> lg_tiles;
    psi = psis ? (C*)psis[sb] : psi0;
    base = insert_zero_bits((tt & ((1ull << lg_tiles) - 1)) << L, p.high, nh);
  };
  // warp 0 only: the runs of tile i into buffer i & 1
  auto issue_load = [&](uint64_t i) {
    C* psi;
    uint64_t base, sb;
    tile_at(i, psi, base, sb);
    const int b = (int)(i & 1);
    if (lane == 0)
      asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(full + b)),
                   "r"((uint32_t)(size * sizeof(C)))
                   : "memory");
    __syncwarp();
    for (uint32_t j = lane; j < nruns; j += 32)
      asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                       smem_u32(tiles + (size_t)b * size + (size_t)j * (1u << L))),
                   "l"(psi + (base | segoff[j])), "r"(runb), "r"(smem_u32(full + b))
                   : "memory");
  };
  if (warp == 0 && my > 0) issue_load(0);
  uint64_t i = 0;
  bool timed_out = false;
  for (; i < my; ++i) {
    const int b = (int)(i & 1);
    if (warp == 0 && i + 1 < my) {
      // buffer b ^ 1 last held tile i - 1: its stores must have read it out
      asm volatile("cp.async.bulk.wait_group.read 0;" ::: "memory");
      issue_load(i + 1);
    }
    const bool ok = mbar_wait(smem_u32(full + b), (uint32_t)((i >> 1) & 1), spin);
    if (__syncthreads_or(!ok)) {
      timed_out = true;
      break;
    }
    C* psi;
    uint64_t base, sb;
    tile_at(i, psi, base, sb);
    C* tile = tiles + (size_t)b * size;
    tile_apply_ops<R, KMAX>(tile, p, ops, gtab0 + sb * gstride, btab, brow0, bstride, sb, mbuf);
    if (warp == 0) {
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");   // the ops' writes, before the bulk reads
      for (uint32_t j = lane; j < nruns; j += 32)
        asm volatile("cp.async.bulk.global.shared::cta.bulk_group [%0], [%1], %2;" ::"l"(psi + (base | segoff[j])),
                     "r"(smem_u32(tile + (size_t)j * (1u << L))), "r"(runb)
                     : "memory");
      asm volatile("cp.async.bulk.commit_group;" ::: "memory");
    }
  }
  if (warp == 0) {
    if (timed_out) {
      if (lane == 0) atomicExch(p.err, 1);
      // the loads issued for tiles i and i + 1 land before the CTA exits
      mbar_wait(smem_u32(full + (i & 1)), (uint32_t)((i >> 1) & 1));
      if (i + 1 < my) mbar_wait(smem_u32(full + ((i + 1) & 1)), (uint32_t)(((i + 1) >> 1) & 1));
    }
    asm volatile("cp.async.bulk.wait_group 0;" ::: "memory");   // stores complete
  }
}

// Per kernel instance: the largest dynamic shared memory configured so far
// and the resident CTAs per SM at that size. Set up by prepare_tile_pass
// (host side, outside any stream capture) before the first launch.
template <typename R, int KMAX, bool BULK>
struct TileCfg {
  static int bytes, per_sm;
};
template <typename R, int KMAX, bool BULK> int TileCfg<R, KMAX, BULK>::bytes = 0;
template <typename R, int KMAX, bool BULK> int TileCfg<R, KMAX, BULK>::per_sm = 0;

template <typename R, int KMAX, bool BULK>
static const void* tile_kernel() {
  if constexpr (BULK) return (const void*)k_tile_bulk<R, KMAX>;
  else return (const void*)k_tile<R, KMAX>;
}

template <typename R, int KMAX, bool BULK>
static cudaError_t prepare_tile_t(size_t smem) {
  if ((int)smem <= TileCfg<R, KMAX, BULK>::bytes) return cudaSuccess;
  cudaError_t e = cudaFuncSetAttribute(tile_kernel<R, KMAX, BULK>(), cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  int per_sm = 0;
  e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, tile_kernel<R, KMAX, BULK>(), kTileThreads, smem);
  if (e != cudaSuccess) return e;
  if (per_sm < 1) return cudaErrorInvalidConfiguration;
  TileCfg<R, KMAX, BULK>::bytes = (int)smem;
  TileCfg<R, KMAX, BULK>::per_sm = per_sm;
  return cudaSuccess;
}

static int sm_count() {
  static int sms = 0;
  if (!sms) {
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  }
  return sms;
}

template <typename R, int KMAX, bool BULK>
static cudaError_t launch_tile_t(void* psi, void* const* psis, int nstates, int64_t gstride, int64_t bstride,
                                 int64_t brow0, int n, const PassDesc& p, const DevOp* ops, const double2* gtab,
                                 const double2* btab, cudaStream_t st, size_t smem) {
  if ((int)smem > TileCfg<R, KMAX, BULK>::bytes) return cudaErrorInvalidConfiguration;   // not prepared
  const int per_sm = TileCfg<R, KMAX, BULK>::per_sm;
  const int sms = sm_count();
  const uint64_t ntiles = 1ull << (n - p.m), total = ntiles * (uint64_t)nstates;
  uint64_t grid = (uint64_t)sms * per_sm;
  if (grid > total) grid = total;
  if constexpr (BULK) {
    if (p.err == nullptr) return cudaErrorInvalidValue;
    k_tile_bulk<R, KMAX><<<(unsigned)grid, kTileThreads, smem, st>>>((typename V2<R>::T*)psi, psis, gstride, bstride,
                                                                      p, ops, gtab, btab, brow0, n - p.m, total);
  } else {
    k_tile<R, KMAX><<<(unsigned)grid, kTileThreads, smem, st>>>((typename GAmp<R>::T*)psi, psis, gstride, bstride, p,
                                                                  ops, gtab, btab, brow0, n - p.m, total);
  }
  note_launch();
  return cudaGetLastError();
}

// kmax -> instance: every block of the pass has at most kmax qubits (0-2 share
// the k = 2 instance). The translation units kernels_tile_f32.cu,
// kernels_tile_f64.cu, kernels_tile_df.cu (FP32 pairs, k <= 4) and
// kernels_tile_df5.cu (FP32 pairs, k = 5) each instantiate the range
// [KLO, KHI] of one arithmetic type, so the tile kernels compile in parallel.
template <typename R, int KLO, int KHI>
static cudaError_t launch_tile_range(int kmax, void* psi, void* const* psis, int nstates, int64_t gstride,
                                     int64_t bstride, int64_t brow0, int n, const PassDesc& p, const DevOp* ops,
                                     const double2* gtab, const double2* btab, cudaStream_t st, size_t smem) {
  if (kmax < 0 || kmax > 5) return cudaErrorInvalidValue;
  const int k = kmax < 2 ? 2 : kmax;
#define QS_TILE_CASE(K)                                                                                  \
  if constexpr (KLO <= K && K <= KHI)                                                                    \
    if (k == K) {                                                                                        \
      if constexpr (!std::is_same<R, dfl>::value)                                                        \
        if (p.bulk) return launch_tile_t<R, K, true>(psi, psis, nstates, gstride, bstride, brow0, n, p, ops, gtab, btab, st, smem); \
      return launch_tile_t<R, K, false>(psi, psis, nstates, gstride, bstride, brow0, n, p, ops, gtab, btab, st, smem); \
    }
  QS_TILE_CASE(2)
  QS_TILE_CASE(3)
  QS_TILE_CASE(4)
  QS_TILE_CASE(5)
#undef QS_TILE_CASE
  return cudaErrorInvalidValue;
}

template <typename R, int KLO, int KHI>
static cudaError_t prepare_tile_range(int kmax, bool bulk, size_t smem) {
  sm_count();   // this translation unit's SM count, read here rather than during a stream capture
  if (kmax < 0 || kmax > 5) return cudaErrorInvalidValue;
  const int k = kmax < 2 ? 2 : kmax;
#define QS_TILE_CASE(K)                                  \
  if constexpr (KLO <= K && K <= KHI)                    \
    if (k == K) {                                        \
      if constexpr (!std::is_same<R, dfl>::value)        \
        if (bulk) return prepare_tile_t<R, K, true>(smem); \
      return prepare_tile_t<R, K, false>(smem);           \
    }
  QS_TILE_CASE(2)
  QS_TILE_CASE(3)
  QS_TILE_CASE(4)
  QS_TILE_CASE(5)
#undef QS_TILE_CASE
  return cudaErrorInvalidValue;
}

#define QS_TILE_PART_DECL(SUFFIX)                                                                         \
  cudaError_t launch_tile_##SUFFIX(int kmax, void* psi, void* const* psis, int nstates, int64_t gstride,   \
                                   int64_t bstride, int64_t brow0, int n, const PassDesc& p, const DevOp* ops, \
                                   const double2* gtab, const double2* btab, cudaStream_t st, size_t smem); \
  cudaError_t prepare_tile_##SUFFIX(int kmax, bool bulk, size_t smem);
QS_TILE_PART_DECL(f32)
QS_TILE_PART_DECL(f64)
QS_TILE_PART_DECL(df)
QS_TILE_PART_DECL(df5)

}  // namespace qs
