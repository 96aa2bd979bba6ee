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
    if constexpr (kDF) tile_io_df<false>(psi, tile, base, segoff, size, L, lmask);
    else tile_io<C, C2, VPT, false>(psi, tile, base, segoff, size, L, lmask);
    __syncthreads();
  }
}

size_t tile_smem_bytes(int m, int nhigh, int mbuf_elems, qs_dtype dt) {
  const size_t amp = dt == QS_C64 ? 8 : 16;
  const size_t runs = nhigh == 0 ? 2 : (1ull << nhigh);   // padded to 16 bytes
  return (amp << m) + 8 * runs + amp * (size_t)(mbuf_elems < 16 ? 16 : mbuf_elems);
}

// Per kernel instance: the largest dynamic shared memory configured so far
// and the resident CTAs per SM at that size. Set up by prepare_tile_pass
// (host side, outside any stream capture) before the first launch.
template <typename R, int KMAX>
struct TileCfg {
  static int bytes, per_sm;
};
template <typename R, int KMAX> int TileCfg<R, KMAX>::bytes = 0;
template <typename R, int KMAX> int TileCfg<R, KMAX>::per_sm = 0;

template <typename R, int KMAX>
static cudaError_t prepare_tile_t(size_t smem) {
  if ((int)smem <= TileCfg<R, KMAX>::bytes) return cudaSuccess;
  cudaError_t e = cudaFuncSetAttribute(k_tile<R, KMAX>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  int per_sm = 0;
  e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_tile<R, KMAX>, kTileThreads, smem);
  if (e != cudaSuccess) return e;
  if (per_sm < 1) return cudaErrorInvalidConfiguration;
  TileCfg<R, KMAX>::bytes = (int)smem;
  TileCfg<R, KMAX>::per_sm = per_sm;
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

template <typename R, int KMAX>
static cudaError_t launch_tile_t(void* psi, void* const* psis, int nstates, int64_t gstride, int64_t bstride,
                                 int64_t brow0, int n, const PassDesc& p, const DevOp* ops, const double2* gtab,
                                 const double2* btab, cudaStream_t st, size_t smem) {
  if ((int)smem > TileCfg<R, KMAX>::bytes) return cudaErrorInvalidConfiguration;   // not prepared
  const int per_sm = TileCfg<R, KMAX>::per_sm;
  const int sms = sm_count();
  const uint64_t ntiles = 1ull << (n - p.m), total = ntiles * (uint64_t)nstates;
  uint64_t grid = (uint64_t)sms * per_sm;
  if (grid > total) grid = total;
  k_tile<R, KMAX><<<(unsigned)grid, kTileThreads, smem, st>>>((typename GAmp<R>::T*)psi, psis, gstride, bstride, p,
                                                                ops, gtab, btab, brow0, n - p.m, total);
  note_launch();
  return cudaGetLastError();
}

cudaError_t launch_tile_pass_batched(void* psi, void* const* psis, int nstates, int64_t gstride, int64_t bstride,
                                     int64_t brow0, int n, qs_dtype dt, const PassDesc& p, const DevOp* ops,
                                     const double2* gtab, const double2* btab, cudaStream_t st) {
  const size_t smem = tile_smem_bytes(p.m, p.nhigh, p.mbuf_elems, dt);
#define QS_TILE_ARGS psi, psis, nstates, gstride, bstride, brow0, n, p, ops, gtab, btab, st, smem
  if (dt == QS_C64) {
    switch (p.kmax) {
      case 0: case 1: case 2: return launch_tile_t<float, 2>(QS_TILE_ARGS);
      case 3: return launch_tile_t<float, 3>(QS_TILE_ARGS);
      case 4: return launch_tile_t<float, 4>(QS_TILE_ARGS);
      case 5: return launch_tile_t<float, 5>(QS_TILE_ARGS);
      default: return cudaErrorInvalidValue;
    }
  }
  if (p.df) {
    switch (p.kmax) {
      case 0: case 1: case 2: return launch_tile_t<dfl, 2>(QS_TILE_ARGS);
      case 3: return launch_tile_t<dfl, 3>(QS_TILE_ARGS);
      case 4: return launch_tile_t<dfl, 4>(QS_TILE_ARGS);
      case 5: return launch_tile_t<dfl, 5>(QS_TILE_ARGS);
      default: return cudaErrorInvalidValue;
    }
  }
  switch (p.kmax) {
    case 0: case 1: case 2: return launch_tile_t<double, 2>(QS_TILE_ARGS);
    case 3: return launch_tile_t<double, 3>(QS_TILE_ARGS);
    case 4: return launch_tile_t<double, 4>(QS_TILE_ARGS);
    case 5: return launch_tile_t<double, 5>(QS_TILE_ARGS);
    default: return cudaErrorInvalidValue;
  }
#undef QS_TILE_ARGS
}

cudaError_t prepare_tile_pass(const PassDesc& p, qs_dtype dt) {
  const size_t smem = tile_smem_bytes(p.m, p.nhigh, p.mbuf_elems, dt);
  sm_count();
  if (dt == QS_C64) {
    switch (p.kmax) {
      case 0: case 1: case 2: return prepare_tile_t<float, 2>(smem);
      case 3: return prepare_tile_t<float, 3>(smem);
      case 4: return prepare_tile_t<float, 4>(smem);
      case 5: return prepare_tile_t<float, 5>(smem);
      default: return cudaErrorInvalidValue;
    }
  }
  if (p.df) {
    switch (p.kmax) {
      case 0: case 1: case 2: return prepare_tile_t<dfl, 2>(smem);
      case 3: return prepare_tile_t<dfl, 3>(smem);
      case 4: return prepare_tile_t<dfl, 4>(smem);
      case 5: return prepare_tile_t<dfl, 5>(smem);
      default: return cudaErrorInvalidValue;
    }
  }
  switch (p.kmax) {
    case 0: case 1: case 2: return prepare_tile_t<double, 2>(smem);
    case 3: return prepare_tile_t<double, 3>(smem);
    case 4: return prepare_tile_t<double, 4>(smem);
    case 5: return prepare_tile_t<double, 5>(smem);
    default: return cudaErrorInvalidValue;
  }
}

cudaError_t launch_tile_pass(void* psi, int n, qs_dtype dt, const PassDesc& p, const DevOp* ops,
                             const double2* gtab, const double2* btab, int /*threads*/, cudaStream_t st) {
  return launch_tile_pass_batched(psi, nullptr, 1, 0, 0, 0, n, dt, p, ops, gtab, btab, st);
}

// ---------------------------------------------------------------- adjoint gradient, tiled reverse sweep

// gadj[16 j + s] = conjugate transpose of gate j's matrix (2x2 in slots 0-3 or
// 4x4 in slots 0-15), and for one-target gates its angle derivative (slots
// 4-7) unchanged.
__global__ void k_adjoint_table(const DevGate* __restrict__ gates, int ngates, const double2* __restrict__ gtab,
                                double2* __restrict__ gadj) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= ngates) return;
  const double2* m = gtab + (int64_t)j * 16;
  double2* a = gadj + (int64_t)j * 16;
  const int d = gates[j].t1 < 0 ? 2 : 4;
  for (int r = 0; r < d; ++r)
    for (int c = 0; c < d; ++c) a[r * d + c] = make_double2(m[c * d + r].x, -m[c * d + r].y);
  if (d == 2)
    for (int s = 4; s < 8; ++s) a[s] = m[s];
}

// Per-thread part of Re<lam| dG phi> over the amplitudes this thread handled in
// apply_gate_op for the same op (same enumeration, so no barrier is needed).
template <typename R>
__device__ __forceinline__ R adjoint_grad_part(const typename V2<R>::T* tphi, const typename V2<R>::T* tlam, int m,
                                               const DevOp& op, const double2* __restrict__ dmat) {
  using C = typename V2<R>::T;
  const C d00 = from_d<R>(dmat[0]), d01 = from_d<R>(dmat[1]), d10 = from_d<R>(dmat[2]), d11 = from_d<R>(dmat[3]);
  const uint32_t count = 1u << (m - op.nins);
  const uint32_t ta = 1u << op.t0;
  R acc = R(0.0);
  if (op.form == FORM_DIAG1) {   // element-wise enumeration (the target is not inserted)
    for (uint32_t p = threadIdx.x; p < count; p += kTileThreads) {
      const uint32_t b = ins0(p, op.ins, op.nins) | op.cmask;
      const C mm = cmul((b & ta) ? d11 : d00, tphi[b]);
      const C l = tlam[b];
      acc += l.x * mm.x + l.y * mm.y;
    }
  } else {
    for (uint32_t p = threadIdx.x; p < count; p += kTileThreads) {
      const uint32_t b = ins0(p, op.ins, op.nins) | op.cmask;
      const C f0 = tphi[b], f1 = tphi[b | ta];
      const C m0 = cfma(d01, f1, cmul(d00, f0)), m1 = cfma(d11, f1, cmul(d10, f0));
      const C l0 = tlam[b], l1 = tlam[b | ta];
      acc += l0.x * m0.x + l0.y * m0.y + l1.x * m1.x + l1.y * m1.y;
    }
  }
  return acc;
}

// Reverse sweep of the adjoint gradient (Jones and Gacon, arXiv:2009.02823)
// over one tile pass: the ops (single gates of the reversed circuit, tile-local
// positions, commuting gates already reordered by the pass scheduler) act on
// a tile of phi and the same tile of lam held together in shared memory:
// phi <- G^dagger phi, then for a parametric gate Re<lam| dG phi> (the sum over
// amplitudes splits over tiles because dG acts inside the tile), then
// lam <- G^dagger lam. Per-warp FP64 slots collect each op's part over the
// CTA's tiles; partials[row * pcols + CTA] receives the CTA's sum (rows from
// grow[gate], -1 for fixed gates).
template <typename R>
__global__ void __launch_bounds__(kTileThreads) k_adjoint_tile(typename GAmp<R>::T* __restrict__ phi,
                                                                typename GAmp<R>::T* __restrict__ lam, PassDesc p,
                                                                const DevOp* __restrict__ ops,
                                                                const double2* __restrict__ gadj,
                                                                const int32_t* __restrict__ grow, int lg_tiles,
                                                                double* __restrict__ partials, int pcols) {
  using C = typename V2<R>::T;
  using C2 = typename std::conditional<sizeof(R) == 4, float4, double2>::type;   // 16-byte vector
  constexpr int VPT = 16 / sizeof(C);
  constexpr int kAdjIo = 1;   // compute-bound: registers go to occupancy (up to 3 CTAs per SM), not transfers
  constexpr int kWarps = kTileThreads / 32;
  constexpr bool kDF = std::is_same<R, dfl>::value;
  extern __shared__ __align__(16) unsigned char smem[];
  const int m = p.m, L = p.L, nh = p.nhigh;
  const int nops = p.op_end - p.op_begin;
  C* tphi = (C*)smem;
  C* tlam = tphi + (1u << m);
  uint64_t* segoff = (uint64_t*)(tlam + (1u << m));
  C* mbuf = (C*)(segoff + ((1u << nh) < 2 ? 2 : (1u << nh)));
  double* gacc = (double*)(mbuf + (p.mbuf_elems < 16 ? 16 : p.mbuf_elems));   // [nops][kWarps]
  for (uint32_t s = threadIdx.x; s < (1u << nh); s += kTileThreads) {
    uint64_t o = 0;
    for (int k = 0; k < nh; ++k) o |= (uint64_t)((s >> k) & 1u) << p.high[k];
    segoff[s] = o;
  }
  for (int i = threadIdx.x; i < nops * kWarps; i += kTileThreads) gacc[i] = 0;
  __syncthreads();
  const uint32_t size = 1u << m, lmask = (1u << L) - 1;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  for (uint64_t t = blockIdx.x; t < (1ull << lg_tiles); t += gridDim.x) {
    const uint64_t base = insert_zero_bits(t << L, p.high, nh);
    if constexpr (kDF) {
      tile_io_df<true, kAdjIo>(phi, tphi, base, segoff, size, L, lmask);
      tile_io_df<true, kAdjIo>(lam, tlam, base, segoff, size, L, lmask);
    } else {
      tile_io<C, C2, VPT, true, kAdjIo>(phi, tphi, base, segoff, size, L, lmask);
      tile_io<C, C2, VPT, true, kAdjIo>(lam, tlam, base, segoff, size, L, lmask);
    }
    __syncthreads();
    for (int o = p.op_begin; o < p.op_end; ++o) {
      const DevOp op = ops[o];
      apply_gate_op<R>(tphi, m, op, gadj, mbuf);
      const int row = grow[op.mat];
      if (row >= 0) {
        double part = (double)adjoint_grad_part<R>(tphi, tlam, m, op, gadj + (int64_t)op.mat * 16 + 4);
        for (int s = 16; s > 0; s >>= 1) part += __shfl_xor_sync(0xffffffffu, part, s);
        if (lane == 0) gacc[(o - p.op_begin) * kWarps + warp] += part;
      }
      if (op.form == FORM_DENSE2) __syncthreads();   // the matrix buffer is loaded again below
      apply_gate_op<R>(tlam, m, op, gadj, mbuf);
      __syncthreads();
    }
    if constexpr (kDF) {
      tile_io_df<false, kAdjIo>(phi, tphi, base, segoff, size, L, lmask);
      tile_io_df<false, kAdjIo>(lam, tlam, base, segoff, size, L, lmask);
    } else {
      tile_io<C, C2, VPT, false, kAdjIo>(phi, tphi, base, segoff, size, L, lmask);
      tile_io<C, C2, VPT, false, kAdjIo>(lam, tlam, base, segoff, size, L, lmask);
    }
    __syncthreads();
  }
  for (int i = threadIdx.x; i < nops; i += kTileThreads) {
    const int row = grow[ops[p.op_begin + i].mat];
    if (row < 0) continue;
    double s = 0;
    for (int w = 0; w < kWarps; ++w) s += gacc[i * kWarps + w];
    partials[(int64_t)row * pcols + blockIdx.x] = s;
  }
}

size_t adjoint_tile_smem_bytes(const PassDesc& p, qs_dtype dt) {
  const size_t amp = dt == QS_C64 ? 8 : 16;
  const size_t runs = p.nhigh == 0 ? 2 : (1ull << p.nhigh);
  return 2 * (amp << p.m) + 8 * runs + amp * (size_t)(p.mbuf_elems < 16 ? 16 : p.mbuf_elems) +
         sizeof(double) * (kTileThreads / 32) * (size_t)(p.op_end - p.op_begin);
}

template <typename R>
struct AdjCfg {
  static int bytes, per_sm;
};
template <typename R> int AdjCfg<R>::bytes = 0;
template <typename R> int AdjCfg<R>::per_sm = 0;

template <typename R>
static cudaError_t prepare_adjoint_t(size_t smem) {
  if ((int)smem <= AdjCfg<R>::bytes) return cudaSuccess;
  cudaError_t e = cudaFuncSetAttribute(k_adjoint_tile<R>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  int per_sm = 0;
  e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_adjoint_tile<R>, kTileThreads, smem);
  if (e != cudaSuccess) return e;
  if (per_sm < 1) return cudaErrorInvalidConfiguration;
  AdjCfg<R>::bytes = (int)smem;
  AdjCfg<R>::per_sm = per_sm;
  return cudaSuccess;
}

cudaError_t prepare_adjoint_tile(const PassDesc& p, qs_dtype dt) {
  const size_t smem = adjoint_tile_smem_bytes(p, dt);
  if (smem > 227 * 1024) return cudaErrorInvalidValue;
  sm_count();
  if (dt == QS_C64) return prepare_adjoint_t<float>(smem);
  return p.df ? prepare_adjoint_t<dfl>(smem) : prepare_adjoint_t<double>(smem);
}

// Grid of the adjoint tile pass: at most `pcols` CTAs (the partial-sum columns).
cudaError_t launch_adjoint_tile(void* phi, void* lam, int n, qs_dtype dt, const PassDesc& p, const DevOp* ops,
                                const double2* gadj, const int32_t* grow, double* partials, int pcols,
                                cudaStream_t st) {
  const size_t smem = adjoint_tile_smem_bytes(p, dt);
  const int per_sm = dt == QS_C64 ? AdjCfg<float>::per_sm : p.df ? AdjCfg<dfl>::per_sm : AdjCfg<double>::per_sm;
  const int bytes = dt == QS_C64 ? AdjCfg<float>::bytes : p.df ? AdjCfg<dfl>::bytes : AdjCfg<double>::bytes;
  if ((int)smem > bytes || per_sm < 1) return cudaErrorInvalidConfiguration;   // not prepared
  uint64_t grid = (uint64_t)sm_count() * per_sm;
  const uint64_t ntiles = 1ull << (n - p.m);
  if (grid > ntiles) grid = ntiles;
  if (grid > (uint64_t)pcols) grid = pcols;
  if (dt == QS_C64)
    k_adjoint_tile<float><<<(unsigned)grid, kTileThreads, smem, st>>>((float2*)phi, (float2*)lam, p, ops, gadj, grow,
                                                                       n - p.m, partials, pcols);
  else if (p.df)
    k_adjoint_tile<dfl><<<(unsigned)grid, kTileThreads, smem, st>>>((double2*)phi, (double2*)lam, p, ops, gadj, grow,
                                                                     n - p.m, partials, pcols);
  else
    k_adjoint_tile<double><<<(unsigned)grid, kTileThreads, smem, st>>>((double2*)phi, (double2*)lam, p, ops, gadj,
                                                                        grow, n - p.m, partials, pcols);
  note_launch();
  return cudaGetLastError();
}

cudaError_t launch_adjoint_table(const DevGate* gates, int ngates, const double2* gtab, double2* gadj,
                                 cudaStream_t st) {
  if (ngates == 0) return cudaSuccess;
  k_adjoint_table<<<(ngates + 127) / 128, 128, 0, st>>>(gates, ngates, gtab, gadj);
  note_launch();
  return cudaGetLastError();
}

}  // namespace qs
