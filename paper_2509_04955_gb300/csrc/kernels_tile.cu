// Tile passes: the dispatcher over the per-type instances (kernels_tile_f32.cu,
// kernels_tile_f64.cu, kernels_tile_df.cu and kernels_tile_df5.cu; kernel code
// in kernels_tile.cuh) and the adjoint gradient's tiled reverse sweep.
#include "kernels_tile.cuh"

namespace qs {

size_t tile_smem_bytes(int m, int nhigh, int mbuf_elems, qs_dtype dt) {
  const size_t amp = dt == QS_C64 ? 8 : 16;
  const size_t runs = nhigh == 0 ? 2 : (1ull << nhigh);   // padded to 16 bytes
  return (amp << m) + 8 * runs + amp * (size_t)(mbuf_elems < 16 ? 16 : mbuf_elems);
}

size_t tile_pass_smem_bytes(const PassDesc& p, qs_dtype dt) {
  const size_t amp = dt == QS_C64 ? 8 : 16;
  return tile_smem_bytes(p.m, p.nhigh, p.mbuf_elems, dt) + (p.bulk ? (amp << p.m) + 16 : 0);
}

cudaError_t launch_tile_pass_batched(void* psi, void* const* psis, int nstates, int64_t gstride, int64_t bstride,
                                     int64_t brow0, int n, qs_dtype dt, const PassDesc& p, const DevOp* ops,
                                     const double2* gtab, const double2* btab, cudaStream_t st) {
  const size_t smem = tile_pass_smem_bytes(p, dt);
  if (dt == QS_C64) return launch_tile_f32(p.kmax, psi, psis, nstates, gstride, bstride, brow0, n, p, ops, gtab, btab, st, smem);
  if (p.df) return launch_tile_df(p.kmax, psi, psis, nstates, gstride, bstride, brow0, n, p, ops, gtab, btab, st, smem);
  return launch_tile_f64(p.kmax, psi, psis, nstates, gstride, bstride, brow0, n, p, ops, gtab, btab, st, smem);
}

cudaError_t prepare_tile_pass(const PassDesc& p, qs_dtype dt) {
  const size_t smem = tile_pass_smem_bytes(p, dt);
  if (dt == QS_C64) return prepare_tile_f32(p.kmax, p.bulk != 0, smem);
  if (p.df) return prepare_tile_df(p.kmax, false, smem);
  return prepare_tile_f64(p.kmax, p.bulk != 0, smem);
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
