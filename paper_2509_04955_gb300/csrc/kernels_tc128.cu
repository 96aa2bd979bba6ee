// Tensor-core pass for complex128 states: one dense 5-qubit block (32 x 32
// complex, FP64 entries) applied with fp16 tcgen05 MMAs whose products and
// sums are exact, so a pass adds an error of about 2^-46 of the row's norm
// (2^-48 between passes that hand over FP32 pairs) with no FP64 instruction.
//
// A fused block of Section 3.4 on qubits Q (|Q| = 5) is psi'[r, :] = U psi[r, :]
// over the 2^(n-5) rows r (the other bits). Over reals with interleaved
// (re, im) columns this is the real GEMM D[r][n] = sum_k A[r][k] W[k][n],
// K = N = 64, with W the real embedding of U (as in the complex64 pass).
//
// Exact slicing (the error-free splitting of Ozaki, Ogita, Oishi and Rump,
// "Error-free transformations of matrix multiplication", 2012, with the
// fixed-point digits used for fp16 tensor cores): every row of A gets one
// power-of-two scale 2^E with |a| < 2^E for the row's 64 reals, and each a is
// written as 2^(E-8) sum_{i<6} d_i 2^(-9 i) with integer digits |d_i| <= 260;
// each W entry (|w| <= 1) as 2^-8 sum_{j<6} g_j 2^(-9 j), |g_j| <= 256. Digits
// are small integers, exact in fp16, and a digit product is exact in the
// MMA. The products A_i W_j with i + j = l (level l, l <= 5) are accumulated
// in FP32 in tensor memory, one accumulator per level; a level sums at most 6
// products of K = 64 terms of magnitude <= 260 * 256, so levels 0..2 (at most
// 3 products) stay below 2^24 and are exact integers (level 3 too, save for an
// adversarial alignment of all 256 of its digit products, which costs at most
// one unit of level 3); levels 4 and 5 round in FP32 at about 2^-24 of
// themselves, far below the result's last bit. The levels,
// D = 2^(E-16) sum_l acc_l 2^(-9 l), are combined in FP32 pairs (TwoSum) and
// written back as FP64 by their bit patterns. The digit chain, the fold and
// the pair output run on (re, im) at once with the packed FP32 instructions of
// sm_100+ (f32x2), and the A digits are stored negated (one instruction per
// chain step fewer), so the levels hold negated sums, which the fold turns
// back; every result is bit-identical to the scalar steps. What is dropped
// (each FP64 value's mantissa bits below its 47th, W's bits below 2^-54,
// levels above 5) bounds the error of an output by 2^-46 ||a||_2 + 2^(E-49),
// ||a||_2 the 2-norm of its row (Cauchy-Schwarz over a unit column of W) and
// 2^E the row's scale (|a| < 2^E <= 2 max |a|); a row read as FP32 pairs
// (48 bits, no truncation) by 2^-48 ||a||_2 + 2^(E-49).
//
// Pipeline (one persistent CTA per SM, 576 threads, tiles of 128 rows x 32
// columns = 4096 amplitudes = 64 KiB, 12 tile qubits: the block's 5 and the 7
// lowest other qubits):
//   warp 16  producer: cp.async.bulk of the tile's runs (>= 2 KiB each) into
//            one of two 64 KiB landing slots;
//   warps 0-7 converters, thread = (row, column half): the row's exponent (the
//            two halves exchange their maxima), then the six digit planes of
//            the tile: planes 0-3 written to tensor memory with tcgen05.st,
//            planes 4-5 to shared memory (the A operand);
//   warp 17  one thread issues the 21 products x 4 k-steps as 8 instructions
//            per k-step (M = 128, N = 64..256, K = 16, W planes from shared
//            memory) and commits;
//   warps 8-15 drainers, thread = (row, column half): levels 4 and 5 of the
//            thread's columns combined into registers (releasing them), then
//            per 8 columns tcgen05.ld of levels 0-3 (the last load releases
//            them), the fold into an FP32 pair, and the stores to HBM (as FP64
//            or as the pair).
// Tensor memory (512 columns): A digit planes 0-3 at 32 p, level-l
// accumulator at 128 + 64 l (l < 6). Both are single-buffered: a tile's digits
// wait for the previous tile's MMAs (the first 8 columns are computed before
// the wait), its level 4-5 products for the previous tile's levels 4-5 to be
// combined and its other products for the previous tile's levels 0-3 to be
// read; the landing slots keep the loads streaming.
//
// Every wait is bounded (`spin` polls; the waits for copies and MMAs already in
// flight at an abort use kTcSpinLimit): a wait that runs out records *err = 1,
// the CTA stops taking tiles, lets its copies land and its MMAs finish, frees
// its tensor memory and returns.
#include <cuda_fp16.h>
#include <cuda_runtime.h>

#include "qs_internal.h"
#include "tcgen05.cuh"

namespace qs {

constexpr int kT2Warps = 16;                              // converters + drainers
constexpr int kT2Threads = (kT2Warps + 2) * 32;           // + producer warp + MMA warp
constexpr int kT2SlotBytes = 65536;                       // 4096 complex128
constexpr int kT2PlaneBytes = 8192;                       // W digit plane: 64 (N) x 64 (K) fp16, SW128
constexpr int kT2WBytes = 6 * kT2PlaneBytes;              // g_0 .. g_5
constexpr int kT2APlaneBytes = 16384;                     // A digit plane in shared memory: 128 (M) x 64 (K) fp16, SW128
constexpr int kT2ASmem = 2 * kT2APlaneBytes;              // A planes 4 and 5
constexpr uint32_t kT2TmemCols = 512;
constexpr uint32_t kT2AccCol = 128;                       // A planes 0-3 at 32 p, level l at 128 + 64 l
// kind::f16, fp16 A and B, FP32 D, both K-major, N = 64 x nplanes (bits 17-22), M = 128 (bits 24-28)
constexpr uint32_t t2_idesc(int nplanes) {
  return (1u << 4) | ((64u * (uint32_t)nplanes >> 3) << 17) | ((128u >> 4) << 24);
}

__device__ __forceinline__ void t2_mma(uint32_t tmem_d, uint32_t tmem_a, uint64_t b, uint32_t idesc, uint32_t acc) {
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "setp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], [%1], %2, %3, p;\n\t}\n" ::"r"(tmem_d),
      "r"(tmem_a), "l"(b), "r"(idesc), "r"(acc));
}

// The same with A from shared memory (a descriptor, like B).
__device__ __forceinline__ void t2_mma_ss(uint32_t tmem_d, uint64_t a, uint64_t b, uint32_t idesc, uint32_t acc) {
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "setp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(tmem_d),
      "l"(a), "l"(b), "r"(idesc), "r"(acc));
}

// The MMA schedule of a tile (per k-step; every entry runs for the 4 k-steps).
// An entry multiplies A digit plane `a` by `nplanes` consecutive W planes
// starting at `w` (B rows 64 x nplanes: the planes lie back to back in shared
// memory) into as many consecutive level accumulators starting at `level`
// (64 tensor-memory columns each, also back to back), so A_a W_j lands in
// level a + j, for the 21 products with a + j <= 5. An instruction costs about
// the same for any N up to 128 (and 1.4 times that at N = 256), so each A
// plane meets all its W planes in one or two instructions: 8 per k-step. A
// planes 0-3 are read from tensor memory, 4 and 5 from shared memory. Phase H
// writes levels 4-5 only, as soon as the previous tile's levels 4-5 have been
// read; phase L the rest, once the previous tile's levels 0-3 have been read.
// `fresh`: the entry's first k-step overwrites its accumulators (the first
// write of each level in the tile).
struct T2Mma {
  int a, w, nplanes, level, fresh;
};
__device__ constexpr T2Mma kT2PhaseH[] = {{0, 4, 2, 4, 1}, {1, 4, 1, 5, 0}, {4, 0, 2, 4, 0}, {5, 0, 1, 5, 0}};
__device__ constexpr T2Mma kT2PhaseL[] = {{0, 0, 4, 0, 1}, {1, 0, 4, 1, 0}, {2, 0, 4, 2, 0}, {3, 0, 3, 3, 0}};

__device__ __forceinline__ void tmem_st8(uint32_t taddr, const uint32_t* v) {
  asm volatile("tcgen05.st.sync.aligned.32x32b.x8.b32 [%0], {%1,%2,%3,%4,%5,%6,%7,%8};" ::"r"(taddr), "r"(v[0]),
               "r"(v[1]), "r"(v[2]), "r"(v[3]), "r"(v[4]), "r"(v[5]), "r"(v[6]), "r"(v[7])
               : "memory");
}

// Loads 8 columns (this thread's lane); the caller waits with tcgen05.wait::ld.
__device__ __forceinline__ void tmem_ld8(uint32_t taddr, uint32_t* r) {
  asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
               : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7])
               : "r"(taddr));
}

constexpr float kT2Magic = 12582912.0f;   // 1.5 * 2^23: x + it rounds x to an integer (|x| < 2^22)

// Loads 16 columns (this thread's lane); the caller waits with tcgen05.wait::ld.
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, uint32_t* r) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]),
        "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
      : "r"(taddr));
}

// The start of the six digits of one FP64 value a (bit pattern whi:wlo) of a
// row whose biased-exponent maximum is emax_b (fe_off = 134 - emax_b):
// s = a 2^(8 - E), E = emax_b - 1022, so |s| < 256, and s ~ sum_{i<6} d_i
// 2^(-9 i); the error is below 2^-39 (the 6 FP64 mantissa bits the split drops) and
// 2^-46. The FP64 mantissa is cut by bits into hi (sign, exponent, top 23
// stored bits) and lo18 (the next 23 bits, pre-scaled by 2^18); the digit
// chain (t2_nchain2) takes digits from hi with exact FP32 steps until hi is
// used up, lo18 joins at digit 2. Values with |s| < 2^-40 (and FP64 zeros /
// subnormals) give zero digits.
__device__ __forceinline__ void t2_hilo(uint32_t whi, uint32_t wlo, int fe_off, float& hi, float& lo18) {
  const uint32_t ex = (whi >> 20) & 0x7ffu;
  const int fe = (int)ex + fe_off;              // biased FP32 exponent of s (<= 134)
  const uint32_t se = (whi & 0x80000000u) | ((uint32_t)fe << 23);
  hi = __uint_as_float(se | (__funnelshift_l(wlo, whi, 3) & 0x7fffffu));
  // lo = m 2^(e_s - 46) with m the remainder's top 23 bits: X - 2^x with
  // X = (1 + m 2^-23) 2^x, x = e_s - 23; pre-scaled by 2^18: x = e_s - 5
  const uint32_t eb = se - (5u << 23);
  lo18 = __fsub_rn(__uint_as_float(eb | ((wlo & 0x1fffffffu) >> 6)), __uint_as_float(eb));
  const bool ok = ex != 0 && fe >= 87;
  hi = ok ? hi : 0.f;
  lo18 = ok ? lo18 : 0.f;
}

// The digit chain on (re, im) at once with packed FP32 instructions, from hi
// (|hi| < 256) and lo18 (the next bits, scaled by 2^18): nd[i] = -d_i, the
// digits negated. Every step is the exact negation of
// rounding to an integer by x + 1.5 2^23 - 1.5 2^23 and of the exact
// residual fma(t, 512, -d): u = t 512 + M holds M + d, M - u = -d is exact,
// and fma(t, 512, -d) continues the chain, one packed instruction each. The
// pass stores the negated digits: every digit product, and so every level,
// changes sign, which the drainers undo when they fold the levels.
__device__ __forceinline__ void t2_nchain2(float2 hi, float2 lo18, float2* nd) {
  const float2 M = make_float2(kT2Magic, kT2Magic), N1 = make_float2(-1.f, -1.f);
  const float2 C512 = make_float2(512.f, 512.f);
  float2 u = __fadd2_rn(hi, M);
  nd[0] = __ffma2_rn(u, N1, M);
  float2 t = __fadd2_rn(hi, nd[0]);                       // hi - d0, exact, |t| <= 1/2
  u = __ffma2_rn(t, C512, M);
  nd[1] = __ffma2_rn(u, N1, M);
  t = __ffma2_rn(t, C512, nd[1]);                         // exact
  u = __fadd2_rn(__ffma2_rn(t, C512, lo18), M);
  nd[2] = __ffma2_rn(u, N1, M);
  t = __fadd2_rn(__ffma2_rn(t, C512, nd[2]), lo18);
  u = __ffma2_rn(t, C512, M);
  nd[3] = __ffma2_rn(u, N1, M);
  t = __ffma2_rn(t, C512, nd[3]);
  u = __ffma2_rn(t, C512, M);
  nd[4] = __ffma2_rn(u, N1, M);
  t = __ffma2_rn(t, C512, nd[4]);
  u = __ffma2_rn(t, C512, M);
  nd[5] = __ffma2_rn(u, N1, M);
}

// The same six digits (negated) of (re, im) held as FP32 pairs s + e (|e| <=
// ulp(s) / 2) of a row with scale 2^E: hi = s 2^(8-E) and lo18 = e 2^(26-E)
// (sc8 = 2^(8-E), sc26 = 2^(26-E), exact power-of-two scalings; tiny values
// flush to zero).
__device__ __forceinline__ void t2_ndigits_pair2(float2 s, float2 e, float2 sc8, float2 sc26, float2* nd) {
  t2_nchain2(__fmul2_rn(s, sc8), __fmul2_rn(e, sc26), nd);
}

// 2^k as a float (-126 <= k <= 127)
__device__ __forceinline__ float t2_pow2(int k) { return __uint_as_float((uint32_t)(k + 127) << 23); }

// (s, e) += c sc on (re, im) at once, with TwoSum (s + e = a + b exactly, b =
// c sc formed inside the FMAs; -bb = a - s, the exact negation of s - a)
__device__ __forceinline__ void t2_absorb2(float2& s, float2& e, float2 c, float2 sc) {
  const float2 N1 = make_float2(-1.f, -1.f);
  const float2 a = s;
  s = __ffma2_rn(c, sc, a);
  const float2 nbb = __ffma2_rn(s, N1, a);
  const float2 x1 = __ffma2_rn(__fadd2_rn(s, nbb), N1, a);   // a - (s - bb)
  const float2 x2 = __ffma2_rn(c, sc, nbb);                   // b - bb
  e = __fadd2_rn(e, __fadd2_rn(x1, x2));
}

// FP64 value 2^(E - 16) (s + e) of an FP32 pair, normalised first with a
// FastTwoSum, built by integer arithmetic on s's widened bit pattern with e
// added in units of 2^-46 of s; below 2^-1022 it flushes to zero.
__device__ __forceinline__ double t2_join(float s, float e, int E) {
  const int emax_b = E + 1022;
  const float s2 = __fadd_rn(s, e);             // FastTwoSum: |s| >= |e| after the level sums
  e = __fsub_rn(e, __fsub_rn(s2, s));
  s = s2;
  const uint32_t us = __float_as_uint(s);
  const int fs = (int)((us >> 23) & 0xffu);     // biased FP32 exponent of s
  const int de = fs + emax_b - 142;             // biased FP64 exponent of the result
  if (fs == 0 || de <= 0) return 0.0;           // |result| < 2^-1022 (or s = 0): flushed
  long long mag = ((long long)de << 52) | ((long long)(us & 0x7fffffu) << 29);
  if (fs >= 46 && fs <= 254) {
    // e in units of 2^(x_s - 46), x_s = fs - 127: |k| <= 2^22
    const float sc = __uint_as_float((uint32_t)(300 - fs) << 23);
    const int k = __float_as_int(__fmaf_rn(e, sc, kT2Magic)) - 0x4B400000;
    long long adj = (long long)((us >> 31) ? -k : k) << 6;   // in units of s's FP64 ulp
    if ((us & 0x7fffffu) == 0 && adj < 0) adj *= 2;        // below a power of two the ulp halves
    mag += adj;
  }
  return __longlong_as_double((long long)((unsigned long long)(us >> 31) << 63) | mag);
}

// PIN / POUT: the pass reads / writes the state as FP32 pairs (the form kept
// between consecutive tensor-core passes: per amplitude the floats
// re.s, im.s, re.e, im.e with value s + e, |e| <= ulp(s) / 2), else as FP64.
template <bool MULTI, bool PIN, bool POUT>
__global__ void __launch_bounds__(kT2Threads, 1)
    k_tc128(double2* __restrict__ psi0, void* const* __restrict__ psis, Tc5PassDesc p,
            const uint4* __restrict__ wimg, int64_t wstride16, int lg_tiles1, uint64_t ntiles,
            int* __restrict__ err, uint32_t spin) {
  extern __shared__ __align__(1024) unsigned char t2_smem_raw[];
  unsigned char* smem = (unsigned char*)(((uintptr_t)t2_smem_raw + 1023) & ~(uintptr_t)1023);
  unsigned char* slots = smem;                                  // 2 x 64 KiB
  unsigned char* W = smem + 2 * kT2SlotBytes;                   // 6 W digit planes
  unsigned char* A45 = W + kT2WBytes;                           // A digit planes 4 and 5
  uint64_t* tbase = (uint64_t*)(A45 + kT2ASmem);                // 4 x 256: tile number byte -> offset
  uint64_t* runoff = tbase + 4 * 256;                           // 32: global offset of run j
  uint64_t* coff = runoff + 32;                                 // 32: global offset of column c
  uint32_t* lamcol = (uint32_t*)(coff + 32);                    // 32: tile-local index of column c
  int32_t* xe = (int32_t*)(lamcol + 32);                        // [2][128][2]: half-row exponent maxima
  int32_t* etab = xe + 2 * 128 * 2;                             // [2][128]: row scale exponents E
  int32_t* qpos = etab + 2 * 128;                               // tile[12], row[7], col[5], p, kq
  // full[2] empty[2] afull mdone dfree efull[2] wfull wfree xbar[2][4] dfree45
  uint64_t* bar = (uint64_t*)(qpos + 26);
  uint32_t* tmem_slot = (uint32_t*)(bar + 20);
  __shared__ int s_abort;

  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  int32_t* s_tile = qpos;
  int32_t* s_row = qpos + 12;
  int32_t* s_col = qpos + 19;
  if (tid == 0) {
    for (int k = 0; k < 12; ++k) s_tile[k] = p.tile[k];
    for (int k = 0; k < 7; ++k) s_row[k] = p.row[k];
    for (int k = 0; k < 5; ++k) s_col[k] = p.col[k];
    int pp = 0;
    while (pp < 12 && p.tile[pp] == pp) ++pp;
    qpos[24] = pp;
    // how many of the three lowest tile qubits are row qubits (the others are
    // the lowest block qubits): the slot's bank group of an element is its
    // tile-local index mod 8, so a warp reading one column for 32 rows sees
    // only 2^kq of the 8 groups
    int kq = 0;
    for (int t = 0; t < 3; ++t) {
      bool is_col = false;
      for (int b = 0; b < 5; ++b) is_col |= p.col[b] == p.tile[t];
      kq += is_col ? 0 : 1;
    }
    qpos[25] = kq;
    s_abort = 0;
    // arrivals: full, wfull, wfree, mdone: 1 (expect_tx / commit); empty, afull, dfree, efull, dfree45:
    // one per warp of 8; xbar (row-exponent exchange of converter warps quad and quad + 4): 2
    const uint32_t cnt[20] = {1, 1, 8, 8, 8, 1, 8, 8, 8, 1, 1, 2, 2, 2, 2, 2, 2, 2, 2, 8};
    for (int i = 0; i < 20; ++i)
      asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar + i)), "r"(cnt[i]));
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  const uint64_t tmask1 = (1ull << lg_tiles1) - 1;
  const bool contig = MULTI && wstride16 != 0;
  const uint64_t chunk_t = (ntiles + gridDim.x - 1) / gridDim.x;
  const uint64_t t_begin = contig ? (uint64_t)blockIdx.x * chunk_t : blockIdx.x;
  const uint64_t tstep = contig ? 1 : gridDim.x;
  const uint64_t t_end = contig ? (t_begin + chunk_t < ntiles ? t_begin + chunk_t : ntiles) : ntiles;
  const uint64_t my = t_begin < t_end ? (t_end - t_begin + tstep - 1) / tstep : 0;
  if (my > 0) {   // a trailing CTA can get an empty range that starts past the last state
    const uint4* w0 = wimg + (contig ? (int64_t)(t_begin >> lg_tiles1) * wstride16 : 0);
    for (int i = tid; i < kT2WBytes / 16; i += kT2Threads) ((uint4*)W)[i] = w0[i];
  }
  __syncthreads();
  const int pr = qpos[24];            // log2 of the run length in amplitudes (7..12)
  const int nruns = 1 << (12 - pr);
  auto lam_of = [&](int q) {          // position of qubit q among the 12 tile qubits
    int l = 0;
    while (l < 11 && s_tile[l] != q) ++l;
    return l;
  };
  for (int e = tid; e < 4 * 256; e += kT2Threads) {
    uint64_t x = (uint64_t)(e & 255) << (8 * (e >> 8));
    for (int k = 0; k < 12; ++k) {
      const int q = s_tile[k];
      x = ((x >> q) << (q + 1)) | (x & ((1ull << q) - 1));
    }
    tbase[e] = x;
  }
  if (tid < 32) {
    uint64_t o = 0;
    uint32_t lc = 0;
    for (int b = 0; b < 5; ++b) {
      o |= (uint64_t)((tid >> b) & 1) << s_col[b];
      lc |= (uint32_t)((tid >> b) & 1) << lam_of(s_col[b]);
    }
    coff[tid] = o;
    lamcol[tid] = lc;
    if (tid < nruns) {
      uint64_t r = 0;
      for (int b = 0; b < 12 - pr; ++b) r |= (uint64_t)((tid >> b) & 1) << s_tile[pr + b];
      runoff[tid] = r;
    }
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                 "r"(kT2TmemCols)
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
  uint64_t* mdone = bar + 5;
  uint64_t* dfree = bar + 6;      // levels 0-3 of the accumulators read
  uint64_t* efull = bar + 7;
  uint64_t* wfull = bar + 9;
  uint64_t* wfree = bar + 10;     // completes when the MMAs on a state's W planes are done
  uint64_t* xbar = bar + 11;      // [parity][quad]
  uint64_t* dfree45 = bar + 19;   // levels 4-5 read (combined and held in registers by the drainers)
  auto tile_of = [&](uint64_t i) -> uint64_t { return t_begin + i * tstep; };
  auto state_ptr = [&](uint64_t tt) -> double2* {
    if constexpr (MULTI) return (double2*)psis[tt >> lg_tiles1];
    else return psi0;
  };
  auto new_state = [&](uint64_t i) -> bool {
    return contig && i > 0 && (tile_of(i) >> lg_tiles1) != (tile_of(i - 1) >> lg_tiles1);
  };
  auto fail = [&](int code) {
    atomicExch(err, code);
    *(volatile int*)&s_abort = 1;
  };
  auto tile_base = [&](uint64_t t) -> uint64_t {
    return tbase[t & 255] | tbase[256 + ((t >> 8) & 255)] | tbase[512 + ((t >> 16) & 255)] |
           tbase[768 + ((t >> 24) & 255)];
  };

  if (warp == kT2Warps) {
    // ---------------- producer: bulk copies of tile runs into the slots
    const uint32_t runb = 16u << pr;
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
                     "r"((uint32_t)kT2SlotBytes)
                     : "memory");
      __syncwarp();
      const uint64_t tt = tile_of(i);
      const double2* src = state_ptr(tt) + tile_base(tt & tmask1);
      for (int j = lane; j < nruns; j += 32)
        asm volatile(
            "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                smem_u32(slots + s * kT2SlotBytes + j * runb)),
            "l"(src + runoff[j]), "r"(runb), "r"(smem_u32(full + s))
            : "memory");
      if (new_state(i)) {
        // W planes of the next state once the MMAs of tile i - 1 (the last on the
        // old planes) are done: wfree completes once per state boundary.
        if (!mbar_wait_warp(smem_u32(wfree), (uint32_t)(w_issued & 1), spin)) {
          if (lane == 0) fail(1);
          ++i;   // tile i's copies are in flight
          break;
        }
        if (lane == 0) {
          asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(wfull)),
                       "r"((uint32_t)kT2WBytes)
                       : "memory");
          asm volatile(
              "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                  smem_u32(W)),
              "l"(wimg + (int64_t)(tt >> lg_tiles1) * wstride16), "r"((uint32_t)kT2WBytes), "r"(smem_u32(wfull))
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
  } else if (warp == kT2Warps + 1) {
    // ---------------- MMA issue (one thread): level l = i + j gets A_i W_j (i + j <= 5)
    if (lane == 0) {
      const uint32_t wb = smem_u32(W), ab = smem_u32(A45);
      auto issue = [&](const T2Mma& m) {
#pragma unroll
        for (int ks = 0; ks < 4; ++ks) {
          const uint32_t d = tmem + kT2AccCol + 64 * m.level, acc = (m.fresh && ks == 0) ? 0u : 1u;
          const uint64_t b = smem_desc(wb + m.w * kT2PlaneBytes + 32 * ks);
          if (m.a < 4) t2_mma(d, tmem + 32 * m.a + 8 * ks, b, t2_idesc(m.nplanes), acc);
          else t2_mma_ss(d, smem_desc(ab + (m.a - 4) * kT2APlaneBytes + 32 * ks), b, t2_idesc(m.nplanes), acc);
        }
      };
      uint64_t i = 0, w_seen = 0;
      for (; i < my; ++i) {
        if (*(volatile int*)&s_abort) break;
        if (new_state(i)) {
          if (!mbar_wait(smem_u32(wfull), (uint32_t)(w_seen & 1), spin)) { fail(1); break; }
          ++w_seen;
        }
        if (!mbar_wait(smem_u32(afull), (uint32_t)(i & 1), spin)) { fail(1); break; }
        if (i >= 1 && !mbar_wait(smem_u32(dfree45), (uint32_t)((i - 1) & 1), spin)) { fail(1); break; }
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
#pragma unroll
        for (int e = 0; e < (int)(sizeof(kT2PhaseH) / sizeof(T2Mma)); ++e) issue(kT2PhaseH[e]);
        if (i >= 1 && !mbar_wait(smem_u32(dfree), (uint32_t)((i - 1) & 1), spin)) {
          mma_commit(smem_u32(mdone));   // the issued MMAs complete before the abort drain below
          ++i;
          fail(1);
          break;
        }
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
#pragma unroll
        for (int e = 0; e < (int)(sizeof(kT2PhaseL) / sizeof(T2Mma)); ++e) issue(kT2PhaseL[e]);
        mma_commit(smem_u32(mdone));
        if (i + 1 < my && new_state(i + 1)) mma_commit(smem_u32(wfree));   // last tile on these planes
      }
      // MMAs still in flight after an abort complete before the memory is released
      if (i > 0 && *(volatile int*)&s_abort) mbar_wait(smem_u32(mdone), (uint32_t)((i - 1) & 1));
    }
  } else {
    // ---------------- warps 0-15: thread = (row, column half h: complex columns 16h .. 16h + 15)
    const bool converter = warp < kT2Warps / 2;
    const int w8 = converter ? warp : warp - kT2Warps / 2;
    const int quad = w8 & 3, h = w8 >> 2;
    const int row = quad * 32 + lane;
    const uint32_t tq = (uint32_t)(quad * 32) << 16;
    bool ok = true;
    if (converter) {
      uint32_t lrow = 0;
      for (int b = 0; b < 7; ++b) lrow |= (uint32_t)((row >> b) & 1) << lam_of(s_row[b]);
      // Column skew: lane l reads column j ^ sg at step j, sg taken from the
      // lane bits above the kq row bits, so the block bits among the three
      // lowest tile bits vary across the lanes too and every 8 lanes cover the
      // 8 bank groups; the digit pass undoes the skew in registers.
      const int kq = qpos[25], mbits = 3 - kq;
      const uint32_t sg = ((uint32_t)lane >> kq) & ((1u << mbits) - 1u);
      const unsigned char* sl0 = slots;
      for (uint64_t i = 0; i < my; ++i) {
        if (__any_sync(0xffffffffu, *(volatile int*)&s_abort)) break;
        const int s = (int)(i & 1), par = (int)(i & 1);
        if (!mbar_wait_warp(smem_u32(full + s), (uint32_t)((i >> 1) & 1), spin)) { ok = false; break; }
        const unsigned char* sl = sl0 + s * kT2SlotBytes;
        // the row's exponent: maximum biased exponent over its 64 reals (of the
        // FP64 values, or of the pairs' leading floats)
        int em = 0;
#pragma unroll 4
        for (int j = 0; j < 16; ++j) {
          const uint4 v = *(const uint4*)(sl + 16u * (lrow | lamcol[16 * h + (j ^ (int)sg)]));
          if constexpr (PIN) {
            em = max(em, (int)((v.x >> 23) & 0xffu));
            em = max(em, (int)((v.y >> 23) & 0xffu));
          } else {
            em = max(em, (int)((v.y >> 20) & 0x7ffu));
            em = max(em, (int)((v.w >> 20) & 0x7ffu));
          }
        }
        // exchange with the warp holding the other half of the same rows (bounded
        // wait, no named barrier: a warp that aborts must not leave its partner stuck)
        xe[(par * 128 + row) * 2 + h] = em;
        __syncwarp();
        if (lane == 0) mbar_arrive(smem_u32(xbar + par * 4 + quad));
        if (!mbar_wait_warp(smem_u32(xbar + par * 4 + quad), (uint32_t)((i >> 1) & 1), spin)) { ok = false; break; }
        em = max(em, xe[(par * 128 + row) * 2 + (h ^ 1)]);
        // row scale 2^E, |a| < 2^E; E >= -101 keeps every scale below a float
        const int E = max(PIN ? em - 126 : em - 1022, -101);
        const int fe_off = -888 - E;                    // FP64 input: biased exponent offset of s
        const float2 sc8 = make_float2(t2_pow2(8 - E), t2_pow2(8 - E));     // pair input
        const float2 sc26 = make_float2(t2_pow2(26 - E), t2_pow2(26 - E));
#pragma unroll 1
        for (int c8 = 0; c8 < 2; ++c8) {
          // digits of 8 columns; the first 8 while the previous tile's MMAs may
          // still read the A planes
          uint32_t pl[6][8];
          uint4 vv[8];
#pragma unroll
          for (int j = 0; j < 8; ++j) vv[j] = *(const uint4*)(sl + 16u * (lrow | lamcol[16 * h + 8 * c8 + (j ^ (int)sg)]));
          // vv[j] holds column 8 c8 + (j ^ sg): swap back, one bit of sg at a time
#pragma unroll
          for (int b = 0; b < 3; ++b) {
            if (b < mbits) {
              const bool sw = (sg >> b) & 1u;
#pragma unroll
              for (int j = 0; j < 8; ++j)
                if (!(j & (1 << b))) {
                  const uint4 x = vv[j], y = vv[j | (1 << b)];
                  vv[j] = sw ? y : x;
                  vv[j | (1 << b)] = sw ? x : y;
                }
            }
          }
#pragma unroll
          for (int j = 0; j < 8; ++j) {
            const uint4 v = vv[j];
            float2 nd[6];
            if constexpr (PIN) {
              t2_ndigits_pair2(make_float2(__uint_as_float(v.x), __uint_as_float(v.y)),
                               make_float2(__uint_as_float(v.z), __uint_as_float(v.w)), sc8, sc26, nd);
            } else {
              float2 hi, lo18;
              t2_hilo(v.y, v.x, fe_off, hi.x, lo18.x);
              t2_hilo(v.w, v.z, fe_off, hi.y, lo18.y);
              t2_nchain2(hi, lo18, nd);
            }
#pragma unroll
            for (int q = 0; q < 6; ++q) {
              const __half2 hv = __float22half2_rn(nd[q]);
              pl[q][j] = *(const uint32_t*)&hv;
            }
          }
          if (c8 == 0) {
            // A planes are free once the previous tile's MMAs are done; that also
            // means the drainers of tile i - 2 (same parity) have read their
            // exponents (they release the accumulators the MMAs of tile i - 1
            // need only after reading them), so this tile's may take their place.
            if (i >= 1 && !mbar_wait_warp(smem_u32(mdone), (uint32_t)((i - 1) & 1), spin)) { ok = false; break; }
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            if (h == 0) etab[par * 128 + row] = E;
            __syncwarp();
            if (lane == 0) mbar_arrive(smem_u32(efull + par));
          }
#pragma unroll
          for (int q = 0; q < 4; ++q) tmem_st8(tmem + tq + 32 * q + 16 * h + 8 * c8, pl[q]);
          // planes 4 and 5 into shared memory: this thread's row, 16-byte chunks
          // 4h + 2c8 and 4h + 2c8 + 1 of its 128-byte K run, 128-byte swizzle
#pragma unroll
          for (int q = 4; q < 6; ++q) {
            unsigned char* ap = A45 + (q - 4) * kT2APlaneBytes + row * 128;
            const int c0 = 4 * h + 2 * c8;
            *(uint4*)(ap + ((c0 ^ (row & 7)) << 4)) = make_uint4(pl[q][0], pl[q][1], pl[q][2], pl[q][3]);
            *(uint4*)(ap + (((c0 + 1) ^ (row & 7)) << 4)) = make_uint4(pl[q][4], pl[q][5], pl[q][6], pl[q][7]);
          }
        }
        if (!ok) break;
        asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory");
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");   // A planes 4-5 are read by the MMA
        asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
        __syncwarp();
        if (lane == 0) {
          mbar_arrive(smem_u32(empty + s));
          mbar_arrive(smem_u32(afull));
        }
      }
    } else {
      uint64_t roff = 0;
      for (int b = 0; b < 7; ++b) roff |= (uint64_t)((row >> b) & 1) << s_row[b];
      for (uint64_t i = 0; i < my; ++i) {
        if (__any_sync(0xffffffffu, *(volatile int*)&s_abort)) break;
        const int par = (int)(i & 1);
        if (!mbar_wait_warp(smem_u32(mdone), (uint32_t)(i & 1), spin)) { ok = false; break; }
        if (!mbar_wait_warp(smem_u32(efull + par), (uint32_t)((i >> 1) & 1), spin)) { ok = false; break; }
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        const int E = etab[par * 128 + row];
        const float osc = t2_pow2(E - 16);   // pair output scale
        const uint64_t tt = tile_of(i);
        double2* __restrict__ psi = state_ptr(tt);
        const uint64_t rb = tile_base(tt & tmask1) | roff;
        // levels 4 and 5 of this thread's 32 columns first, combined into one
        // FP32 value per column (t = -(2^-36 L4 + 2^-45 L5), the levels holding
        // negated sums), which releases them to the next tile's phase H; then
        // per 8 columns levels 0-3 folded with t into an FP32 pair and stored
        const uint32_t col0 = tmem + tq + kT2AccCol + 32 * h;
        float t45[32];
        {
          uint32_t l4[32], l5[32];
          tmem_ld16(col0 + 64 * 4, l4);
          tmem_ld16(col0 + 64 * 4 + 16, l4 + 16);
          tmem_ld16(col0 + 64 * 5, l5);
          tmem_ld16(col0 + 64 * 5 + 16, l5 + 16);
          asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
          asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
          __syncwarp();
          if (lane == 0) mbar_arrive(smem_u32(dfree45));
#pragma unroll
          for (int k = 0; k < 32; k += 2) {
            const float2 v4 = make_float2(__uint_as_float(l4[k]), __uint_as_float(l4[k + 1]));
            const float2 v5 = make_float2(__uint_as_float(l5[k]), __uint_as_float(l5[k + 1]));
            const float2 t = __ffma2_rn(v5, make_float2(-2.842170943040401e-14f, -2.842170943040401e-14f),
                                        __fmul2_rn(v4, make_float2(-1.4551915228366852e-11f, -1.4551915228366852e-11f)));
            t45[k] = t.x;
            t45[k + 1] = t.y;
          }
        }
#pragma unroll
        for (int c4 = 0; c4 < 4; ++c4) {
          const uint32_t col = col0 + 8 * c4;
          uint32_t a[4][8];
#pragma unroll
          for (int l = 0; l < 4; ++l) tmem_ld8(col + 64 * l, a[l]);
          asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
          if (c4 == 3) {   // levels 0-3 read; the last fold and stores follow
            asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
            __syncwarp();
            if (lane == 0) mbar_arrive(smem_u32(dfree));
          }
#pragma unroll
          for (int k = 0; k < 8; k += 2) {
            // the levels hold the negated sums (the A digits are negated)
            auto lv = [&](int l) { return make_float2(__uint_as_float(a[l][k]), __uint_as_float(a[l][k + 1])); };
            float2 sk = __fmul2_rn(lv(0), make_float2(-1.f, -1.f));
            float2 ek = make_float2(t45[8 * c4 + k], t45[8 * c4 + k + 1]);
            t2_absorb2(sk, ek, lv(1), make_float2(-0.001953125f, -0.001953125f));
            t2_absorb2(sk, ek, lv(2), make_float2(-3.814697265625e-06f, -3.814697265625e-06f));
            t2_absorb2(sk, ek, lv(3), make_float2(-7.450580596923828e-09f, -7.450580596923828e-09f));
            double2* dst = psi + (rb | coff[16 * h + 4 * c4 + (k >> 1)]);
            if constexpr (POUT) {
              const float2 t2 = __fadd2_rn(sk, ek);                                   // FastTwoSum
              const float2 f2 = __fadd2_rn(ek, __ffma2_rn(t2, make_float2(-1.f, -1.f), sk));   // e - (t - s)
              const float2 osc2 = make_float2(osc, osc);
              const float2 o1 = __fmul2_rn(t2, osc2), o2 = __fmul2_rn(f2, osc2);
              *(float4*)dst = make_float4(o1.x, o1.y, o2.x, o2.y);
            } else {
              double2 o;
              o.x = t2_join(sk.x, ek.x, E);
              o.y = t2_join(sk.y, ek.y, E);
              *dst = o;
            }
          }
        }
      }
    }
    if (!ok && lane == 0) fail(1);
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (warp == 0)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kT2TmemCols) : "memory");
}

size_t tc128_smem_bytes() {
  return 2 * (size_t)kT2SlotBytes + kT2WBytes + kT2ASmem + 4 * 256 * 8 + 32 * 8 * 2 + 32 * 4 + 2 * 128 * 2 * 4 + 2 * 128 * 4 +
         26 * 4 + 20 * 8 + 16 + 1024;
}

static bool g_tc128_ready = false;
static int g_tc128_sms = 0;

// Host-side set-up (outside any stream capture): shared-memory attribute and SM count.
template <bool MULTI, bool PIN, bool POUT>
static cudaError_t set_tc128_attribute(int smem) {
  return cudaFuncSetAttribute(k_tc128<MULTI, PIN, POUT>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
}

cudaError_t prepare_tc128_pass() {
  if (g_tc128_ready) return cudaSuccess;
  const int smem = (int)tc128_smem_bytes();
  cudaError_t e = set_tc128_attribute<false, false, false>(smem);
  if (e == cudaSuccess) e = set_tc128_attribute<false, false, true>(smem);
  if (e == cudaSuccess) e = set_tc128_attribute<false, true, false>(smem);
  if (e == cudaSuccess) e = set_tc128_attribute<false, true, true>(smem);
  if (e == cudaSuccess) e = set_tc128_attribute<true, false, false>(smem);
  if (e == cudaSuccess) e = set_tc128_attribute<true, false, true>(smem);
  if (e == cudaSuccess) e = set_tc128_attribute<true, true, false>(smem);
  if (e == cudaSuccess) e = set_tc128_attribute<true, true, true>(smem);
  if (e != cudaSuccess) return e;
  g_tc128_sms = device_sm_count();
  g_tc128_ready = true;
  return cudaSuccess;
}

template <bool MULTI, bool PIN, bool POUT>
static void launch_tc128_instance(unsigned grid, size_t smem, cudaStream_t st, double2* psi, void* const* psis,
                                  const Tc5PassDesc& p, const uint4* w, int64_t ws16, int lg, uint64_t ntiles, int* err,
                                  uint32_t spin) {
  k_tc128<MULTI, PIN, POUT><<<grid, kT2Threads, smem, st>>>(psi, psis, p, w, ws16, lg, ntiles, err, spin);
}

cudaError_t launch_tc128_pass(void* psi, void* const* psis, int nstates, int64_t wstride, int n,
                              const Tc5PassDesc& p, const void* wimg, int* err, cudaStream_t st, uint32_t spin) {
  if (!g_tc128_ready) return cudaErrorInvalidConfiguration;   // not prepared
  if (n < 12) return cudaErrorInvalidValue;
  if (spin == 0) spin = kTcSpinLimit;
  const uint64_t ntiles = (1ull << (n - 12)) * (uint64_t)nstates;
  const unsigned grid = (unsigned)(ntiles < (uint64_t)g_tc128_sms ? ntiles : (uint64_t)g_tc128_sms);
  const size_t smem = tc128_smem_bytes();
  const uint4* w = (const uint4*)wimg;
  const int64_t ws16 = wstride / 8;   // uint16 elements -> uint4
  double2* ps = (double2*)psi;
  const int lg = n - 12;
  const int fmt = (p.in_pairs ? 1 : 0) | (p.out_pairs ? 2 : 0);
  if (psis != nullptr) {
    if (fmt == 0) launch_tc128_instance<true, false, false>(grid, smem, st, nullptr, psis, p, w, ws16, lg, ntiles, err, spin);
    else if (fmt == 1) launch_tc128_instance<true, true, false>(grid, smem, st, nullptr, psis, p, w, ws16, lg, ntiles, err, spin);
    else if (fmt == 2) launch_tc128_instance<true, false, true>(grid, smem, st, nullptr, psis, p, w, ws16, lg, ntiles, err, spin);
    else launch_tc128_instance<true, true, true>(grid, smem, st, nullptr, psis, p, w, ws16, lg, ntiles, err, spin);
  } else {
    if (fmt == 0) launch_tc128_instance<false, false, false>(grid, smem, st, ps, nullptr, p, w, ws16, lg, ntiles, err, spin);
    else if (fmt == 1) launch_tc128_instance<false, true, false>(grid, smem, st, ps, nullptr, p, w, ws16, lg, ntiles, err, spin);
    else if (fmt == 2) launch_tc128_instance<false, false, true>(grid, smem, st, ps, nullptr, p, w, ws16, lg, ntiles, err, spin);
    else launch_tc128_instance<false, true, true>(grid, smem, st, ps, nullptr, p, w, ws16, lg, ntiles, err, spin);
  }
  note_launch();
  return cudaGetLastError();
}

}  // namespace qs
