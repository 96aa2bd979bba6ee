// Internal declarations shared by the host runtime (C++) and the CUDA kernels.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "qsim_gb300.h"

#ifdef __CUDACC__
#define QS_HD __host__ __device__ __forceinline__
#else
#define QS_HD inline
#endif

namespace qs {

constexpr int kMaxQubits = 40;
constexpr int kMaxControls = 2;
constexpr int kMaxBlockQubits = 6;   // dense block width handled by any kernel

// ---------------------------------------------------------------------------
// Gate descriptors as the kernels see them. Matrices live in a device table of
// FP64 complex entries (16 per gate: 2x2 uses the first 4); parametric entries
// are filled on the device from theta by k_resolve (one table per batch row).

enum GateForm : int32_t {
  FORM_DENSE1 = 0,   // 2x2 general on one target
  FORM_ANTI1 = 1,    // 2x2 anti-diagonal (X, Y): pairs swap with phases
  FORM_DIAG1 = 2,    // 2x2 diagonal
  FORM_PHASE1 = 3,   // 2x2 diagonal with m00 == 1 for every angle (Z, S, T, P)
  FORM_SWAP2 = 4,    // two-target SWAP
  FORM_DENSE2 = 5,   // two-target 4x4 general
  FORM_REAL1 = 6,    // 2x2 with real entries (H, RY): 4 FMA per amplitude
  FORM_RXLIKE1 = 7,  // real diagonal, imaginary off-diagonal (RX): 4 FMA per amplitude
  FORM_X1 = 8        // X: the pair swaps, no arithmetic
};

struct DevGate {
  int32_t form;
  int32_t t0, t1;          // targets (t1 = -1 for one-target forms)
  int32_t nins;            // number of sorted bit positions to insert (targets + controls)
  int32_t ins[4];          // ascending bit positions of targets and controls
  uint64_t cmask;          // control bits
  int32_t kind;            // qs_gate_kind, for k_resolve
  int32_t param_index;     // -1 = fixed
  double param, scale;
};

// Op inside a tile pass, in tile-local bit positions.
enum OpType : int32_t {
  OP_GATE = 0,    // one original gate: form + tile-local positions, matrix from the gate table
  OP_DENSE = 1,   // dense k-qubit block, matrix (2^k x 2^k) in the block table
  OP_DIAG = 2,    // diagonal k-qubit block, 2^k phases in the block table
  OP_TC = 3,      // dense block on tensor cores (its own pass): 6 qubits for complex64, 5 for complex128
  OP_PHASE = 4    // diagonal phase polynomial of a gate run over the whole register (its own pass)
};

// A contracted block whose matrix depends on theta: rebuilt on the device from
// the resolved gate table (one CTA per block and batch row), FP64.
struct DevBlock {
  int32_t k;               // block qubits (D = 2^k <= 64)
  int32_t kind;            // 0 dense (D*D entries), 1 diagonal (D entries), 2 tensor-core W image
  int32_t mem_begin, mem_end;   // member gates in the DevMember array, program order
  int64_t out;             // complex offset in the block table, or W image index
};
struct DevMember {
  int32_t gate;            // row in the gate table
  int32_t nt;              // targets: 1 or 2
  int32_t t0, t1;          // block-local target bits
  uint32_t cmask;          // block-local control bits
  int32_t form;            // GateForm of the target matrix (structure known for every theta)
};
cudaError_t prepare_build_blocks();
cudaError_t prepare_tc_pass();
// Tensor-core W images (blocks of kind 2): wmode 0 = 64x64 complex64-pass image as bf16 hi / lo,
// 1 = the same as fp16 hi / lo (precision 4), 2 = the five fp16 digit planes of a 32x32 block for
// the complex128 pass; image i of row r at wimg + r * wstride + i * wpass (uint16 elements).
cudaError_t launch_build_blocks(const DevBlock* blocks, int nblocks, const DevMember* mem, const double2* gtab,
                                int64_t gstride, int rows, double2* btab, int64_t bstride, uint16_t* wimg,
                                int64_t wstride, int wmode, int64_t wpass, cudaStream_t st);

// Tensor-core pass over tiles of 128 rows x 64 columns (13 qubits).
struct TcPassDesc {
  int32_t row[7];          // global qubits of the row bits, ascending (bit b of the row index)
  int32_t col[6];          // block qubits, ascending (bit j of the column index = local bit j)
  int32_t tile[13];        // row and column qubits together, ascending
};
// pipeline 0: bulk-copy staged kernel (k_tc_bulk); 1: register-staged kernel (k_tc_block).
// spin: polls per pipeline wait of the bulk-copy kernel before it gives up and
// sets *err (0 = the default bound).
cudaError_t launch_tc_pass(void* psi, int n, const TcPassDesc& p, const void* wimg, int prec, int pipeline,
                           int* err, cudaStream_t st, uint32_t spin = 0);
size_t tc_smem_bytes();
size_t tc_bulk_smem_bytes();

// Complex128 tensor-core pass over tiles of 128 rows x 32 columns (12 qubits):
// a dense 5-qubit block as exact fp16 digit products (kernels_tc128.cu).
struct Tc5PassDesc {
  int32_t row[7];          // global qubits of the row bits, ascending
  int32_t col[5];          // block qubits, ascending (bit j of the column index = local bit j)
  int32_t tile[12];        // row and column qubits together, ascending
  // 1 = the pass reads / writes the state as FP32 pairs (between consecutive
  // complex128 tensor-core passes; per amplitude the floats re.s, im.s, re.e,
  // im.e, value s + e), 0 = as complex128
  int32_t in_pairs, out_pairs;
};
// uint16 elements of one pass's W digit planes g_0..g_5, 4096 each
constexpr int64_t kTc128WElems = 6 * 4096;
cudaError_t prepare_tc128_pass();
size_t tc128_smem_bytes();
// psis: device array of nstates state pointers (psi unused), else psi alone; wstride (uint16
// elements) between the W planes of consecutive states, 0 = one set for all; spin as launch_tc_pass
cudaError_t launch_tc128_pass(void* psi, void* const* psis, int nstates, int64_t wstride, int n,
                              const Tc5PassDesc& p, const void* wimg, int* err, cudaStream_t st, uint32_t spin = 0);

// Diagonal phase pass: amplitude x times prod_j exp(i alpha_j s_j(x)),
// s_j(x) = (-1)^popcount(mask_j & x), alpha_j = alpha0 + coef * theta[pidx]
// (pidx >= 0) or alpha0.
struct DevPhaseTerm {
  uint64_t mask;
  int32_t pidx;
  int32_t pad;
  double alpha0, coef;
};
constexpr int kPhaseChunkBits = 12;   // amplitudes per warp chunk: 2^12 (lo = bits 0..11)
constexpr int kPhaseMaxTerms = 1024;
constexpr int kPhaseMaxMixed = 16;
// A pass's terms, in class order (relative to term_off): LOW [0, nlow) (only
// bits below 12, at least two), LIN [lin_off[u], lin_off[u + 1]) for the one
// bit u < 12 they have (lin_off[0] = nlow, lin_off[12] = high_begin), HIGH
// [high_begin, mixed_begin) (no bit below 12), MIXED [mixed_begin, nterms).
struct PhasePassDesc {
  int32_t term_off, nterms;
  int32_t nlow;
  int32_t lin_off[kPhaseChunkBits + 1];
  int32_t high_begin, mixed_begin;
  int32_t occ;             // resident CTAs per SM, set by prepare_phase_pass
  int32_t df;              // complex128 computed in FP32 pairs
};
size_t phase_smem_bytes(int nterms, qs_dtype dt);
cudaError_t prepare_phase_pass(PhasePassDesc& d, qs_dtype dt);
// psis: device array of nstates state pointers (psi unused), else psi alone;
// theta rows ntheta apart, one per state (may be null when no term has pidx >= 0)
cudaError_t launch_phase_pass(void* psi, void* const* psis, int nstates, int n, qs_dtype dt,
                              const DevPhaseTerm* terms, const PhasePassDesc& d, const double* theta,
                              int64_t ntheta, cudaStream_t st);

struct DevOp {
  int32_t type;
  int32_t form;            // for OP_GATE
  int32_t k;               // qubits of a block op
  int32_t nins;            // OP_GATE: positions to insert (targets + controls), ascending
  int32_t ins[6];          // OP_GATE: sorted insert positions; blocks: op qubit positions ascending
  int32_t t0, t1;          // OP_GATE target positions (tile-local)
  uint32_t cmask;          // OP_GATE control mask (tile-local)
  int32_t mat;             // OP_GATE: gate index in the gate table; blocks: complex offset in block table
  int32_t per_row;         // blocks: 1 = rebuilt per batch row (parametric), table rows bstride apart
};

struct PassDesc {
  int32_t m;               // tile qubits
  int32_t L;               // low qubits 0..L-1 contained in the tile
  int32_t nhigh;           // tile qubits above L-1
  int32_t high[14];        // their global positions, ascending
  int32_t kmax;            // widest dense block op in the pass (selects the kernel instance)
  int32_t mbuf_elems;      // matrix staging entries the pass needs (max over its ops)
  int32_t op_begin, op_end;
  int32_t df;              // complex128 tile computed in FP32 pairs (double-float), else FP64
  int32_t bulk;            // tiles moved by bulk asynchronous copies into two shared-memory buffers
  uint32_t spin;           // bulk staging: polls per wait for a tile (0 = default bound)
  int* err;                // bulk staging: device error flag (set to 1 when a wait runs out)
};

// Kernel attributes / occupancy of a pass's instance; host side, never during a capture.
cudaError_t prepare_tile_pass(const PassDesc& p, qs_dtype dt);
// Shared memory of one tile CTA: tile + run offsets + matrix staging buffer.
size_t tile_smem_bytes(int m, int nhigh, int mbuf_elems, qs_dtype dt);
// The same for a pass as launched: with bulk staging, a second tile buffer and two barriers.
size_t tile_pass_smem_bytes(const PassDesc& p, qs_dtype dt);

// ---------------------------------------------------------------------------
// Bit helpers.

QS_HD uint64_t insert_zero_bits(uint64_t x, const int32_t* pos, int npos) {
  // pos ascending: make room for a zero bit at each position in turn.
  for (int k = 0; k < npos; ++k) {
    const uint64_t lo = x & ((1ull << pos[k]) - 1);
    x = ((x >> pos[k]) << (pos[k] + 1)) | lo;
  }
  return x;
}

// Same, with the loop unrolled to MAXN steps so `pos` can stay in registers.
template <int MAXN, typename U>
QS_HD U insert_zero_bits_u(U x, const int32_t* pos, int npos) {
#ifdef __CUDACC__
#pragma unroll
#endif
  for (int k = 0; k < MAXN; ++k) {
    if (k < npos) {
      const U lo = x & ((U(1) << pos[k]) - 1);
      x = ((x >> pos[k]) << (pos[k] + 1)) | lo;
    }
  }
  return x;
}

// ---------------------------------------------------------------------------
// Kernel launch wrappers (kernels_*.cu). All return cudaError_t of the launch.

template <typename R> struct Cplx;
template <> struct Cplx<float> { using T = float2; };
template <> struct Cplx<double> { using T = double2; };

cudaError_t launch_set_basis(void* psi, int n, qs_dtype dt, uint64_t x, cudaStream_t st);
// out[k] = psi[idx[k]] (device arrays)
cudaError_t launch_gather(const void* psi, qs_dtype dt, const uint64_t* idx, uint64_t count, void* out,
                          cudaStream_t st);
cudaError_t launch_resolve(const DevGate* gates, const int32_t* param_gates, int nparam_gates,
                           const double* theta, int64_t ntheta, int batch, double2* table,
                           int64_t table_stride, cudaStream_t st);
cudaError_t launch_gate(void* psi, int n, qs_dtype dt, const DevGate& g, const double2* mat,
                        bool adjoint, cudaStream_t st);
// Staggered multi-gate group (Section 3.3, Tab. 3): S = 2^lgS one-target
// gates on distinct qubits; the state is cut into S segments by lgS qubits no
// member targets; at time step T gate j updates segment (T + j) mod S.
constexpr int kSmgpMax = 8;
struct SmgpDesc {
  int32_t S, lgS;
  int32_t gate[kSmgpMax];     // gate-table rows
  int32_t form[kSmgpMax];     // GateForm of the target matrix (diagonal forms applied as 2x2)
  int32_t t[kSmgpMax];        // target qubits
  int32_t pos[kSmgpMax][4];   // ascending: the segment qubits and t[j] (lgS + 1 entries)
  uint64_t seg_or[kSmgpMax];  // segment s -> its bits on the segment qubits
};
// One time step of group d (device descriptor), a 2-D block: x = amplitude pairs, y = member gate.
cudaError_t launch_smgp_step(void* psi, int n, qs_dtype dt, const SmgpDesc* d_desc, const SmgpDesc& h_desc, int T,
                             const double2* gtab, cudaStream_t st);
// Batched forms: psis = device array of nstates state pointers (psi unused);
// gate table rows gstride apart (gtab points at the first state's row);
// blocks rebuilt per row are read from block-table row brow0 + state, bstride
// apart (fixed blocks from row 0).
cudaError_t launch_tile_pass_batched(void* psi, void* const* psis, int nstates, int64_t gstride, int64_t bstride,
                                     int64_t brow0, int n, qs_dtype dt, const PassDesc& p, const DevOp* ops,
                                     const double2* gtab, const double2* btab, cudaStream_t st);
// wstride (uint16 elements) between the W images of consecutive states; 0 = one image for all
cudaError_t launch_tc_pass_batched(void* psi, void* const* psis, int nstates, int64_t wstride, int n,
                                   const TcPassDesc& p, const void* wimg, int prec, int pipeline, int* err,
                                   cudaStream_t st, uint32_t spin = 0);
// Batched <P> for every group in one launch per wave of L2-resident states:
// out[b * Z + zi] = per-string sum of state b (string zl[zi], groups (gx, gz, gc));
// partials hold nstates * Z * expval_wave_ctas(expval_wave_states(...)) doubles.
int expval_wave_states(int n, qs_dtype dt, int nstates);
int expval_wave_ctas(int wave_states);
// glist orders the groups: [0, ngroups1) hold one string each, the rest up to 8.
cudaError_t launch_expval_groups_batched(const void* const* psis, int nstates, int n, qs_dtype dt,
                                         const uint64_t* gx, const int32_t* gz, const int32_t* gc,
                                         const int32_t* glist, int ngroups1, int ngroups, const uint64_t* zl, int Z,
                                         double* partials, double* out, cudaStream_t st);
cudaError_t launch_tile_pass(void* psi, int n, qs_dtype dt, const PassDesc& p, const DevOp* ops,
                             const double2* gate_table, const double2* block_table, int threads,
                             cudaStream_t st);

// Adjoint gradient, tiled reverse sweep: G^dagger table (with the angle
// derivatives), then one launch per tile pass of the reversed circuit over phi
// and lam; partials[row * pcols + CTA] for the parametric gates (rows via grow).
cudaError_t launch_adjoint_table(const DevGate* gates, int ngates, const double2* gtab, double2* gadj,
                                 cudaStream_t st);
cudaError_t prepare_adjoint_tile(const PassDesc& p, qs_dtype dt);
size_t adjoint_tile_smem_bytes(const PassDesc& p, qs_dtype dt);
cudaError_t launch_adjoint_tile(void* phi, void* lam, int n, qs_dtype dt, const PassDesc& p, const DevOp* ops,
                                const double2* gadj, const int32_t* grow, double* partials, int pcols,
                                cudaStream_t st);

// Reductions write FP64 partials into `partials` (capacity >= reduce_blocks()).
int reduce_blocks();
cudaError_t launch_norm(const void* psi, int n, qs_dtype dt, double* partials, double* out,
                        cudaStream_t st);
cudaError_t launch_inner(const void* a, const void* b, int n, qs_dtype dt, double* partials,
                         double* out2, cudaStream_t st);
cudaError_t launch_expval_x(const void* psi, int n, qs_dtype dt, uint64_t xmask,
                            const uint64_t* zmasks, const double* coeffs, int nz, double* partials,
                            double* out, cudaStream_t st);
cudaError_t launch_apply_pauli(const void* psi, void* out, int n, qs_dtype dt,
                               const uint64_t* xm, const uint64_t* zm, const double* coeff, int nt,
                               cudaStream_t st);
// partials[0..RB) = per-CTA max |a - b|, partials[RB..2RB) = per-CTA sum |a - b|^2
cudaError_t launch_diff(const void* a, qs_dtype da, const void* b, qs_dtype db, int n, double* partials,
                        cudaStream_t st);
cudaError_t launch_sum_rows(const double* partials, int rows, int cols, double* out,
                            cudaStream_t st);

void note_launch(int64_t k = 1);
// While suspended (graph capture), launches are not counted; replays are.
void suspend_launch_count(bool on);
// Device allocations (cudaMalloc) made by the library so far (diagnostics).
void note_device_alloc();
int64_t device_alloc_count();
// SM count of the current device (queried once per process; grids of
// streaming kernels are sized from it).
int device_sm_count();

// Pauli strings one expectation launch (k_expval_x) handles: callers split
// longer groups of equal x mask into launches of at most this many strings.
constexpr int kExpvalMaxZ = 8;

namespace rt {
// Sign and factor turning k_expval_x's per-string sum into <P> (runtime.cpp).
double term_factor(const qs_pauli_term& t);
}  // namespace rt

}  // namespace qs
