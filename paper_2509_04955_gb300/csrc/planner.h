// Circuit IR, gate DAG and dependency-aware contraction (Section 3.4), host side, FP64.
#pragma once

#include <complex>
#include <cstdint>
#include <string>
#include <vector>

#include "qs_internal.h"

namespace qs {

using cd = std::complex<double>;

struct HGate {
  int kind = 0;
  int nt = 1, t[2] = {-1, -1};
  int nc = 0, c[2] = {-1, -1};
  uint64_t cmask = 0, qmask = 0;
  uint64_t dmask = 0;        // qubits on which the gate is diagonal (controls; all qubits of a diagonal gate)
  int param_index = -1;
  double param = 0, scale = 1;
  bool parametric = false;
  int form = FORM_DENSE1;
  cd fixed[16];              // target matrix (2x2 in the first 4) when not parametric
  cd custom[16];             // U1 / U2 input matrix
};

// Validates and resolves the caller's gates. Throws qs::Error on bad input.
// Gates of one circuit are indexed with 32-bit integers: longer lists are an
// argument error.
constexpr size_t kMaxGates = size_t(1) << 30;
void resolve_gates(int n, const qs_gate* g, size_t ng, std::vector<HGate>& out);
// Target matrix (2x2 or 4x4 row-major) for given theta (may be null when not parametric).
void target_matrix(const HGate& g, const double* theta, cd* m);
// Device descriptor with global bit positions; `pairs` forces the pair
// enumeration of DENSE1 (used by the adjoint step for diagonal gates).
DevGate make_dev_gate(const HGate& g, bool pairs = false);
// Fraction of a state sweep (read + write of all amplitudes) one gate moves
// when applied alone: 1 for a dense one-target gate, 1/2 per control, 1/2 for
// phase gates (only the |1> half changes), 1/2 for SWAP.
double gate_sweep_fraction(const HGate& g);
// FMA instructions per amplitude of one gate applied alone.
double gate_fma_per_amp(const HGate& g);

struct Block {
  std::vector<int> gates;    // program order
  std::vector<int> qubits;   // ascending; local bit j <-> qubits[j]
  uint64_t dmask = 0;        // qubits on which every member gate is diagonal
  bool diag = false;         // every member gate is diagonal
  bool parametric = false;   // some member depends on theta
  int rep = OP_GATE;         // OP_GATE (members applied one by one), OP_DENSE, OP_DIAG or OP_TC
};

struct PlanOptions {
  int k = 1;                 // block width
  bool paper = false;        // only the merges of Section 3.4
  bool cost_model = true;    // keep gates separate when the dense block costs more
  double fp_weight = 1.0;    // cost of one FMA of the state's precision, in FP32-FMA units
  double smem_weight = 1.0;  // cost of one byte of shared-memory traffic, in FP32-FMA units
  int amp_bytes = 8;
  bool fuse_parametric = false;   // parametric gates may join multi-gate blocks
  bool search = true;              // also grow block qubit sets by legal scans (slower planning)
  bool no_merge = false;           // every gate its own block (the adjoint reverse sweep keeps gates apart)
};

// DAGC-k greedy contraction. Returns blocks in emission order.
std::vector<Block> contract(int n, const std::vector<HGate>& gates, const PlanOptions& o);

// Dense 2^k x 2^k matrix of a block (local bit j <-> block.qubits[j]), ordered
// product of the member gates (Eq. 7 for distinct qubits, M2 M1 on one qubit).
void block_matrix(const Block& b, const std::vector<HGate>& gates, const double* theta, std::vector<cd>& M);

// Phase polynomial of a diagonal run: the run multiplies amplitude x by
// prod_j exp(i alpha_j s_j(x)), s_j(x) = (-1)^popcount(mask_j & x), with
// alpha_j = alpha0 + coef * theta[pidx] (pidx >= 0) or alpha0 (pidx < 0).
struct PhaseTerm {
  uint64_t mask = 0;
  int pidx = -1;
  double alpha0 = 0, coef = 0;
};
// A contiguous run of program gates [begin, end) made of CNOTs, SWAPs and
// diagonal gates (at most one control) whose GF(2) permutation of the basis
// composes to the identity: the run is then a diagonal operator on the whole
// register, exp(i sum_j alpha_j s_j(x)) (the cost layer of QAOA, Section 4.1's
// third circuit class, is one such run per layer).
struct PhaseRun {
  int begin = 0, end = 0;
  uint64_t qmask = 0;
  std::vector<PhaseTerm> terms;
};
// Runs of at least min_gates gates, at most max_terms terms of which at most
// max_mixed have >= 2 mask bits below low_bits together with a bit above.
std::vector<PhaseRun> find_phase_runs(int n, const std::vector<HGate>& gates, int min_gates, int max_terms,
                                      int max_mixed, int low_bits);

struct OpRec {               // one op of the fused program (global qubit positions)
  int type;                  // OP_GATE / OP_DENSE / OP_DIAG / OP_TC / OP_PHASE
  int gate = -1;             // OP_GATE: gate index
  int block = -1;            // block ops: block index; OP_PHASE: run index
  uint64_t qmask = 0;
  uint64_t dmask = 0;        // qubits on which the op is diagonal
};

struct PassRec {
  std::vector<int> tile;     // tile qubits, ascending (contains 0..L-1)
  int op_begin = 0, op_end = 0;
};

// Groups ops into tile passes of <= m qubits that always contain qubits
// 0..L-1 (the same greedy over the op DAG, width m). order_out lists the op
// indices pass by pass; a pass covers order_out[op_begin .. op_end).
std::vector<PassRec> schedule_passes(int n, const std::vector<OpRec>& ops, int m, int L,
                                     std::vector<int>& order_out);

}  // namespace qs
