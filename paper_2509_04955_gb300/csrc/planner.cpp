// Circuit IR resolution, gate DAG and dependency-aware gate contraction.
//
// Section 3.4 builds a DAG with an edge from each earlier gate that shares a
// qubit (controls included) and merges gates greedily; it names three merges:
// two one-qubit gates on distinct qubits into M2 (x) M1 (Eq. 7), two gates on
// one qubit into M2 M1, and two CU gates on the same (c, t) into C(U2 U1).
// The greedy is not spelled out; the reading implemented here (DAGC-k):
//   1. the next block starts at the earliest gate not yet emitted;
//   2. later gates are scanned in program order; a gate joins the block when
//      all of its DAG predecessors are emitted or already in the block and the
//      block's qubit set stays within k qubits; a gate that does not join
//      blocks its qubits for the rest of the scan;
//   3. the block's unitary is the ordered product of its gates (FP64).
// Paper mode keeps only the three merges above (k = 2).
// The cost rule of Section 3.4 (a merged gate must cost fewer operations than
// its parts) decides whether a block is applied as one dense matrix or as its
// member gates in sequence; the cost counts FMA instructions and shared-memory
// bytes per amplitude.
#include "planner.h"

#include <algorithm>
#include <cmath>
#include <cstring>
#include <stdexcept>

#include "qs_error.h"

namespace qs {

static bool kind_is_parametric(int k) {
  return k == QS_GATE_RX || k == QS_GATE_RY || k == QS_GATE_RZ || k == QS_GATE_P;
}

static bool kind_is_diag(int k) {
  switch (k) {
    case QS_GATE_Z: case QS_GATE_S: case QS_GATE_SDG: case QS_GATE_T: case QS_GATE_TDG:
    case QS_GATE_RZ: case QS_GATE_P:
      return true;
    default:
      return false;
  }
}

static bool kind_is_phase(int k) {  // diagonal with m00 == 1 for every angle
  return kind_is_diag(k) && k != QS_GATE_RZ;
}

static void fixed_matrix(int kind, double a, const cd* custom, cd* m) {
  const double r2 = 1.0 / std::sqrt(2.0);
  const cd I(0, 1);
  const double c = std::cos(0.5 * a), s = std::sin(0.5 * a);
  for (int i = 0; i < 16; ++i) m[i] = 0;
  switch (kind) {
    case QS_GATE_H: m[0] = r2; m[1] = r2; m[2] = r2; m[3] = -r2; break;
    case QS_GATE_X: m[1] = 1; m[2] = 1; break;
    case QS_GATE_Y: m[1] = -I; m[2] = I; break;
    case QS_GATE_Z: m[0] = 1; m[3] = -1; break;
    case QS_GATE_S: m[0] = 1; m[3] = I; break;
    case QS_GATE_SDG: m[0] = 1; m[3] = -I; break;
    case QS_GATE_T: m[0] = 1; m[3] = std::polar(1.0, M_PI / 4); break;
    case QS_GATE_TDG: m[0] = 1; m[3] = std::polar(1.0, -M_PI / 4); break;
    case QS_GATE_RX: m[0] = c; m[1] = -I * s; m[2] = -I * s; m[3] = c; break;
    case QS_GATE_RY: m[0] = c; m[1] = -s; m[2] = s; m[3] = c; break;
    case QS_GATE_RZ: m[0] = std::polar(1.0, -0.5 * a); m[3] = std::polar(1.0, 0.5 * a); break;
    case QS_GATE_P: m[0] = 1; m[3] = std::polar(1.0, a); break;
    case QS_GATE_U1: for (int i = 0; i < 4; ++i) m[i] = custom[i]; break;
    case QS_GATE_SWAP: m[0] = 1; m[6] = 1; m[9] = 1; m[15] = 1; break;
    case QS_GATE_U2: for (int i = 0; i < 16; ++i) m[i] = custom[i]; break;
    default: throw Error(QS_ERR_ARG, "unknown gate kind");
  }
}

void target_matrix(const HGate& g, const double* theta, cd* m) {
  if (!g.parametric) {
    for (int i = 0; i < 16; ++i) m[i] = g.fixed[i];
    return;
  }
  const double a = g.param + g.scale * theta[g.param_index];
  fixed_matrix(g.kind, a, g.custom, m);
}

void resolve_gates(int n, const qs_gate* gs, size_t ng, std::vector<HGate>& out) {
  if (ng > kMaxGates) throw Error(QS_ERR_ARG, "too many gates (at most 2^30 per circuit)");
  out.clear();
  out.reserve(ng);
  for (size_t i = 0; i < ng; ++i) {
    const qs_gate& q = gs[i];
    HGate g;
    g.kind = q.kind;
    if (q.kind < QS_GATE_H || q.kind > QS_GATE_U2)
      throw Error(QS_ERR_ARG, "gate " + std::to_string(i) + ": unknown kind " + std::to_string(q.kind));
    const bool two = q.kind == QS_GATE_SWAP || q.kind == QS_GATE_U2;
    g.nt = two ? 2 : 1;
    if (q.nq != g.nt)
      throw Error(QS_ERR_ARG, "gate " + std::to_string(i) + ": wrong number of targets");
    if (q.nctrl < 0 || q.nctrl > kMaxControls)
      throw Error(QS_ERR_ARG, "gate " + std::to_string(i) + ": at most two controls");
    g.nc = q.nctrl;
    uint64_t seen = 0;
    auto take = [&](int b) {
      if (b < 0 || b >= n) throw Error(QS_ERR_ARG, "gate " + std::to_string(i) + ": qubit out of range");
      if (seen & (1ull << b)) throw Error(QS_ERR_ARG, "gate " + std::to_string(i) + ": repeated qubit");
      seen |= 1ull << b;
    };
    for (int k = 0; k < g.nt; ++k) { take(q.q[k]); g.t[k] = q.q[k]; }
    for (int k = 0; k < g.nc; ++k) { take(q.ctrl[k]); g.c[k] = q.ctrl[k]; g.cmask |= 1ull << q.ctrl[k]; }
    g.qmask = seen;
    g.param = q.param;
    g.scale = q.scale;
    g.parametric = kind_is_parametric(q.kind) && q.param_index >= 0;
    g.param_index = g.parametric ? q.param_index : -1;
    for (int k = 0; k < 16; ++k) g.custom[k] = cd(q.mat[2 * k], q.mat[2 * k + 1]);
    if (!g.parametric) fixed_matrix(g.kind, q.param, g.custom, g.fixed);
    g.dmask = g.cmask | (kind_is_diag(q.kind) ? g.qmask : 0);
    if (g.nt == 2) g.form = q.kind == QS_GATE_SWAP ? FORM_SWAP2 : FORM_DENSE2;
    else if (kind_is_phase(q.kind)) g.form = FORM_PHASE1;
    else if (kind_is_diag(q.kind)) g.form = FORM_DIAG1;
    else if (q.kind == QS_GATE_X) g.form = FORM_X1;
    else if (q.kind == QS_GATE_Y) g.form = FORM_ANTI1;
    else if (q.kind == QS_GATE_H || q.kind == QS_GATE_RY) g.form = FORM_REAL1;
    else if (q.kind == QS_GATE_RX) g.form = FORM_RXLIKE1;
    else g.form = FORM_DENSE1;
    out.push_back(g);
  }
}

DevGate make_dev_gate(const HGate& g, bool pairs) {
  DevGate d;
  std::memset(&d, 0, sizeof(d));
  d.form = g.form;
  if (pairs && (g.form == FORM_PHASE1 || g.form == FORM_DIAG1)) d.form = FORM_DENSE1;
  d.t0 = g.t[0];
  d.t1 = g.nt == 2 ? g.t[1] : -1;
  std::vector<int> ins;
  if (d.form != FORM_DIAG1)
    for (int k = 0; k < g.nt; ++k) ins.push_back(g.t[k]);
  for (int k = 0; k < g.nc; ++k) ins.push_back(g.c[k]);
  std::sort(ins.begin(), ins.end());
  d.nins = (int)ins.size();
  for (int k = 0; k < d.nins; ++k) d.ins[k] = ins[k];
  d.cmask = g.cmask;
  d.kind = g.kind;
  d.param_index = g.param_index;
  d.param = g.param;
  d.scale = g.scale;
  return d;
}

double gate_sweep_fraction(const HGate& g) {
  const double ctl = std::ldexp(1.0, -g.nc);
  switch (g.form) {
    case FORM_PHASE1: return 0.5 * ctl;
    case FORM_SWAP2: return 0.5 * ctl;
    default: return ctl;
  }
}

double gate_fma_per_amp(const HGate& g) {
  const double ctl = std::ldexp(1.0, -g.nc);
  switch (g.form) {
    case FORM_DENSE1: return 8 * ctl;
    case FORM_ANTI1: return 4 * ctl;
    case FORM_REAL1: return 4 * ctl;
    case FORM_RXLIKE1: return 4 * ctl;
    case FORM_X1: return 0;
    case FORM_DIAG1: return 4 * ctl;
    case FORM_PHASE1: return 2 * ctl;
    case FORM_SWAP2: return 0;
    default: return 16 * ctl;
  }
}

// ---------------------------------------------------------------- contraction

static int popc(uint64_t v) { return __builtin_popcountll(v); }

static std::vector<int> mask_bits(uint64_t m) {
  std::vector<int> v;
  for (int b = 0; b < 64; ++b)
    if (m & (1ull << b)) v.push_back(b);
  return v;
}

// Paper-mode merge test (Section 3.4): one-qubit gates on <= 2 distinct qubits,
// or controlled one-target gates with identical (controls, target).
static bool paper_mergeable(const HGate& a, const HGate& b, uint64_t Q) {
  const bool a1 = a.nt == 1 && a.nc == 0, b1 = b.nt == 1 && b.nc == 0;
  if (a1 && b1) return popc(Q | b.qmask) <= 2;
  if (a.nt == 1 && b.nt == 1 && a.nc > 0 && b.nc > 0)
    return a.t[0] == b.t[0] && a.cmask == b.cmask;
  return false;
}

// The fields the scans read, packed (an HGate carries two 4x4 complex
// matrices, so scanning HGates would touch a cache line per gate field).
struct GateLite {
  uint64_t qmask, dmask;
  bool parametric;
};

static std::vector<GateLite> lite_of(const std::vector<HGate>& gates) {
  std::vector<GateLite> v(gates.size());
  for (size_t i = 0; i < gates.size(); ++i) v[i] = GateLite{gates[i].qmask, gates[i].dmask, gates[i].parametric};
  return v;
}

// One greedy scan from `first`: absorbs later gates that commute with every
// gate skipped so far and keep the block within kcap qubits (and within
// `allowed`, when given). Returns the absorbed gates in program order.
// With `members` NULL only the count is returned (the growth searches).
static int scan_block(const std::vector<HGate>& gates, const std::vector<GateLite>& lite,
                      const std::vector<char>& done, int first, int kcap, uint64_t allowed, const PlanOptions& o,
                      uint64_t all, std::vector<int>* members) {
  const int G = (int)gates.size();
  if (members) members->assign(1, first);
  int count = 1;
  uint64_t Q = lite[first].qmask, blk_nd = 0, blk_d = 0;
  const bool lone = !o.fuse_parametric && lite[first].parametric;   // stays a gate op
  for (int h = first + 1; h < G && !lone; ++h) {
    if (done[h]) continue;
    const GateLite& gh = lite[h];
    const uint64_t qh = gh.qmask;
    const bool movable = (qh & blk_nd) == 0 && (qh & blk_d & ~gh.dmask) == 0;
    bool ok = movable && popc(Q | qh) <= kcap && (qh & ~allowed) == 0;
    if (ok && !o.fuse_parametric && gh.parametric) ok = false;
    if (ok && o.paper) ok = paper_mergeable(gates[first], gates[h], Q);
    if (ok) {
      if (members) members->push_back(h);
      ++count;
      Q |= qh;
    } else {
      blk_nd |= qh & ~gh.dmask;
      blk_d |= qh & gh.dmask;
    }
    // no later gate can join once every admissible qubit is blocked by a skipped
    // gate that is not diagonal there, or the block is full and all of it blocked
    if ((allowed & all & ~blk_nd) == 0) break;
    if (popc(Q) >= kcap && (Q & ~blk_nd) == 0) break;
  }
  return count;
}

static std::vector<int> scan_members(const std::vector<HGate>& gates, const std::vector<GateLite>& lite,
                                     const std::vector<char>& done, int first, int kcap, uint64_t allowed,
                                     const PlanOptions& o, uint64_t all) {
  std::vector<int> m;
  scan_block(gates, lite, done, first, kcap, allowed, o, all, &m);
  return m;
}

// Qubit set planned from the next unemitted gates: starting from the first
// gate's qubits, repeatedly add the qubit that makes the most gates of the
// window fit inside the set.
static uint64_t plan_qubits(const std::vector<HGate>& gates, const std::vector<char>& done, int first, int kcap,
                            int n) {
  const int G = (int)gates.size();
  std::vector<uint64_t> win;
  for (int h = first; h < G && (int)win.size() < 4 * n; ++h)
    if (!done[h]) win.push_back(gates[h].qmask);
  uint64_t Q = gates[first].qmask;
  while (popc(Q) < kcap) {
    int best_q = -1, best = 0;
    for (int q = 0; q < n; ++q) {
      if (Q & (1ull << q)) continue;
      const uint64_t Qq = Q | (1ull << q);
      int cnt = 0;
      for (uint64_t m : win)
        if ((m & (1ull << q)) && (m & ~Qq) == 0) ++cnt;
      if (cnt > best) { best = cnt; best_q = q; }
    }
    if (best_q < 0) break;
    Q |= 1ull << best_q;
  }
  return Q;
}

// Qubit set grown by legal scans: at each step add the qubit whose admission
// lets the scan absorb the most gates.
static uint64_t grow_qubits(const std::vector<HGate>& gates, const std::vector<GateLite>& lite,
                            const std::vector<char>& done, int first, int kcap, int n, const PlanOptions& o,
                            uint64_t all) {
  uint64_t Q = gates[first].qmask;
  // candidates: qubits of the next unemitted gates
  uint64_t cand = 0;
  int seen = 0;
  for (int h = first; h < (int)gates.size() && seen < 4 * n; ++h)
    if (!done[h]) { cand |= gates[h].qmask; ++seen; }
  while (popc(Q) < kcap) {
    int best_q = -1;
    size_t best = 0;
    for (int q = 0; q < n; ++q) {
      if ((Q & (1ull << q)) || !(cand & (1ull << q))) continue;
      const size_t c = (size_t)scan_block(gates, lite, done, first, kcap, Q | (1ull << q), o, all, nullptr);
      if (c > best) { best = c; best_q = q; }
    }
    if (best_q < 0) break;
    Q |= 1ull << best_q;
  }
  return Q;
}

// As grow_qubits, but each step may also add two qubits at once (a pair that
// only pays off together, such as both ends of a two-qubit gate).
static uint64_t grow_qubits_pairs(const std::vector<HGate>& gates, const std::vector<GateLite>& lite,
                                  const std::vector<char>& done, int first, int kcap, int n, const PlanOptions& o,
                                  uint64_t all) {
  uint64_t Q = gates[first].qmask;
  uint64_t cand = 0;
  int seen = 0;
  for (int h = first; h < (int)gates.size() && seen < 4 * n; ++h)
    if (!done[h]) { cand |= gates[h].qmask; ++seen; }
  std::vector<int> cq;
  for (int q = 0; q < n; ++q)
    if (cand & (1ull << q)) cq.push_back(q);
  while (popc(Q) < kcap) {
    uint64_t best_add = 0;
    double best = 0;
    for (size_t i = 0; i < cq.size(); ++i) {
      const uint64_t a = 1ull << cq[i];
      if (Q & a) continue;
      const double c1 = (double)scan_block(gates, lite, done, first, kcap, Q | a, o, all, nullptr);
      if (c1 > best) { best = c1; best_add = a; }
      if (popc(Q) + 2 > kcap) continue;
      for (size_t j = i + 1; j < cq.size(); ++j) {
        const uint64_t b2 = 1ull << cq[j];
        if (Q & b2) continue;
        // a pair costs two slots: compare per added qubit, favouring progress
        const double c2 = (double)scan_block(gates, lite, done, first, kcap, Q | a | b2, o, all, nullptr);
        if (c2 - 0.5 > best) { best = c2 - 0.5; best_add = a | b2; }
      }
    }
    if (!best_add) break;
    Q |= best_add;
  }
  return Q;
}

std::vector<Block> contract(int n, const std::vector<HGate>& gates, const PlanOptions& o) {
  // A later gate may join the block (move ahead of the gates skipped so far)
  // when it commutes with every skipped gate: on each shared qubit both are
  // diagonal there (Z-basis diagonal gates and controls commute). This is the
  // dependency structure of Section 3.4's DAG with commuting diagonal gates
  // left unordered. Growth strategies tried per block: first-fit, a qubit set
  // planned from the next gates, and (o.search) a set grown by legal scans;
  // the one absorbing the most gates is kept.
  const int G = (int)gates.size();
  std::vector<char> done(G, 0);   // emitted
  const std::vector<GateLite> lite = lite_of(gates);
  std::vector<Block> blocks;
  int first = 0;
  const uint64_t all = n >= 64 ? ~0ull : ((1ull << n) - 1);
  while (first < G) {
    while (first < G && done[first]) ++first;
    if (first >= G) break;
    Block blk;
    const int kcap = o.paper ? 2 : std::max(o.k, popc(gates[first].qmask));
    std::vector<int> a = o.no_merge ? std::vector<int>{first} : scan_members(gates, lite, done, first, kcap, all, o, all);
    if (!o.no_merge && !o.paper && kcap > 2 && (o.fuse_parametric || !gates[first].parametric)) {
      std::vector<int> b = scan_members(gates, lite, done, first, kcap, plan_qubits(gates, done, first, kcap, n), o, all);
      if (b.size() > a.size()) a.swap(b);
      if (o.search) {
        std::vector<int> c = scan_members(gates, lite, done, first, kcap,
                                          grow_qubits(gates, lite, done, first, kcap, n, o, all), o, all);
        if (c.size() > a.size()) a.swap(c);
        if (n <= 40 && gates.size() <= 40000) {
          std::vector<int> d = scan_members(gates, lite, done, first, kcap,
                                            grow_qubits_pairs(gates, lite, done, first, kcap, n, o, all), o, all);
          if (d.size() > a.size()) a.swap(d);
        }
      }
    }
    blk.gates = a;
    uint64_t Q = 0;
    for (int g : blk.gates) Q |= gates[g].qmask;
    for (int g : blk.gates) done[g] = 1;
    blk.qubits = mask_bits(Q);
    blk.dmask = Q;
    for (int g : blk.gates) blk.dmask &= gates[g].dmask | ~gates[g].qmask;
    blk.diag = true;
    for (int g : blk.gates) {
      blk.diag = blk.diag && (gates[g].form == FORM_PHASE1 || gates[g].form == FORM_DIAG1);
      blk.parametric = blk.parametric || gates[g].parametric;
    }
    // Representation (Section 3.4's cost rule, in FMA + shared-memory bytes).
    const int k = (int)blk.qubits.size();
    if (blk.gates.size() == 1) {
      blk.rep = OP_GATE;
    } else if (o.paper) {
      blk.rep = blk.diag ? OP_DIAG : OP_DENSE;
    } else {
      // Cost of an op per amplitude in FP32-FMA-instruction units: arithmetic
      // (FP64 weighted by fp_weight) and the shared-memory round trip of the
      // amplitudes it touches (smem_weight per byte) run on different pipes,
      // so an op costs the larger of the two.
      auto op_cost = [&](double fma, double frac) {
        return std::max(o.fp_weight * fma, o.smem_weight * 2.0 * o.amp_bytes * frac);
      };
      double sep = 0;
      for (int g : blk.gates) sep += op_cost(gate_fma_per_amp(gates[g]), gate_sweep_fraction(gates[g]));
      const double dense = op_cost(4.0 * (1 << k), 1.0);
      const double dg = op_cost(4.0, 1.0);
      if (blk.diag) blk.rep = dg < sep ? OP_DIAG : OP_GATE;
      else blk.rep = (!o.cost_model || dense < sep) ? OP_DENSE : OP_GATE;
    }
    blocks.push_back(std::move(blk));
  }
  return blocks;
}

// Applies one gate, given in block-local bit positions, to a 2^k vector.
static void apply_local(const HGate& g, const int* lpos_t, uint64_t lcmask, const cd* m, cd* v, int k) {
  const uint64_t dim = 1ull << k;
  if (g.nt == 1) {
    const uint64_t tb = 1ull << lpos_t[0];
    for (uint64_t i = 0; i < dim; ++i) {
      if ((i & lcmask) != lcmask || (i & tb)) continue;
      const cd a0 = v[i], a1 = v[i | tb];
      v[i] = m[0] * a0 + m[1] * a1;
      v[i | tb] = m[2] * a0 + m[3] * a1;
    }
  } else {
    const uint64_t ta = 1ull << lpos_t[0], tb = 1ull << lpos_t[1];
    for (uint64_t i = 0; i < dim; ++i) {
      if ((i & lcmask) != lcmask || (i & (ta | tb))) continue;
      const uint64_t idx[4] = {i, i | ta, i | tb, i | ta | tb};
      cd a[4], r[4];
      for (int j = 0; j < 4; ++j) a[j] = v[idx[j]];
      for (int r_ = 0; r_ < 4; ++r_) {
        r[r_] = 0;
        for (int j = 0; j < 4; ++j) r[r_] += m[4 * r_ + j] * a[j];
      }
      for (int j = 0; j < 4; ++j) v[idx[j]] = r[j];
    }
  }
}

void block_matrix(const Block& b, const std::vector<HGate>& gates, const double* theta, std::vector<cd>& M) {
  const int k = (int)b.qubits.size();
  const uint64_t D = 1ull << k;
  M.assign(D * D, cd(0));
  auto local = [&](int q) {
    for (int j = 0; j < k; ++j)
      if (b.qubits[j] == q) return j;
    throw Error(QS_ERR_ARG, "internal: qubit not in block");
  };
  // each member's matrix and block-local positions, once
  struct Local {
    cd m[16];
    int lt[2];
    uint64_t lc;
  };
  std::vector<Local> loc(b.gates.size());
  for (size_t i = 0; i < b.gates.size(); ++i) {
    const HGate& g = gates[b.gates[i]];
    target_matrix(g, theta, loc[i].m);
    loc[i].lt[0] = local(g.t[0]);
    loc[i].lt[1] = g.nt == 2 ? local(g.t[1]) : 0;
    loc[i].lc = 0;
    for (int j = 0; j < g.nc; ++j) loc[i].lc |= 1ull << local(g.c[j]);
  }
  std::vector<cd> col(D);
  for (uint64_t c = 0; c < D; ++c) {
    std::fill(col.begin(), col.end(), cd(0));
    col[c] = 1;
    for (size_t i = 0; i < b.gates.size(); ++i)
      apply_local(gates[b.gates[i]], loc[i].lt, loc[i].lc, loc[i].m, col.data(), k);
    for (uint64_t r = 0; r < D; ++r) M[r * D + c] = col[r];
  }
}

// ---------------------------------------------------------------- phase runs

// Phase-polynomial tracking: rows[q] is the parity mask, over the bits of the
// index at the start of the run, that bit q holds now. A CNOT (c -> t) sets
// rows[t] ^= rows[c]; a SWAP exchanges two rows; a diagonal gate on bit q
// contributes terms in rows[q] (and rows[c] for a control). Where every row is
// its own unit vector again, the run so far is diagonal in the original index.
static bool phase_terms_of(const HGate& g, const std::vector<uint64_t>& rows, std::vector<PhaseTerm>& out) {
  // angle a of the gate: RZ(a) = exp(-i a/2 Z), P(a) = diag(1, e^{ia})
  double a0 = 0, ascale = 0;
  int pidx = -1;
  bool rz = false;
  switch (g.kind) {
    case QS_GATE_Z: a0 = M_PI; break;
    case QS_GATE_S: a0 = M_PI / 2; break;
    case QS_GATE_SDG: a0 = -M_PI / 2; break;
    case QS_GATE_T: a0 = M_PI / 4; break;
    case QS_GATE_TDG: a0 = -M_PI / 4; break;
    case QS_GATE_RZ: rz = true; [[fallthrough]];
    case QS_GATE_P:
      a0 = g.param;
      if (g.parametric) { ascale = g.scale; pidx = g.param_index; }
      break;
    default: return false;
  }
  if (g.nt != 1 || g.nc > 1) return false;
  auto add = [&](uint64_t mask, double c) { out.push_back(PhaseTerm{mask, pidx, c * a0, c * ascale}); };
  const uint64_t mt = rows[g.t[0]];
  if (g.nc == 0) {
    // RZ(a): e^{-i a/2 s}; P(a) = e^{i a b}, b = (1 - s)/2
    add(mt, -0.5);
    if (!rz) add(0, 0.5);
  } else {
    // controlled on b_c = (1 - s_c)/2: RZ gives e^{-i a/4 s_t} e^{+i a/4 s_c s_t};
    // P gives e^{i a b_c b_t} = e^{i a/4 (1 - s_c - s_t + s_c s_t)}
    const uint64_t mc = rows[g.c[0]];
    add(mt, -0.25);
    add(mc ^ mt, 0.25);
    if (!rz) {
      add(mc, -0.25);
      add(0, 0.25);
    }
  }
  return true;
}

std::vector<PhaseRun> find_phase_runs(int n, const std::vector<HGate>& gates, int min_gates, int max_terms,
                                      int max_mixed, int low_bits) {
  std::vector<PhaseRun> runs;
  const int G = (int)gates.size();
  const uint64_t low = low_bits >= 64 ? ~0ull : ((1ull << low_bits) - 1);
  auto mixed = [&](uint64_t m) { return popc(m & low) >= 2 && (m & ~low) != 0; };
  std::vector<uint64_t> rows(n);
  std::vector<PhaseTerm> terms;
  int i = 0;
  while (i < G) {
    for (int q = 0; q < n; ++q) rows[q] = 1ull << q;
    terms.clear();
    int off = 0, nmixed = 0;        // rows not equal to their unit vector; mixed terms so far
    int best_end = -1;
    size_t best_terms = 0;
    uint64_t qm = 0, best_qm = 0;
    auto set_row = [&](int q, uint64_t v) {
      off -= rows[q] != (1ull << q);
      rows[q] = v;
      off += rows[q] != (1ull << q);
    };
    for (int h = i; h < G && h - i < 8192; ++h) {
      const HGate& g = gates[h];
      const size_t t0 = terms.size();
      if (g.kind == QS_GATE_X && g.nt == 1 && g.nc == 1) {
        set_row(g.t[0], rows[g.t[0]] ^ rows[g.c[0]]);
      } else if (g.kind == QS_GATE_SWAP && g.nc == 0) {
        const uint64_t a = rows[g.t[0]], b = rows[g.t[1]];
        set_row(g.t[0], b);
        set_row(g.t[1], a);
      } else if (!phase_terms_of(g, rows, terms)) {
        break;
      }
      for (size_t k = t0; k < terms.size(); ++k) nmixed += mixed(terms[k].mask);
      if ((int)terms.size() > max_terms || nmixed > max_mixed) break;
      qm |= g.qmask;
      if (off == 0) {
        best_end = h + 1;
        best_terms = terms.size();
        best_qm = qm;
      }
    }
    if (best_end - i >= min_gates) {
      PhaseRun r;
      r.begin = i;
      r.end = best_end;
      r.qmask = best_qm;
      r.terms.assign(terms.begin(), terms.begin() + best_terms);
      runs.push_back(std::move(r));
      i = best_end;
    } else {
      ++i;
    }
  }
  return runs;
}

// ---------------------------------------------------------------- passes

std::vector<PassRec> schedule_passes(int n, const std::vector<OpRec>& ops, int m, int L,
                                     std::vector<int>& order_out) {
  // Same greedy as the contraction, with width m and qubits 0..L-1 always in
  // the tile; ops move ahead of skipped ops they commute with.
  const int N = (int)ops.size();
  const uint64_t low = L >= 64 ? ~0ull : ((1ull << L) - 1);
  const uint64_t all = n >= 64 ? ~0ull : ((1ull << n) - 1);
  std::vector<char> done(N, 0);
  std::vector<PassRec> passes;
  std::vector<int> order;   // ops reordered pass by pass
  order.reserve(N);
  int first = 0;
  while (true) {
    while (first < N && done[first]) ++first;
    if (first >= N) break;
    PassRec pr;
    pr.op_begin = (int)order.size();
    std::vector<int> members{first};
    uint64_t Q = low | ops[first].qmask, blk_nd = 0, blk_d = 0;
    for (int h = first + 1; h < N; ++h) {
      if (done[h]) continue;
      const uint64_t qh = ops[h].qmask, dh = ops[h].dmask;
      const bool movable = (qh & blk_nd) == 0 && (qh & blk_d & ~dh) == 0;
      if (movable && popc(Q | qh) <= m) {
        members.push_back(h);
        Q |= qh;
      } else {
        blk_nd |= qh & ~dh;
        blk_d |= qh & dh;
      }
      if (blk_nd == all) break;
      if (popc(Q) >= m && (Q & ~blk_nd) == 0) break;
    }
    for (int h : members) { done[h] = 1; order.push_back(h); }
    // pad the tile to m qubits with the lowest unused qubits
    for (int b = 0; b < n && popc(Q) < m; ++b) Q |= 1ull << b;
    pr.tile = mask_bits(Q);
    pr.op_end = (int)order.size();
    passes.push_back(pr);
  }
  order_out = order;
  return passes;
}

}  // namespace qs
