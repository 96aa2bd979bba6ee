// C ABI of the simulator: state objects, plans, observables, adjoint gradient,
// batched execution. Host code only; every arithmetic step on a state runs in
// the CUDA kernels of kernels_*.cu.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <functional>
#include <map>
#include <memory>
#include <mutex>
#include <new>
#include <string>
#include <vector>

#include "planner.h"
#include "qs_error.h"
#include "qs_internal.h"

namespace qs {
int64_t launch_count();
}

using namespace qs;

namespace {

thread_local std::string g_err;

#define CK(expr)                                                                        \
  do {                                                                                  \
    cudaError_t _e = (expr);                                                            \
    if (_e != cudaSuccess)                                                              \
      throw Error(_e == cudaErrorMemoryAllocation ? QS_ERR_OOM : QS_ERR_CUDA,           \
                  std::string(#expr) + ": " + cudaGetErrorString(_e));                  \
  } while (0)

template <class F>
qs_status guard(F&& f) {
  try {
    f();
    return QS_OK;
  } catch (const Error& e) {
    g_err = e.what();
    return e.code;
  } catch (const std::bad_alloc&) {
    g_err = "host allocation failed";
    return QS_ERR_OOM;
  } catch (const std::exception& e) {
    g_err = e.what();
    return QS_ERR_CUDA;
  }
}

void require(bool c, const char* msg) {
  if (!c) throw Error(QS_ERR_ARG, msg);
}

void require_device() {
  int cnt = 0;
  cudaError_t e = cudaGetDeviceCount(&cnt);
  if (e != cudaSuccess || cnt == 0)
    throw Error(QS_ERR_CUDA, std::string("no CUDA device: ") + cudaGetErrorString(e));
}

// Device buffer (owning).
struct DevBuf {
  void* p = nullptr;
  size_t bytes = 0;
  DevBuf() = default;
  DevBuf(const DevBuf&) = delete;
  DevBuf& operator=(const DevBuf&) = delete;
  ~DevBuf() { release(); }
  void release() {
    if (p) cudaFree(p);
    p = nullptr;
    bytes = 0;
  }
  void ensure(size_t b) {
    if (b <= bytes) return;
    release();
    CK(cudaMalloc(&p, b));
    bytes = b;
  }
  template <class T> T* as() const { return (T*)p; }
};

size_t amp_bytes(qs_dtype dt) { return dt == QS_C64 ? 8 : 16; }

}  // namespace

namespace qs {
void set_last_error(const std::string& msg) { g_err = msg; }
}  // namespace qs

struct qs_state_s {
  int n = 0;
  qs_dtype dt = QS_C64;
  void* d = nullptr;
  bool owned = false;
  cudaStream_t st = nullptr;
  DevBuf scratch;     // reduction partials and small device arrays
  DevBuf scratch2;    // term lists
  size_t bytes() const { return amp_bytes(dt) << n; }
};

struct StreamPass {
  std::vector<int> gates;          // program order
  uint64_t high_mask = 0;          // batch-index qubits (>= l) the pass's gates touch
};

struct qs_plan_s {
  int n = 0;
  qs_dtype dt = QS_C64;
  qs_plan_opts opts{};
  int mode = QS_MODE_PER_GATE;
  std::vector<HGate> gates;
  std::vector<DevGate> dgates;
  std::vector<int32_t> pgates;     // indices of parametric gates
  int64_t nparams = 0;             // max param_index + 1
  // fused program
  std::vector<Block> blocks;
  std::vector<PassDesc> pdesc;
  std::vector<DevOp> dops;
  std::vector<OpRec> exec_ops;     // dops in global terms (introspection)
  std::vector<std::vector<int>> pass_tiles;
  std::vector<std::pair<int, int>> pass_ops;   // op range of each step in exec_ops
  std::vector<int64_t> block_off;  // complex offset in the block table, -1 if gate-wise
  // tensor-core passes and the execution order of all passes
  struct Step {
    int kind;   // 0 = tile pass (pdesc[idx]), 1 = tensor-core pass (tcdesc[idx]), 2 = phase pass (phdesc[idx])
    int idx;
  };
  // staggered multi-gate groups (per-gate plans built with QS_MODE_SMGP):
  // steps in program order, (group, -1) or (-1, gate)
  bool smgp = false;
  std::vector<SmgpDesc> smgp_groups;
  std::vector<std::pair<int, int>> smgp_steps;
  // diagonal phase runs (their own passes)
  std::vector<PhaseRun> runs;
  std::vector<PhasePassDesc> phdesc;
  std::vector<DevPhaseTerm> h_pterms;
  int64_t theta_stride = 0;        // entries per theta row of the last resolve
  bool theta_needed = false;       // some phase term depends on theta
  std::vector<Step> steps;
  std::vector<TcPassDesc> tcdesc;
  std::vector<uint16_t> h_wimg;    // per TC pass: bf16 hi image then lo image (64 KiB)
  int tc_prec = 3;
  int tc_pipe = 0;                 // single-state tensor-core pass: 0 bulk-copy staged, 1 register-staged
  bool df = false;                 // complex128 tile passes computed in FP32 pairs
  int64_t btab_elems = 0;
  // blocks whose matrices depend on theta, rebuilt on the device per batch row
  std::vector<DevBlock> h_dblocks;
  std::vector<DevMember> h_dmem;
  std::vector<char> tc_param;      // per tensor-core pass: its W image is rebuilt per row
  int btab_rows = 0, wimg_rows = 0; // rows allocated in d_btab / d_wimg
  std::vector<double2> h_btab;
  // device
  bool uploaded = false;
  DevBuf d_gates, d_pg, d_gtab, d_theta, d_ops, d_btab, d_wimg, d_err, d_dblocks, d_dmem, d_pterms, d_smgp;
  int gtab_rows = 0;
  qs_plan_info info{};
  // batched graph cache; captured and replayed on a plan-owned stream
  cudaGraphExec_t graph = nullptr;
  std::vector<void*> graph_key;
  cudaStream_t cap_stream = nullptr;
  cudaEvent_t ev_in = nullptr, ev_out = nullptr;
  DevBuf d_psis;                   // state pointers of the batch
  int64_t graph_launches = 0;      // kernel launches in one replay of the graph
  // measurement: events bracketing each launch of qs_plan_execute
  bool timing = false;
  std::vector<cudaEvent_t> events;
  std::vector<int> event_kind;     // launch kind of each bracketed launch (0 tile/per-gate, 1 tensor core)
  size_t events_used = 0;
  ~qs_plan_s() {
    if (graph) cudaGraphExecDestroy(graph);
    for (cudaEvent_t e : events) cudaEventDestroy(e);
    if (ev_in) cudaEventDestroy(ev_in);
    if (ev_out) cudaEventDestroy(ev_out);
    if (cap_stream) cudaStreamDestroy(cap_stream);
  }
  cudaEvent_t next_event() {
    if (events_used == events.size()) {
      cudaEvent_t e;
      CK(cudaEventCreate(&e));
      events.push_back(e);
    }
    return events[events_used++];
  }
};

namespace {

void fill_fixed_table(const qs_plan_s& p, std::vector<double2>& tab) {
  tab.assign(p.gates.size() * 16, make_double2(0, 0));
  for (size_t g = 0; g < p.gates.size(); ++g) {
    if (p.gates[g].parametric) continue;
    const int d = p.gates[g].nt == 1 ? 4 : 16;
    for (int k = 0; k < d; ++k) tab[g * 16 + k] = make_double2(p.gates[g].fixed[k].real(), p.gates[g].fixed[k].imag());
  }
}

void compute_blocks(qs_plan_s& p, const double* theta, bool only_parametric) {
  std::vector<cd> M;
  for (size_t b = 0; b < p.blocks.size(); ++b) {
    const Block& blk = p.blocks[b];
    if (p.block_off[b] < 0) continue;
    if (only_parametric && !blk.parametric) continue;
    if (blk.parametric && !theta) continue;
    block_matrix(blk, p.gates, theta, M);
    const size_t D = (size_t)1 << blk.qubits.size();
    double2* dst = p.h_btab.data() + p.block_off[b];
    if (blk.rep == OP_DIAG)
      for (size_t i = 0; i < D; ++i) dst[i] = make_double2(M[i * D + i].real(), M[i * D + i].imag());
    else
      for (size_t i = 0; i < D * D; ++i) dst[i] = make_double2(M[i].real(), M[i].imag());
  }
}

void ensure_gtab_rows(qs_plan_s& p, int rows) {
  if (rows <= p.gtab_rows) return;
  const size_t G = std::max<size_t>(1, p.gates.size());
  DevBuf nb;
  nb.ensure(sizeof(double2) * 16 * G * rows);
  std::vector<double2> tab;
  fill_fixed_table(p, tab);
  for (int r = 0; r < rows; ++r)
    CK(cudaMemcpy(nb.as<double2>() + (size_t)r * 16 * G, tab.data(), sizeof(double2) * 16 * p.gates.size(),
                  cudaMemcpyHostToDevice));
  std::swap(p.d_gtab.p, nb.p);
  std::swap(p.d_gtab.bytes, nb.bytes);
  p.gtab_rows = rows;
}

// Block table and W images with `rows` rows (batch rows for blocks rebuilt on
// the device); host-built entries live in row 0 and are read with stride 0.
void ensure_block_rows(qs_plan_s& p, int rows) {
  const bool per_row = !p.h_dblocks.empty();
  const int want = per_row ? rows : 1;
  if (want > p.btab_rows) {
    p.d_btab.release();
    p.d_btab.ensure(sizeof(double2) * std::max<int64_t>(1, p.btab_elems) * want);
    if (p.btab_elems)
      CK(cudaMemcpy(p.d_btab.p, p.h_btab.data(), sizeof(double2) * p.btab_elems, cudaMemcpyHostToDevice));
    p.btab_rows = want;
  }
  if (!p.tcdesc.empty() && want > p.wimg_rows) {
    p.d_wimg.release();
    p.d_wimg.ensure(sizeof(uint16_t) * p.h_wimg.size() * want);
    CK(cudaMemcpy(p.d_wimg.p, p.h_wimg.data(), sizeof(uint16_t) * p.h_wimg.size(), cudaMemcpyHostToDevice));
    p.wimg_rows = want;
  }
}

void build_device_blocks(qs_plan_s& p, int rows, cudaStream_t st) {
  if (p.h_dblocks.empty()) return;
  if (p.gtab_rows < rows || p.btab_rows < rows || (!p.tcdesc.empty() && p.wimg_rows < rows))
    throw Error(QS_ERR_CUDA, "internal: block tables have fewer rows than the batch");
  const size_t G = std::max<size_t>(1, p.gates.size());
  CK(launch_build_blocks(p.d_dblocks.as<DevBlock>(), (int)p.h_dblocks.size(), p.d_dmem.as<DevMember>(),
                         p.d_gtab.as<double2>(), (int64_t)(16 * G), rows, p.d_btab.as<double2>(), p.btab_elems,
                         p.d_wimg.as<uint16_t>(), (int64_t)p.h_wimg.size(), p.tc_prec == 4 ? 1 : 0, st));
}

void upload(qs_plan_s& p) {
  if (p.uploaded) return;
  const size_t G = p.gates.size();
  p.d_gates.ensure(sizeof(DevGate) * std::max<size_t>(1, G));
  if (G) CK(cudaMemcpy(p.d_gates.p, p.dgates.data(), sizeof(DevGate) * G, cudaMemcpyHostToDevice));
  p.d_pg.ensure(sizeof(int32_t) * std::max<size_t>(1, p.pgates.size()));
  if (!p.pgates.empty())
    CK(cudaMemcpy(p.d_pg.p, p.pgates.data(), sizeof(int32_t) * p.pgates.size(), cudaMemcpyHostToDevice));
  ensure_gtab_rows(p, 1);
  if (!p.dops.empty()) {
    p.d_ops.ensure(sizeof(DevOp) * p.dops.size());
    CK(cudaMemcpy(p.d_ops.p, p.dops.data(), sizeof(DevOp) * p.dops.size(), cudaMemcpyHostToDevice));
  }
  ensure_block_rows(p, 1);
  if (!p.h_dblocks.empty()) {
    p.d_dblocks.ensure(sizeof(DevBlock) * p.h_dblocks.size());
    CK(cudaMemcpy(p.d_dblocks.p, p.h_dblocks.data(), sizeof(DevBlock) * p.h_dblocks.size(), cudaMemcpyHostToDevice));
    p.d_dmem.ensure(sizeof(DevMember) * std::max<size_t>(1, p.h_dmem.size()));
    if (!p.h_dmem.empty())
      CK(cudaMemcpy(p.d_dmem.p, p.h_dmem.data(), sizeof(DevMember) * p.h_dmem.size(), cudaMemcpyHostToDevice));
  }
  if (!p.h_pterms.empty()) {
    p.d_pterms.ensure(sizeof(DevPhaseTerm) * p.h_pterms.size());
    CK(cudaMemcpy(p.d_pterms.p, p.h_pterms.data(), sizeof(DevPhaseTerm) * p.h_pterms.size(), cudaMemcpyHostToDevice));
  }
  for (PhasePassDesc& d : p.phdesc) CK(prepare_phase_pass(d, p.dt));
  if (!p.smgp_groups.empty()) {
    p.d_smgp.ensure(sizeof(SmgpDesc) * p.smgp_groups.size());
    CK(cudaMemcpy(p.d_smgp.p, p.smgp_groups.data(), sizeof(SmgpDesc) * p.smgp_groups.size(),
                  cudaMemcpyHostToDevice));
  }
  p.d_err.ensure(sizeof(int) * 4);
  CK(cudaMemset(p.d_err.p, 0, sizeof(int) * 4));
  // kernel attributes and occupancy, here and never during a stream capture
  for (const PassDesc& pd : p.pdesc) CK(prepare_tile_pass(pd, p.dt));
  if (!p.tcdesc.empty()) CK(prepare_tc_pass());
  if (!p.h_dblocks.empty()) CK(prepare_build_blocks());
  p.uploaded = true;
}

void check_state(const qs_state_s* s) { require(s != nullptr && s->d != nullptr, "null state"); }

// Issues the kernels of one circuit execution on `st` for batch row `row` of
// the gate table (theta already resolved into it).
void issue_circuit(qs_plan_s& p, void* psi, int row, cudaStream_t st, bool timed = false) {
  const size_t G = std::max<size_t>(1, p.gates.size());
  const double2* gtab = p.d_gtab.as<double2>() + (size_t)row * 16 * G;
  if (p.smgp) {
    for (const auto& s : p.smgp_steps) {
      if (timed) {
        CK(cudaEventRecord(p.next_event(), st));
        p.event_kind.push_back(0);
      }
      if (s.first < 0) {
        CK(launch_gate(psi, p.n, p.dt, p.dgates[s.second], gtab + (size_t)s.second * 16, false, st));
      } else {
        const SmgpDesc& d = p.smgp_groups[s.first];
        for (int T = 0; T < d.S; ++T)
          CK(launch_smgp_step(psi, p.n, p.dt, p.d_smgp.as<SmgpDesc>() + s.first, d, T, gtab, st));
      }
      if (timed) CK(cudaEventRecord(p.next_event(), st));
    }
    return;
  }
  const size_t nl = p.mode == QS_MODE_PER_GATE ? p.gates.size() : p.steps.size();
  for (size_t i = 0; i < nl; ++i) {
    if (timed) {
      CK(cudaEventRecord(p.next_event(), st));
      p.event_kind.push_back(p.mode != QS_MODE_PER_GATE && p.steps[i].kind == 1 ? 1 : 0);
    }
    if (p.mode == QS_MODE_PER_GATE) {
      CK(launch_gate(psi, p.n, p.dt, p.dgates[i], gtab + i * 16, false, st));
    } else if (p.steps[i].kind == 0) {
      CK(launch_tile_pass(psi, p.n, p.dt, p.pdesc[p.steps[i].idx], p.d_ops.as<DevOp>(), gtab,
                          p.d_btab.as<double2>(), 0, st));
    } else if (p.steps[i].kind == 2) {
      const double* th = p.theta_needed ? p.d_theta.as<double>() + (size_t)row * p.theta_stride : nullptr;
      CK(launch_phase_pass(psi, nullptr, 1, p.n, p.dt, p.d_pterms.as<DevPhaseTerm>(), p.phdesc[p.steps[i].idx], th,
                           p.theta_stride, st));
    } else {
      const int t = p.steps[i].idx;
      CK(launch_tc_pass(psi, p.n, p.tcdesc[t], p.d_wimg.as<uint16_t>() + (size_t)t * 32768, p.tc_prec,
                        p.tc_pipe, p.d_err.as<int>(), st));
    }
    if (timed) CK(cudaEventRecord(p.next_event(), st));
  }
}

// One launch per pass for all B states (fused / tensor plans): the kernels
// take the device array of state pointers and gate-table rows 16 G apart.
// States per wave of the batched schedule. Default: each pass covers the whole
// batch (one launch per pass). With reserved[4] = 1, when at least two states
// fit in about half of the L2 (64 MiB), every pass runs on one wave before the
// next wave starts, so after the first pass a wave's states come from L2; on
// GB300 the extra launches cost more than that saves (UCC n = 20, B = 64:
// 131 ms per batch in 8 waves against 106 ms pass by pass).
int batched_wave(const qs_plan_s& p, int B) {
  if (p.opts.reserved[4] != 1) return B;
  const int w = expval_wave_states(p.n, p.dt, B);
  return w >= 2 ? w : B;
}

// after_wave(w0, nb) runs once per wave, after its passes (the expectation values,
// while the wave is still in L2).
void issue_circuit_batched(qs_plan_s& p, void* const* d_psis, int B, cudaStream_t st,
                           const std::function<void(int, int)>& after_wave = nullptr) {
  const size_t G = std::max<size_t>(1, p.gates.size());
  if (p.gtab_rows < B || (!p.h_dblocks.empty() && (p.btab_rows < B || (!p.tcdesc.empty() && p.wimg_rows < B))))
    throw Error(QS_ERR_CUDA, "internal: tables have fewer rows than the batch");
  const int wave = batched_wave(p, B);
  for (int w0 = 0; w0 < B; w0 += wave) {
    const int nb = std::min(wave, B - w0);
    void* const* ps = d_psis + w0;
    for (const auto& stp : p.steps) {
      if (stp.kind == 2) {
        CK(launch_phase_pass(nullptr, ps, nb, p.n, p.dt, p.d_pterms.as<DevPhaseTerm>(), p.phdesc[stp.idx],
                             p.theta_needed ? p.d_theta.as<double>() + (size_t)w0 * p.theta_stride : nullptr,
                             p.theta_stride, st));
      } else if (stp.kind == 0) {
        CK(launch_tile_pass_batched(nullptr, ps, nb, (int64_t)(16 * G), p.btab_elems, w0, p.n, p.dt, p.pdesc[stp.idx],
                                    p.d_ops.as<DevOp>(), p.d_gtab.as<double2>() + (size_t)w0 * 16 * G,
                                    p.d_btab.as<double2>(), st));
      } else {
        const int64_t wstride = p.tc_param[stp.idx] ? (int64_t)p.h_wimg.size() : 0;
        CK(launch_tc_pass_batched(nullptr, ps, nb, wstride, p.n, p.tcdesc[stp.idx],
                                  p.d_wimg.as<uint16_t>() + (size_t)stp.idx * 32768 + (size_t)w0 * wstride, p.tc_prec,
                                  p.tc_pipe, p.d_err.as<int>(), st));
      }
    }
    if (after_wave) after_wave(w0, nb);
  }
}

void resolve_theta(qs_plan_s& p, const double* theta, size_t ntheta, int rows, cudaStream_t st) {
  if (p.pgates.empty()) return;
  if (p.gtab_rows < rows) throw Error(QS_ERR_CUDA, "internal: gate table has fewer rows than requested");
  require(theta != nullptr, "circuit has parameters but theta is NULL");
  require((int64_t)ntheta >= p.nparams, "theta has fewer entries than the circuit's parameter indices");
  p.d_theta.ensure(sizeof(double) * ntheta * rows);
  CK(cudaMemcpyAsync(p.d_theta.p, theta, sizeof(double) * ntheta * rows, cudaMemcpyHostToDevice, st));
  p.theta_stride = (int64_t)ntheta;
  const size_t G = std::max<size_t>(1, p.gates.size());
  CK(launch_resolve(p.d_gates.as<DevGate>(), p.d_pg.as<int32_t>(), (int)p.pgates.size(), p.d_theta.as<double>(),
                    (int64_t)ntheta, rows, p.d_gtab.as<double2>(), (int64_t)16 * G, st));
}

void execute(qs_plan_s& p, qs_state_s& s, const double* theta, size_t ntheta) {
  require(p.n == s.n && p.dt == s.dt, "plan and state differ in qubit count or dtype");
  upload(p);
  resolve_theta(p, theta, ntheta, 1, s.st);
  build_device_blocks(p, 1, s.st);
  issue_circuit(p, s.d, 0, s.st, p.timing);
  if (!p.tcdesc.empty()) {
    int err = 0;
    CK(cudaMemcpyAsync(&err, p.d_err.p, sizeof(int), cudaMemcpyDeviceToHost, s.st));
    CK(cudaStreamSynchronize(s.st));
    if (err) throw Error(QS_ERR_TIMEOUT, "tensor-core pass: an MMA completion wait timed out");
  }
}

// ---------------------------------------------------------------- plans

// bf16 with round-to-nearest-even (host side, for the tensor-core W image).
uint16_t bf16_rne(float f) {
  uint32_t u;
  std::memcpy(&u, &f, 4);
  if ((u & 0x7fffffffu) > 0x7f800000u) return (uint16_t)((u >> 16) | 0x40);
  u += 0x7fffu + ((u >> 16) & 1u);
  return (uint16_t)(u >> 16);
}

float bf16_to_float(uint16_t h) {
  const uint32_t u = (uint32_t)h << 16;
  float f;
  std::memcpy(&f, &u, 4);
  return f;
}

// fp16 with round-to-nearest-even (host side, for the tensor-core W image);
// subnormals kept, |f| >= 65520 rounds to infinity.
uint16_t f16_rne(float f) {
  uint32_t x;
  std::memcpy(&x, &f, 4);
  const uint16_t sign = (uint16_t)((x >> 16) & 0x8000u);
  const uint32_t ax = x & 0x7fffffffu;
  if (ax > 0x7f800000u) return (uint16_t)(sign | 0x7e00u);
  if (ax >= 0x477ff000u) return (uint16_t)(sign | 0x7c00u);
  if (ax < 0x38800000u) {   // below 2^-14: a multiple of 2^-24 (the scaling is exact)
    const float q = std::fabs(f) * 16777216.0f;
    return (uint16_t)(sign | (uint16_t)std::nearbyint(q));   // 1024 encodes the smallest normal
  }
  uint32_t h = ((ax >> 23) - 112u) << 10 | ((ax >> 13) & 0x3ffu);
  const uint32_t rem = ax & 0x1fffu;
  if (rem > 0x1000u || (rem == 0x1000u && (h & 1u))) ++h;
  return (uint16_t)(sign | h);
}

float f16_to_float(uint16_t h) {
  const uint32_t e = (h >> 10) & 0x1fu, m = h & 0x3ffu;
  float v;
  if (e == 0) v = std::ldexp((float)m, -24);
  else if (e == 31) v = m ? NAN : INFINITY;
  else v = std::ldexp((float)(m | 0x400u), (int)e - 25);
  return (h & 0x8000u) ? -v : v;
}

// Byte offset of a 16-bit element (row, k) in a K-major 128-byte-swizzled operand
// of 128 rows (two 16 KiB atoms of 64 elements along K).
size_t sw128_offset_host(uint32_t row, uint32_t k) {
  const uint32_t atom = k >> 6, kk = k & 63;
  const uint32_t chunk = (kk >> 3) ^ (row & 7);
  return (size_t)atom * 16384 + row * 128 + chunk * 16 + (kk & 7) * 2;
}

// W image of a 64x64 complex block U: element (n, k) of the N x K operand is
// W[k][n] of the real embedding (see the tensor-core kernel), rounded to FP32
// and split into hi (first 32 KiB) and lo (second 32 KiB) parts: fp16 for
// tensor-core precision 4, bf16 otherwise (the same steps as the device builder).
void build_w_image(const double2* U, uint16_t* img, bool half) {
  for (uint32_t nn = 0; nn < 128; ++nn)
    for (uint32_t k = 0; k < 128; ++k) {
      const uint32_t co = nn >> 1, b = nn & 1, ci = k >> 1, a = k & 1;
      const float ur = (float)U[co * 64 + ci].x, ui = (float)U[co * 64 + ci].y;
      const float w = (a == 0) ? (b == 0 ? ur : ui) : (b == 0 ? -ui : ur);
      uint16_t hi, lo;
      if (half) {
        hi = f16_rne(w);
        lo = f16_rne(w - f16_to_float(hi));
      } else {
        hi = bf16_rne(w);
        lo = bf16_rne(w - bf16_to_float(hi));
      }
      const size_t off = sw128_offset_host(nn, k) / 2;
      img[off] = hi;
      img[16384 + off] = lo;
    }
}

float w_to_float(uint16_t v, bool half) { return half ? f16_to_float(v) : bf16_to_float(v); }

// Records a block whose matrix is rebuilt on the device from theta (kind: 0
// dense, 1 diagonal, 2 tensor-core W image; out = table offset or image index).
void register_device_block(qs_plan_s& P, const Block& blk, int kind, int64_t out) {
  DevBlock d;
  std::memset(&d, 0, sizeof(d));
  d.k = (int)blk.qubits.size();
  d.kind = kind;
  d.out = out;
  d.mem_begin = (int)P.h_dmem.size();
  auto local = [&](int q) {
    return (int)(std::lower_bound(blk.qubits.begin(), blk.qubits.end(), q) - blk.qubits.begin());
  };
  for (int gi : blk.gates) {
    const HGate& g = P.gates[gi];
    DevMember m;
    std::memset(&m, 0, sizeof(m));
    m.gate = gi;
    m.nt = g.nt;
    m.t0 = local(g.t[0]);
    m.t1 = g.nt == 2 ? local(g.t[1]) : 0;
    for (int k = 0; k < g.nc; ++k) m.cmask |= 1u << local(g.c[k]);
    m.form = g.form;
    P.h_dmem.push_back(m);
  }
  d.mem_end = (int)P.h_dmem.size();
  P.h_dblocks.push_back(d);
}

void emit_tile_passes(qs_plan_s& P, const std::vector<OpRec>& ops, const std::vector<PassRec>& passes,
                      const std::vector<int>& order, int low_qubits, qs_plan_info& in) {
  const qs_dtype dt = P.dt;
  for (const PassRec& pr : passes) {
    PassDesc pd;
    std::memset(&pd, 0, sizeof(pd));
    pd.df = P.df ? 1 : 0;
    pd.m = (int)pr.tile.size();
    pd.L = std::min(low_qubits, pd.m);
    pd.nhigh = pd.m - pd.L;
    for (int j = 0; j < pd.nhigh; ++j) pd.high[j] = pr.tile[pd.L + j];
    for (int j = 0; j < pd.L; ++j) require(pr.tile[j] == j, "internal: tile lacks low qubits");
    auto local = [&](int q) {
      return (int)(std::lower_bound(pr.tile.begin(), pr.tile.end(), q) - pr.tile.begin());
    };
    pd.op_begin = (int)P.dops.size();
    pd.kmax = 0;
    for (int oi = pr.op_begin; oi < pr.op_end; ++oi) {
      const OpRec& r = ops[order[oi]];
      DevOp d;
      std::memset(&d, 0, sizeof(d));
      d.type = r.type;
      if (r.type == OP_GATE) {
        const HGate& g = P.gates[r.gate];
        d.form = g.form;
        d.t0 = local(g.t[0]);
        d.t1 = g.nt == 2 ? local(g.t[1]) : -1;
        std::vector<int> ins;
        if (g.form != FORM_DIAG1)
          for (int k = 0; k < g.nt; ++k) ins.push_back(local(g.t[k]));
        for (int k = 0; k < g.nc; ++k) {
          ins.push_back(local(g.c[k]));
          d.cmask |= 1u << local(g.c[k]);
        }
        std::sort(ins.begin(), ins.end());
        d.nins = (int)ins.size();
        for (int k = 0; k < d.nins; ++k) d.ins[k] = ins[k];
        d.mat = r.gate;
        pd.mbuf_elems = std::max(pd.mbuf_elems, 16);
        in.flops_per_amp += 2 * gate_fma_per_amp(g);
        in.max_block_qubits = std::max(in.max_block_qubits, __builtin_popcountll(g.qmask));
      } else {
        const Block& blk = P.blocks[r.block];
        d.k = (int)blk.qubits.size();
        for (int j = 0; j < d.k; ++j) d.ins[j] = local(blk.qubits[j]);
        d.mat = (int32_t)P.block_off[r.block];
        d.per_row = blk.parametric ? 1 : 0;
        if (r.type == OP_DENSE) {
          pd.kmax = std::max(pd.kmax, d.k);
          pd.mbuf_elems = std::max(pd.mbuf_elems, 1 << (2 * d.k));
          in.flops_per_amp += 8.0 * (1 << d.k);
        } else {
          pd.mbuf_elems = std::max(pd.mbuf_elems, 1 << d.k);
          in.flops_per_amp += 8.0;
        }
        in.max_block_qubits = std::max(in.max_block_qubits, d.k);
      }
      P.dops.push_back(d);
      P.exec_ops.push_back(r);
    }
    pd.op_end = (int)P.dops.size();
    require(tile_smem_bytes(pd.m, pd.nhigh, pd.mbuf_elems, dt) <= 227 * 1024,
            "tile does not fit in shared memory: lower tile_qubits");
    P.steps.push_back({0, (int)P.pdesc.size()});
    P.pdesc.push_back(pd);
    P.pass_tiles.push_back(pr.tile);
    P.pass_ops.push_back({pd.op_begin, pd.op_end});
  }
}

// Terms of a phase run sorted into the classes the phase kernel expects
// (repeated (mask, parameter) pairs merged), appended to the plan's array.
void emit_phase_pass(qs_plan_s& P, const OpRec& r, qs_plan_info& in) {
  const PhaseRun& run = P.runs[r.block];
  const uint64_t low = (1ull << kPhaseChunkBits) - 1;
  std::map<std::pair<uint64_t, int>, PhaseTerm> merged;
  for (const PhaseTerm& t : run.terms) {
    PhaseTerm& m = merged[{t.mask, t.pidx}];
    m.mask = t.mask;
    m.pidx = t.pidx;
    m.alpha0 += t.alpha0;
    m.coef += t.coef;
  }
  auto cls = [&](uint64_t m) {   // 0 LOW, 1 + u LIN, 13 HIGH, 14 MIXED
    const int nlo = __builtin_popcountll(m & low);
    if (nlo == 0) return kPhaseChunkBits + 1;
    if (nlo == 1) return 1 + __builtin_ctzll(m & low);
    return (m & ~low) ? kPhaseChunkBits + 2 : 0;
  };
  std::vector<PhaseTerm> ts;
  for (auto& kv : merged) ts.push_back(kv.second);
  std::stable_sort(ts.begin(), ts.end(), [&](const PhaseTerm& a, const PhaseTerm& b) { return cls(a.mask) < cls(b.mask); });
  PhasePassDesc d;
  std::memset(&d, 0, sizeof(d));
  d.term_off = (int32_t)P.h_pterms.size();
  d.nterms = (int32_t)ts.size();
  d.df = P.df ? 1 : 0;
  int k = 0;
  auto skip_class = [&](int c) { while (k < (int)ts.size() && cls(ts[k].mask) == c) ++k; };
  skip_class(0);
  d.nlow = k;
  for (int u = 0; u < kPhaseChunkBits; ++u) {
    d.lin_off[u] = k;
    skip_class(1 + u);
  }
  d.lin_off[kPhaseChunkBits] = k;
  d.high_begin = k;
  skip_class(kPhaseChunkBits + 1);
  d.mixed_begin = k;
  require(d.nterms <= kPhaseMaxTerms && d.nterms - d.mixed_begin <= kPhaseMaxMixed, "internal: phase run too large");
  for (const PhaseTerm& t : ts) {
    DevPhaseTerm dt;
    std::memset(&dt, 0, sizeof(dt));
    dt.mask = t.mask;
    dt.pidx = t.pidx;
    dt.alpha0 = t.alpha0;
    dt.coef = t.coef;
    P.h_pterms.push_back(dt);
    if (t.pidx >= 0 && t.coef != 0) P.theta_needed = true;
  }
  DevOp op;
  std::memset(&op, 0, sizeof(op));
  op.type = OP_PHASE;
  const int b = (int)P.dops.size();
  P.dops.push_back(op);
  P.exec_ops.push_back(r);
  P.steps.push_back({2, (int)P.phdesc.size()});
  P.phdesc.push_back(d);
  std::vector<int> qs;
  for (int q = 0; q < P.n; ++q)
    if (run.qmask & (1ull << q)) qs.push_back(q);
  P.pass_tiles.push_back(qs);
  P.pass_ops.push_back({b, b + 1});
  in.flops_per_amp += 18.0;   // three complex products per amplitude
}

void emit_tc_pass(qs_plan_s& P, const OpRec& r, qs_plan_info& in) {
  const Block& blk = P.blocks[r.block];
  TcPassDesc t;
  std::memset(&t, 0, sizeof(t));
  for (int j = 0; j < 6; ++j) t.col[j] = blk.qubits[j];
  int nr = 0;
  for (int q = 0; q < P.n && nr < 7; ++q)
    if (std::find(blk.qubits.begin(), blk.qubits.end(), q) == blk.qubits.end()) t.row[nr++] = q;
  require(nr == 7, "internal: tensor-core tile needs 7 row qubits");
  std::vector<int> tile(t.row, t.row + 7);
  tile.insert(tile.end(), t.col, t.col + 6);
  std::sort(tile.begin(), tile.end());
  for (int j = 0; j < 13; ++j) t.tile[j] = tile[j];
  const size_t w0 = P.h_wimg.size();
  P.h_wimg.resize(w0 + 32768);
  if (blk.parametric)
    register_device_block(P, blk, 2, (int64_t)P.tcdesc.size());   // W image rebuilt per row on the device
  else
    build_w_image(P.h_btab.data() + P.block_off[r.block], P.h_wimg.data() + w0, P.tc_prec == 4);
  P.tc_param.push_back(blk.parametric ? 1 : 0);
  DevOp d;
  std::memset(&d, 0, sizeof(d));
  d.type = OP_TC;
  d.k = 6;
  const int b = (int)P.dops.size();
  P.dops.push_back(d);
  P.exec_ops.push_back(r);
  P.steps.push_back({1, (int)P.tcdesc.size()});
  P.tcdesc.push_back(t);
  P.pass_tiles.push_back(tile);
  P.pass_ops.push_back({b, b + 1});
  in.flops_per_amp += 8.0 * 64;
  in.max_block_qubits = std::max(in.max_block_qubits, 6);
}


void default_opts(qs_plan_opts& o, qs_dtype dt, int n) {
  if (o.fuse_k <= 0) o.fuse_k = dt == QS_C64 ? 4 : 3;
  if (o.tile_qubits <= 0) o.tile_qubits = dt == QS_C64 ? 12 : 11;
  if (o.low_qubits <= 0) o.low_qubits = dt == QS_C64 ? 5 : 4;
  if (o.tile_qubits > n) o.tile_qubits = n;
  if (o.low_qubits > o.tile_qubits) o.low_qubits = o.tile_qubits;
}

// Staggered multi-gate groups (Section 3.3): runs of consecutive uncontrolled
// one-target gates on distinct qubits, S = the largest power of two <= 8 that
// the run and the register allow (S targets plus lg S segment qubits); the
// segment qubits are the highest qubits no member targets.
void plan_smgp(qs_plan_s& p) {
  const int G = (int)p.gates.size(), n = p.n;
  qs_plan_info& in = p.info;
  in.launches = 0;
  in.sweeps = 0;
  int i = 0;
  while (i < G) {
    uint64_t used = 0;
    int cnt = 0;
    while (i + cnt < G && cnt < kSmgpMax) {
      const HGate& g = p.gates[i + cnt];
      if (g.nt != 1 || g.nc != 0 || (used & g.qmask)) break;
      used |= g.qmask;
      ++cnt;
    }
    int S = 1, lgS = 0;
    while (2 * S <= cnt && 2 * S + lgS + 1 <= n) {
      S *= 2;
      ++lgS;
    }
    if (S < 2) {
      p.smgp_steps.push_back({-1, i});
      in.launches += 1;
      in.sweeps += gate_sweep_fraction(p.gates[i]);
      ++i;
      continue;
    }
    SmgpDesc d;
    std::memset(&d, 0, sizeof(d));
    d.S = S;
    d.lgS = lgS;
    uint64_t targets = 0;
    for (int j = 0; j < S; ++j) targets |= p.gates[i + j].qmask;
    std::vector<int> seg;
    for (int q = n - 1; q >= 0 && (int)seg.size() < lgS; --q)
      if (!(targets & (1ull << q))) seg.push_back(q);
    std::sort(seg.begin(), seg.end());
    for (int s = 0; s < S; ++s) {
      uint64_t o = 0;
      for (int b = 0; b < lgS; ++b) o |= (uint64_t)((s >> b) & 1) << seg[b];
      d.seg_or[s] = o;
    }
    for (int j = 0; j < S; ++j) {
      const HGate& g = p.gates[i + j];
      d.gate[j] = i + j;
      d.form[j] = g.form;
      d.t[j] = g.t[0];
      std::vector<int> pos(seg);
      pos.push_back(g.t[0]);
      std::sort(pos.begin(), pos.end());
      for (int k = 0; k < 4; ++k) d.pos[j][k] = k < (int)pos.size() ? pos[k] : 63;
    }
    p.smgp_steps.push_back({(int)p.smgp_groups.size(), -1});
    p.smgp_groups.push_back(d);
    in.launches += S;
    in.sweeps += S;
    i += S;
  }
  in.passes = in.launches;
}

// no_merge: every gate stays its own op (the reverse sweep of the adjoint gradient).
qs_plan_s* create_plan(int n, qs_dtype dt, const qs_gate* gates, size_t ng, const qs_plan_opts* opts,
                       bool no_merge = false) {
  require(n >= 1 && n <= kMaxQubits, "n out of range");
  require(dt == QS_C64 || dt == QS_C128, "bad dtype");
  require(ng == 0 || gates != nullptr, "gates is NULL");
  auto p = std::make_unique<qs_plan_s>();
  p->n = n;
  p->dt = dt;
  if (opts) p->opts = *opts;
  p->mode = p->opts.mode;
  require(p->mode == QS_MODE_PER_GATE || p->mode == QS_MODE_FUSED || p->mode == QS_MODE_TENSOR ||
          p->mode == QS_MODE_SMGP, "bad mode");
  if (p->mode == QS_MODE_SMGP) {   // a per-gate plan whose independent gate runs are staggered
    p->smgp = true;
    p->mode = QS_MODE_PER_GATE;
  }
  resolve_gates(n, gates, ng, p->gates);
  for (size_t g = 0; g < p->gates.size(); ++g) {
    p->dgates.push_back(make_dev_gate(p->gates[g]));
    if (p->gates[g].parametric) {
      p->pgates.push_back((int32_t)g);
      p->nparams = std::max<int64_t>(p->nparams, p->gates[g].param_index + 1);
    }
  }
  qs_plan_info& in = p->info;
  in.gates = (int64_t)ng;
  for (const HGate& g : p->gates) in.per_gate_sweeps += gate_sweep_fraction(g);
  if (p->mode == QS_MODE_PER_GATE) {
    in.blocks = (int64_t)ng;
    in.passes = (int64_t)ng;
    in.launches = (int64_t)ng;
    in.sweeps = in.per_gate_sweeps;
    if (p->smgp) plan_smgp(*p);
    for (const HGate& g : p->gates) in.flops_per_amp += 2 * gate_fma_per_amp(g);
    in.max_block_qubits = 0;
    for (const HGate& g : p->gates) in.max_block_qubits = std::max(in.max_block_qubits, __builtin_popcountll(g.qmask));
    return p.release();
  }
  qs_plan_opts& o = p->opts;
  require(o.tile_qubits <= 14 && o.tile_qubits >= 0, "tile_qubits out of range (1..14)");
  require(o.low_qubits >= 0 && o.fuse_k >= 0, "negative option");
  bool tensor = p->mode == QS_MODE_TENSOR;
  if (tensor) {
    if (dt != QS_C64) throw Error(QS_ERR_UNSUPPORTED, "tensor-core mode needs complex64 states");
    require(o.tc_precision == 0 || o.tc_precision == 1 || o.tc_precision == 3 || o.tc_precision == 4,
            "tc_precision must be 1, 3 or 4");
    p->tc_prec = o.tc_precision == 0 ? 4 : o.tc_precision;
    require(o.reserved[1] == 0 || o.reserved[1] == 1, "tensor-core pipeline (reserved[1]) must be 0 or 1");
    p->tc_pipe = o.reserved[1];
    if (n < 13) tensor = false;   // a tensor-core tile needs 13 qubits; smaller states use CUDA-core blocks
  }
  const int user_k = o.fuse_k;
  if (tensor) o.fuse_k = 0;
  default_opts(o, dt, n);
  require(o.fuse_k >= 1 && o.fuse_k <= 5, "fuse_k out of range (1..5 on CUDA cores)");
  require(o.tile_qubits >= 1 && o.tile_qubits <= 14, "tile_qubits out of range");
  require(o.low_qubits >= 1, "low_qubits must be >= 1");
  require(o.tile_qubits - o.low_qubits >= std::min(o.fuse_k, n - o.low_qubits) || o.tile_qubits == n,
          "tile_qubits - low_qubits must be >= fuse_k");
  int widest = 0;
  for (const HGate& g : p->gates) widest = std::max(widest, __builtin_popcountll(g.qmask));
  require(o.low_qubits + std::max(widest, o.fuse_k) <= 14 || o.tile_qubits == n,
          "low_qubits + widest gate must fit a 14-qubit tile");
  PlanOptions po;
  po.k = o.paper_mode ? 2 : (tensor ? (user_k == 5 ? 5 : 6) : o.fuse_k);
  po.paper = o.paper_mode != 0;
  po.amp_bytes = (int)amp_bytes(dt);
  // GB300: FP32 FMA 128 lanes/clk/SM, FP64 about 1/59 of that (measured),
  // shared memory 128 B/clk/SM -> one byte costs one FP32 FMA slot.
  // reserved[3] = 1: complex128 tile passes in FP32 pairs, about 15 FP32
  // instructions per FMA (a pair product and a pair sum)
  require(o.reserved[3] == 0 || o.reserved[3] == 1, "complex128 arithmetic (reserved[3]) must be 0 or 1");
  p->df = dt == QS_C128 && o.reserved[3] == 1;
  po.fp_weight = dt == QS_C64 ? 1.0 : (p->df ? 15.0 : 59.0);
  po.smem_weight = 1.0;
  po.fuse_parametric = o.fuse_parametric != 0;
  po.no_merge = no_merge;
  // Diagonal phase runs (reserved[2]: least gates per run, 0 = 2n, < 0 = none)
  // become their own passes; the gates between them are contracted segment by
  // segment, so no block moves across a run.
  const int phase_min = o.reserved[2] == 0 ? std::max(16, 2 * n) : o.reserved[2];
  if (!no_merge && !po.paper && phase_min > 0 && n >= kPhaseChunkBits)
    p->runs = find_phase_runs(n, p->gates, phase_min, kPhaseMaxTerms, kPhaseMaxMixed, kPhaseChunkBits);
  std::vector<std::pair<int, int>> items;   // (0, block) or (1, run) in program order
  {
    int pos = 0;
    auto contract_range = [&](int b, int e) {
      if (b >= e) return;
      std::vector<HGate> sub(p->gates.begin() + b, p->gates.begin() + e);
      for (Block& blk : contract(n, sub, po)) {
        for (int& g : blk.gates) g += b;
        items.push_back({0, (int)p->blocks.size()});
        p->blocks.push_back(std::move(blk));
      }
    };
    for (size_t r = 0; r < p->runs.size(); ++r) {
      contract_range(pos, p->runs[r].begin);
      items.push_back({1, (int)r});
      pos = p->runs[r].end;
    }
    contract_range(pos, (int)p->gates.size());
  }
  if (tensor) {
    // A block worth a tensor-core pass (one HBM sweep) carries many gates;
    // it is padded to 6 qubits with the highest qubits it does not touch.
    const int tc_min_gates = o.reserved[0] > 0 ? o.reserved[0] : 10;
    for (Block& blk : p->blocks) {
      if ((int)blk.gates.size() >= tc_min_gates) {
        blk.rep = OP_TC;
        blk.diag = false;
        for (int q = n - 1; q >= 0 && blk.qubits.size() < 6; --q)
          if (std::find(blk.qubits.begin(), blk.qubits.end(), q) == blk.qubits.end()) blk.qubits.push_back(q);
        std::sort(blk.qubits.begin(), blk.qubits.end());
      } else if (blk.qubits.size() > 5 || (blk.rep == OP_DENSE && (int)blk.qubits.size() > o.fuse_k)) {
        blk.rep = OP_GATE;
      }
    }
  }
  // ops in emission order
  std::vector<OpRec> ops;
  p->block_off.assign(p->blocks.size(), -1);
  for (const auto& it : items) {
    if (it.first == 1) {
      const PhaseRun& run = p->runs[it.second];
      ops.push_back(OpRec{OP_PHASE, -1, it.second, run.qmask, run.qmask});
      continue;
    }
    const size_t b = (size_t)it.second;
    const Block& blk = p->blocks[b];
    uint64_t qm = 0;
    for (int q : blk.qubits) qm |= 1ull << q;
    if (blk.rep == OP_GATE) {
      for (int g : blk.gates) ops.push_back(OpRec{OP_GATE, g, -1, p->gates[g].qmask, p->gates[g].dmask});
    } else {
      ops.push_back(OpRec{blk.rep, -1, (int)b, qm, blk.rep == OP_TC ? 0 : blk.dmask});
      p->block_off[b] = p->btab_elems;
      const int64_t D = 1ll << blk.qubits.size();
      p->btab_elems += blk.rep == OP_DIAG ? D : D * D;
      if (blk.parametric && blk.rep != OP_TC)
        register_device_block(*p, blk, blk.rep == OP_DIAG ? 1 : 0, p->block_off[b]);
    }
  }
  p->h_btab.assign(std::max<int64_t>(1, p->btab_elems), make_double2(0, 0));
  compute_blocks(*p, nullptr, false);
  in.blocks = 0;
  for (const Block& b : p->blocks) in.blocks += b.rep == OP_GATE ? (int64_t)b.gates.size() : 1;
  in.blocks += (int64_t)p->runs.size();
  in.max_block_qubits = 0;
  // Runs of CUDA-core ops between tensor-core ops become tile passes.
  std::vector<OpRec> seg;
  auto flush = [&]() {
    if (seg.empty()) return;
    std::vector<int> order;
    std::vector<PassRec> passes = schedule_passes(n, seg, o.tile_qubits, o.low_qubits, order);
    emit_tile_passes(*p, seg, passes, order, o.low_qubits, in);
    seg.clear();
  };
  for (const OpRec& r : ops) {
    if (r.type != OP_TC && r.type != OP_PHASE) {
      seg.push_back(r);
      continue;
    }
    flush();
    if (r.type == OP_TC)
      emit_tc_pass(*p, r, in);
    else
      emit_phase_pass(*p, r, in);
  }
  flush();
  in.passes = (int64_t)p->steps.size();
  in.launches = in.passes;
  in.sweeps = (double)in.passes;
  in.tile_qubits = o.tile_qubits;
  in.low_qubits = o.low_qubits;
  return p.release();
}

// ---------------------------------------------------------------- observables

struct TermGroup {
  uint64_t x;
  std::vector<int> idx;   // term indices
};

std::vector<TermGroup> group_terms(int n, const qs_pauli_term* t, size_t nt) {
  std::map<uint64_t, std::vector<int>> m;
  const uint64_t valid = n >= 64 ? ~0ull : ((1ull << n) - 1);
  for (size_t j = 0; j < nt; ++j) {
    require(((t[j].xmask | t[j].zmask) & ~valid) == 0, "Pauli term acts on a qubit >= n");
    m[t[j].xmask].push_back((int)j);
  }
  std::vector<TermGroup> g;
  for (auto& kv : m) g.push_back(TermGroup{kv.first, kv.second});
  return g;
}

// Sign and factor turning the kernel's per-string sum into <P> (see k_expval_x).
double term_factor(const qs_pauli_term& t) {
  if (t.xmask == 0) return 1.0;
  const int ny = __builtin_popcountll(t.xmask & t.zmask);
  if ((ny & 1) == 0) return ((ny / 2) & 1) ? -2.0 : 2.0;
  return (((ny + 1) / 2) & 1) ? -2.0 : 2.0;
}

struct PreparedTerms {
  std::vector<TermGroup> groups;
  std::vector<uint64_t> zlist;        // group order
  std::vector<int> term_of;           // term index per zlist entry
  std::vector<std::pair<int, int>> launches;   // (group, offset into zlist) per launch, count via chunk
  std::vector<int> counts;
};

constexpr int kZPerLaunch = 8;

PreparedTerms prepare_terms(int n, const qs_pauli_term* t, size_t nt) {
  PreparedTerms P;
  P.groups = group_terms(n, t, nt);
  for (size_t gi = 0; gi < P.groups.size(); ++gi) {
    const auto& g = P.groups[gi];
    for (size_t c = 0; c < g.idx.size(); c += kZPerLaunch) {
      const int cnt = (int)std::min<size_t>(kZPerLaunch, g.idx.size() - c);
      P.launches.push_back({(int)gi, (int)P.zlist.size()});
      P.counts.push_back(cnt);
      for (int k = 0; k < cnt; ++k) {
        P.zlist.push_back(t[g.idx[c + k]].zmask);
        P.term_of.push_back(g.idx[c + k]);
      }
    }
  }
  return P;
}

// Issues the expval kernels; per-string results land in d_out[zlist order].
void issue_expval(const qs_state_s& s, const PreparedTerms& P, const uint64_t* d_z, double* d_partials,
                  double* d_out, cudaStream_t st) {
  for (size_t l = 0; l < P.launches.size(); ++l) {
    const auto& L = P.launches[l];
    CK(launch_expval_x(s.d, s.n, s.dt, P.groups[L.first].x, d_z + L.second, nullptr, P.counts[l], d_partials,
                       d_out + L.second, st));
  }
}

double combine_expval(const PreparedTerms& P, const qs_pauli_term* t, const double* vals) {
  double e = 0;
  for (size_t k = 0; k < P.term_of.size(); ++k) {
    const qs_pauli_term& tt = t[P.term_of[k]];
    e += tt.coeff * term_factor(tt) * vals[k];
  }
  return e;
}

size_t partial_bytes(int rows) { return sizeof(double) * (size_t)reduce_blocks() * rows; }

double expval_sync(qs_state_s& s, const qs_pauli_term* t, size_t nt) {
  if (nt == 0) return 0.0;
  require(t != nullptr, "terms is NULL");
  PreparedTerms P = prepare_terms(s.n, t, nt);
  const size_t zb = sizeof(uint64_t) * P.zlist.size();
  const size_t ob = sizeof(double) * P.zlist.size();
  s.scratch.ensure(partial_bytes(kZPerLaunch) + ob);
  s.scratch2.ensure(zb);
  double* d_part = s.scratch.as<double>();
  double* d_out = d_part + (size_t)reduce_blocks() * kZPerLaunch;
  CK(cudaMemcpyAsync(s.scratch2.p, P.zlist.data(), zb, cudaMemcpyHostToDevice, s.st));
  issue_expval(s, P, s.scratch2.as<uint64_t>(), d_part, d_out, s.st);
  std::vector<double> vals(P.zlist.size());
  CK(cudaMemcpyAsync(vals.data(), d_out, ob, cudaMemcpyDeviceToHost, s.st));
  CK(cudaStreamSynchronize(s.st));
  return combine_expval(P, t, vals.data());
}

// Uploads x, z and c * i^{ny} for H|psi>; returns device pointers inside `buf`.
void upload_pauli_apply(const qs_pauli_term* t, size_t nt, DevBuf& buf, cudaStream_t st, uint64_t** dx,
                        uint64_t** dz, double2** dph, std::vector<unsigned char>& host) {
  const size_t b = (sizeof(uint64_t) * 2 + sizeof(double2)) * nt;
  host.resize(std::max<size_t>(b, 1));
  uint64_t* hx = (uint64_t*)host.data();
  uint64_t* hz = hx + nt;
  double2* hp = (double2*)(hz + nt);
  for (size_t j = 0; j < nt; ++j) {
    hx[j] = t[j].xmask;
    hz[j] = t[j].zmask;
    const int ny = __builtin_popcountll(t[j].xmask & t[j].zmask) & 3;
    const double c = t[j].coeff;
    hp[j] = ny == 0 ? make_double2(c, 0) : ny == 1 ? make_double2(0, c) : ny == 2 ? make_double2(-c, 0)
                                                                                  : make_double2(0, -c);
  }
  buf.ensure(std::max<size_t>(b, 16));
  CK(cudaMemcpyAsync(buf.p, host.data(), b, cudaMemcpyHostToDevice, st));
  *dx = buf.as<uint64_t>();
  *dz = *dx + nt;
  *dph = (double2*)(*dz + nt);
}

}  // namespace

// ---------------------------------------------------------------- autotuner

struct TuneEntry {
  qs_plan_opts opts;
  double ms;
};
std::mutex g_tune_mu;
std::map<std::vector<uint64_t>, TuneEntry> g_tune_cache;

uint64_t fnv1a(const void* data, size_t bytes, uint64_t h = 1469598103934665603ull) {
  const unsigned char* p = (const unsigned char*)data;
  for (size_t i = 0; i < bytes; ++i) {
    h ^= p[i];
    h *= 1099511628211ull;
  }
  return h;
}

std::vector<qs_plan_opts> tune_candidates(int n, qs_dtype dt) {
  std::vector<qs_plan_opts> c;
  auto add = [&](int mode, int k, int m, int L, int tcmin) {
    qs_plan_opts o;
    std::memset(&o, 0, sizeof(o));
    o.mode = mode;
    o.fuse_k = k;
    o.tile_qubits = m;
    o.low_qubits = L;
    o.reserved[0] = tcmin;
    c.push_back(o);
  };
  add(QS_MODE_PER_GATE, 0, 0, 0, 0);
  const int ks[] = {1, 2, 3, 4};
  for (int k : ks) {
    if (dt == QS_C64) {
      add(QS_MODE_FUSED, k, 12, 4, 0);
      add(QS_MODE_FUSED, k, 13, 4, 0);
    } else {
      add(QS_MODE_FUSED, k, 11, 3, 0);
      add(QS_MODE_FUSED, k, 12, 4, 0);
    }
  }
  if (dt == QS_C64 && n >= 13) {
    const int tm[] = {2, 4, 8};
    for (int t : tm) add(QS_MODE_TENSOR, 2, 13, 4, t);
  }
  return c;
}

// ---------------------------------------------------------------- host-resident states (Section 3.2)

// Streamed passes: the tile-pass scheduler with the l low qubits always in the
// "tile" and at most h batch-index qubits (>= l) beside them; gates move ahead
// of the gates they commute with, so a pass gathers every gate that fits.
// Each pass moves the state once through the host link in each direction.
std::vector<StreamPass> plan_stream_passes(int n, const std::vector<HGate>& gates, int l, int h) {
  std::vector<OpRec> ops;
  for (size_t g = 0; g < gates.size(); ++g) {
    if (__builtin_popcountll(gates[g].qmask >> l) > h)
      throw Error(QS_ERR_ARG, "gate " + std::to_string(g) + " touches more batch qubits than pass_qubits");
    ops.push_back(OpRec{OP_GATE, (int)g, -1, gates[g].qmask, gates[g].dmask});
  }
  std::vector<int> order;
  const std::vector<PassRec> pr = schedule_passes(n, ops, l + h, l, order);
  std::vector<StreamPass> out;
  for (const PassRec& r : pr) {
    StreamPass sp;
    for (int i = r.op_begin; i < r.op_end; ++i) {
      sp.gates.push_back(ops[order[i]].gate);
      sp.high_mask |= gates[ops[order[i]].gate].qmask & ~((1ull << l) - 1);
    }
    out.push_back(std::move(sp));
  }
  return out;
}

// =================================================================== C ABI

extern "C" {

const char* qs_last_error(void) { return g_err.c_str(); }

qs_status qs_plan_set_timing(qs_plan_t p, int enable) {
  return guard([&] {
    require(p != nullptr, "plan is NULL");
    p->timing = enable != 0;
    p->events_used = 0;
    p->event_kind.clear();
  });
}

qs_status qs_plan_timing_read(qs_plan_t p, double* total_ms, int64_t* launches) {
  return qs_plan_timing_read_kinds(p, total_ms, launches, nullptr, nullptr);
}

qs_status qs_plan_timing_read_kinds(qs_plan_t p, double* total_ms, int64_t* launches, double* kind_ms,
                                    int64_t* kind_launches) {
  return guard([&] {
    require(p != nullptr, "plan is NULL");
    double t = 0, km[2] = {0, 0};
    int64_t kn[2] = {0, 0};
    for (size_t i = 0; i + 1 < p->events_used; i += 2) {
      CK(cudaEventSynchronize(p->events[i + 1]));
      float ms = 0;
      CK(cudaEventElapsedTime(&ms, p->events[i], p->events[i + 1]));
      t += ms;
      const int k = p->event_kind[i / 2];
      km[k] += ms;
      kn[k] += 1;
    }
    if (total_ms) *total_ms = t;
    if (launches) *launches = (int64_t)(p->events_used / 2);
    if (kind_ms) { kind_ms[0] = km[0]; kind_ms[1] = km[1]; }
    if (kind_launches) { kind_launches[0] = kn[0]; kind_launches[1] = kn[1]; }
    p->events_used = 0;
    p->event_kind.clear();
  });
}

qs_status qs_plan_check_device_blocks(qs_plan_t p, qs_state_t s, const double* theta, size_t ntheta,
                                      double* max_abs_diff, int64_t* nblocks) {
  return guard([&] {
    require(p != nullptr, "plan is NULL");
    check_state(s);
    require(p->n == s->n && p->dt == s->dt, "plan and state differ");
    upload(*p);
    resolve_theta(*p, theta, ntheta, 1, s->st);
    build_device_blocks(*p, 1, s->st);
    std::vector<double2> dev(std::max<int64_t>(1, p->btab_elems));
    CK(cudaMemcpyAsync(dev.data(), p->d_btab.p, sizeof(double2) * dev.size(), cudaMemcpyDeviceToHost, s->st));
    std::vector<uint16_t> wdev(p->h_wimg.size());
    if (!wdev.empty())
      CK(cudaMemcpyAsync(wdev.data(), p->d_wimg.p, sizeof(uint16_t) * wdev.size(), cudaMemcpyDeviceToHost, s->st));
    CK(cudaStreamSynchronize(s->st));
    std::vector<double2> saved = p->h_btab;
    compute_blocks(*p, theta, true);   // host FP64 products for the parametric blocks
    double worst = 0;
    int64_t cnt = 0;
    for (size_t b = 0; b < p->blocks.size(); ++b) {
      const Block& blk = p->blocks[b];
      if (!blk.parametric || p->block_off[b] < 0) continue;
      const int64_t D = 1ll << blk.qubits.size();
      const int64_t m = blk.rep == OP_DIAG ? D : D * D;
      for (int64_t i = 0; i < m; ++i) {
        const double2 a = dev[p->block_off[b] + i], h = p->h_btab[p->block_off[b] + i];
        if (blk.rep != OP_TC) worst = std::max(worst, std::hypot(a.x - h.x, a.y - h.y));
      }
      if (blk.rep == OP_TC) {
        // compare the W image with one built on the host from the host product: the
        // value the MMAs use is hi + lo (hi and lo alone may trade one ulp at a tie)
        std::vector<uint16_t> img(32768);
        build_w_image(p->h_btab.data() + p->block_off[b], img.data(), p->tc_prec == 4);
        for (size_t st = 0; st < p->steps.size(); ++st)
          if (p->steps[st].kind == 1 && p->exec_ops[p->pass_ops[st].first].block == (int)b) {
            const uint16_t* dv = wdev.data() + (size_t)p->steps[st].idx * 32768;
            for (int e = 0; e < 16384; ++e) {
              const bool hf = p->tc_prec == 4;
              const double wh = (double)w_to_float(img[e], hf) + (double)w_to_float(img[16384 + e], hf);
              const double wd = (double)w_to_float(dv[e], hf) + (double)w_to_float(dv[16384 + e], hf);
              worst = std::max(worst, std::fabs(wh - wd));
            }
          }
      }
      ++cnt;
    }
    p->h_btab = saved;
    if (max_abs_diff) *max_abs_diff = worst;
    if (nblocks) *nblocks = cnt;
  });
}

qs_status qs_plan_op_count(qs_plan_t p, int64_t* nops, int64_t* npasses) {
  return guard([&] {
    require(p != nullptr, "plan is NULL");
    const bool pg = p->mode == QS_MODE_PER_GATE;
    if (nops) *nops = pg ? (int64_t)p->gates.size() : (int64_t)p->exec_ops.size();
    if (npasses) *npasses = pg ? (int64_t)p->gates.size() : (int64_t)p->steps.size();
  });
}

qs_status qs_plan_op_get(qs_plan_t p, int64_t i, int32_t* type, int32_t* qubits, int32_t* nq, int32_t* gate_index,
                         double* mat) {
  return guard([&] {
    require(p != nullptr, "plan is NULL");
    const bool pg = p->mode == QS_MODE_PER_GATE;
    const int64_t N = pg ? (int64_t)p->gates.size() : (int64_t)p->exec_ops.size();
    require(i >= 0 && i < N, "op index out of range");
    OpRec r = pg ? OpRec{OP_GATE, (int)i, -1, p->gates[i].qmask, p->gates[i].dmask} : p->exec_ops[i];
    if (type) *type = r.type;
    int k = 0;
    for (int b = 0; b < 64; ++b)
      if (r.qmask & (1ull << b)) {
        if (qubits) qubits[k] = b;
        ++k;
      }
    if (nq) *nq = k;
    if (gate_index) *gate_index = r.gate;
    if (mat && r.type != OP_GATE && r.type != OP_PHASE) {
      const int64_t off = p->block_off[r.block];
      const int64_t D = 1ll << k;
      const int64_t cnt = r.type == OP_DIAG ? D : D * D;
      for (int64_t j = 0; j < cnt; ++j) {
        mat[2 * j] = p->h_btab[off + j].x;
        mat[2 * j + 1] = p->h_btab[off + j].y;
      }
    }
  });
}

qs_status qs_plan_phase_terms(qs_plan_t p, int64_t i, uint64_t* masks, int32_t* param_index, double* alpha0,
                              double* coef, int64_t cap, int64_t* nterms) {
  return guard([&] {
    require(p != nullptr, "plan is NULL");
    require(p->mode != QS_MODE_PER_GATE && i >= 0 && i < (int64_t)p->exec_ops.size(), "op index out of range");
    const OpRec& r = p->exec_ops[i];
    require(r.type == OP_PHASE, "op is not a phase pass");
    int64_t step = -1;
    for (size_t s = 0; s < p->steps.size(); ++s)
      if (p->steps[s].kind == 2 && p->pass_ops[s].first == i) step = (int64_t)s;
    require(step >= 0, "internal: phase op without a pass");
    const PhasePassDesc& d = p->phdesc[p->steps[step].idx];
    if (nterms) *nterms = d.nterms;
    for (int64_t j = 0; j < d.nterms && j < cap; ++j) {
      const DevPhaseTerm& t = p->h_pterms[d.term_off + j];
      if (masks) masks[j] = t.mask;
      if (param_index) param_index[j] = t.pidx;
      if (alpha0) alpha0[j] = t.alpha0;
      if (coef) coef[j] = t.coef;
    }
  });
}

qs_status qs_plan_pass_get(qs_plan_t p, int64_t i, int32_t* tile_qubits, int32_t* m, int64_t* op_begin,
                           int64_t* op_end) {
  return guard([&] {
    require(p != nullptr, "plan is NULL");
    if (p->mode == QS_MODE_PER_GATE) {
      require(i >= 0 && i < (int64_t)p->gates.size(), "pass index out of range");
      if (m) *m = 0;
      if (op_begin) *op_begin = i;
      if (op_end) *op_end = i + 1;
      return;
    }
    require(i >= 0 && i < (int64_t)p->steps.size(), "pass index out of range");
    const auto& t = p->pass_tiles[i];
    if (tile_qubits)
      for (size_t j = 0; j < t.size(); ++j) tile_qubits[j] = t[j];
    if (m) *m = (int32_t)t.size();
    if (op_begin) *op_begin = p->pass_ops[i].first;
    if (op_end) *op_end = p->pass_ops[i].second;
  });
}
int64_t qs_launch_count(void) { return qs::launch_count(); }
const char* qs_version(void) { return "gb300-statevec 0.1 (sm_103a)"; }

qs_status qs_state_alloc(int n, qs_dtype dtype, void* stream, qs_state_t* out) {
  return guard([&] {
    require(out != nullptr, "out is NULL");
    require(n >= 1 && n <= kMaxQubits, "n out of range (1..40)");
    require(dtype == QS_C64 || dtype == QS_C128, "bad dtype");
    require_device();
    auto s = std::make_unique<qs_state_s>();
    s->n = n;
    s->dt = dtype;
    s->st = (cudaStream_t)stream;
    cudaError_t e = cudaMalloc(&s->d, s->bytes());
    if (e != cudaSuccess) {
      cudaGetLastError();
      throw Error(QS_ERR_OOM, "cannot allocate " + std::to_string(s->bytes()) + " bytes for the state");
    }
    s->owned = true;
    CK(launch_set_basis(s->d, n, dtype, 0, s->st));
    *out = s.release();
  });
}

qs_status qs_state_wrap(void* dev_ptr, int n, qs_dtype dtype, void* stream, qs_state_t* out) {
  return guard([&] {
    require(out != nullptr && dev_ptr != nullptr, "NULL argument");
    require(((uintptr_t)dev_ptr & 15) == 0, "device pointer must be 16-byte aligned");
    require(n >= 1 && n <= kMaxQubits, "n out of range (1..40)");
    require(dtype == QS_C64 || dtype == QS_C128, "bad dtype");
    require_device();
    auto s = std::make_unique<qs_state_s>();
    s->n = n;
    s->dt = dtype;
    s->st = (cudaStream_t)stream;
    s->d = dev_ptr;
    s->owned = false;
    *out = s.release();
  });
}

qs_status qs_state_free(qs_state_t s) {
  return guard([&] {
    if (!s) return;
    if (s->owned && s->d) cudaFree(s->d);
    delete s;
  });
}

qs_status qs_state_info(qs_state_t s, int* n, qs_dtype* dtype, void** dev_ptr) {
  return guard([&] {
    check_state(s);
    if (n) *n = s->n;
    if (dtype) *dtype = s->dt;
    if (dev_ptr) *dev_ptr = s->d;
  });
}

qs_status qs_state_set_stream(qs_state_t s, void* stream) {
  return guard([&] {
    check_state(s);
    s->st = (cudaStream_t)stream;
  });
}

qs_status qs_state_set_basis(qs_state_t s, uint64_t x) {
  return guard([&] {
    check_state(s);
    require(x < (1ull << s->n), "basis index >= 2^n");
    CK(launch_set_basis(s->d, s->n, s->dt, x, s->st));
  });
}

qs_status qs_state_copy_from_host(qs_state_t s, const void* host, size_t bytes) {
  return guard([&] {
    check_state(s);
    require(host != nullptr, "host is NULL");
    require(bytes == s->bytes(), "byte count must equal 2^n * amplitude size");
    CK(cudaMemcpyAsync(s->d, host, bytes, cudaMemcpyHostToDevice, s->st));
    CK(cudaStreamSynchronize(s->st));
  });
}

qs_status qs_state_copy_to_host(qs_state_t s, void* host, size_t bytes) {
  return guard([&] {
    check_state(s);
    require(host != nullptr, "host is NULL");
    require(bytes == s->bytes(), "byte count must equal 2^n * amplitude size");
    CK(cudaMemcpyAsync(host, s->d, bytes, cudaMemcpyDeviceToHost, s->st));
    CK(cudaStreamSynchronize(s->st));
  });
}

qs_status qs_state_get_amplitudes(qs_state_t s, const uint64_t* idx, size_t count, void* out) {
  return guard([&] {
    check_state(s);
    if (count == 0) return;
    require(idx != nullptr && out != nullptr, "NULL argument");
    const uint64_t dim = 1ull << s->n;
    for (size_t k = 0; k < count; ++k) require(idx[k] < dim, "amplitude index >= 2^n");
    const size_t ab = amp_bytes(s->dt);
    DevBuf didx, dout;
    didx.ensure(sizeof(uint64_t) * count);
    dout.ensure(ab * count);
    CK(cudaMemcpyAsync(didx.p, idx, sizeof(uint64_t) * count, cudaMemcpyHostToDevice, s->st));
    CK(launch_gather(s->d, s->dt, didx.as<uint64_t>(), count, dout.p, s->st));
    CK(cudaMemcpyAsync(out, dout.p, ab * count, cudaMemcpyDeviceToHost, s->st));
    CK(cudaStreamSynchronize(s->st));
  });
}

qs_status qs_state_copy(qs_state_t dst, qs_state_t src) {
  return guard([&] {
    check_state(dst);
    check_state(src);
    require(dst->n == src->n && dst->dt == src->dt, "states differ in n or dtype");
    CK(cudaMemcpyAsync(dst->d, src->d, src->bytes(), cudaMemcpyDeviceToDevice, dst->st));
  });
}

qs_status qs_plan_create(int n, qs_dtype dtype, const qs_gate* gates, size_t ngates, const qs_plan_opts* opts,
                         qs_plan_t* out) {
  return guard([&] {
    require(out != nullptr, "out is NULL");
    *out = create_plan(n, dtype, gates, ngates, opts);
  });
}

qs_status qs_plan_info_get(qs_plan_t p, qs_plan_info* info) {
  return guard([&] {
    require(p && info, "NULL argument");
    *info = p->info;
  });
}

qs_status qs_plan_free(qs_plan_t p) {
  return guard([&] { delete p; });
}

qs_status qs_plan_autotune(qs_state_t s, const qs_gate* gates, size_t ngates, const double* theta, size_t ntheta,
                           qs_plan_opts* best, double* best_ms) {
  return guard([&] {
    check_state(s);
    require(best != nullptr, "best is NULL");
    require(ngates == 0 || gates != nullptr, "gates is NULL");
    std::vector<uint64_t> key{(uint64_t)s->n, (uint64_t)s->dt, (uint64_t)ngates,
                              fnv1a(gates, sizeof(qs_gate) * ngates)};
    {
      std::lock_guard<std::mutex> lock(g_tune_mu);
      auto it = g_tune_cache.find(key);
      if (it != g_tune_cache.end()) {
        *best = it->second.opts;
        if (best_ms) *best_ms = it->second.ms;
        return;
      }
    }
    cudaEvent_t e0, e1;
    CK(cudaEventCreate(&e0));
    CK(cudaEventCreate(&e1));
    bool have = false;
    TuneEntry top{};
    try {
      for (const qs_plan_opts& o : tune_candidates(s->n, s->dt)) {
        std::unique_ptr<qs_plan_s> p;
        try {
          p.reset(create_plan(s->n, s->dt, gates, ngates, &o));
        } catch (const Error& e) {
          if (e.code == QS_ERR_ARG || e.code == QS_ERR_UNSUPPORTED) continue;   // option not valid here
          throw;
        }
        execute(*p, *s, theta, ntheta);            // warm-up (uploads, attributes)
        CK(cudaEventRecord(e0, s->st));
        execute(*p, *s, theta, ntheta);
        CK(cudaEventRecord(e1, s->st));
        CK(cudaEventSynchronize(e1));
        float ms = 0;
        CK(cudaEventElapsedTime(&ms, e0, e1));
        if (!have || ms < top.ms) {
          top.opts = o;
          top.ms = ms;
          have = true;
        }
      }
    } catch (...) {
      cudaEventDestroy(e0);
      cudaEventDestroy(e1);
      throw;
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    require(have, "no candidate plan is valid for this circuit");
    {
      std::lock_guard<std::mutex> lock(g_tune_mu);
      g_tune_cache[key] = top;
    }
    *best = top.opts;
    if (best_ms) *best_ms = top.ms;
  });
}

qs_status qs_plan_execute(qs_plan_t p, qs_state_t s, const double* theta, size_t ntheta) {
  return guard([&] {
    require(p != nullptr, "plan is NULL");
    check_state(s);
    execute(*p, *s, theta, ntheta);
  });
}

qs_status qs_plan_execute_host(qs_plan_t p, qs_state_t* work, int nwork, const void* const* host_in,
                               void* const* host_out, int count, const double* theta, size_t ntheta,
                               double* norms) {
  return guard([&] {
    require(p != nullptr && work != nullptr && nwork >= 1 && count >= 0, "bad arguments");
    require(count == 0 || host_in != nullptr, "host_in is NULL");
    for (int b = 0; b < nwork; ++b) {
      check_state(work[b]);
      require(work[b]->n == p->n && work[b]->dt == p->dt, "work state and plan differ in qubit count or dtype");
      for (int c = 0; c < b; ++c) require(work[c] != work[b], "work states must be distinct");
    }
    for (int i = 0; i < count; ++i) require(host_in[i] != nullptr, "host_in has a NULL entry");
    const size_t bytes = amp_bytes(p->dt) << p->n;
    upload(*p);
    cudaStream_t si = nullptr, sc = nullptr, so = nullptr;
    std::vector<cudaEvent_t> loaded(nwork, nullptr), computed(nwork, nullptr), stored(nwork, nullptr);
    auto cleanup = [&]() {
      for (int b = 0; b < nwork; ++b) {
        if (loaded[b]) cudaEventDestroy(loaded[b]);
        if (computed[b]) cudaEventDestroy(computed[b]);
        if (stored[b]) cudaEventDestroy(stored[b]);
      }
      if (si) cudaStreamDestroy(si);
      if (sc) cudaStreamDestroy(sc);
      if (so) cudaStreamDestroy(so);
    };
    try {
      CK(cudaStreamCreateWithFlags(&si, cudaStreamNonBlocking));
      CK(cudaStreamCreateWithFlags(&sc, cudaStreamNonBlocking));
      CK(cudaStreamCreateWithFlags(&so, cudaStreamNonBlocking));
      for (int b = 0; b < nwork; ++b) {
        CK(cudaEventCreateWithFlags(&loaded[b], cudaEventDisableTiming));
        CK(cudaEventCreateWithFlags(&computed[b], cudaEventDisableTiming));
        CK(cudaEventCreateWithFlags(&stored[b], cudaEventDisableTiming));
        // earlier work queued on the work states' own streams comes first
        CK(cudaEventRecord(stored[b], work[b]->st));
        work[b]->scratch.ensure(partial_bytes(1) + sizeof(double));
      }
      resolve_theta(*p, theta, ntheta, 1, sc);
      build_device_blocks(*p, 1, sc);
      for (int i = 0; i < count; ++i) {
        const int b = i % nwork;
        qs_state_s& w = *work[b];
        CK(cudaStreamWaitEvent(si, stored[b], 0));
        CK(cudaMemcpyAsync(w.d, host_in[i], bytes, cudaMemcpyHostToDevice, si));
        CK(cudaEventRecord(loaded[b], si));
        CK(cudaStreamWaitEvent(sc, loaded[b], 0));
        issue_circuit(*p, w.d, 0, sc);
        double* d_part = w.scratch.as<double>();
        if (norms) CK(launch_norm(w.d, w.n, w.dt, d_part, d_part + reduce_blocks(), sc));
        CK(cudaEventRecord(computed[b], sc));
        CK(cudaStreamWaitEvent(so, computed[b], 0));
        if (host_out && host_out[i]) CK(cudaMemcpyAsync(host_out[i], w.d, bytes, cudaMemcpyDeviceToHost, so));
        if (norms) CK(cudaMemcpyAsync(&norms[i], d_part + reduce_blocks(), sizeof(double), cudaMemcpyDeviceToHost, so));
        CK(cudaEventRecord(stored[b], so));
      }
      CK(cudaStreamSynchronize(so));
      CK(cudaStreamSynchronize(sc));
      CK(cudaStreamSynchronize(si));
      for (int b = 0; b < nwork; ++b) CK(cudaStreamWaitEvent(work[b]->st, stored[b], 0));
      if (!p->tcdesc.empty()) {
        int err = 0;
        CK(cudaMemcpy(&err, p->d_err.p, sizeof(int), cudaMemcpyDeviceToHost));
        if (err) throw Error(QS_ERR_TIMEOUT, "tensor-core pass: an MMA completion wait timed out");
      }
    } catch (...) {
      if (si) cudaStreamSynchronize(si);
      if (sc) cudaStreamSynchronize(sc);
      if (so) cudaStreamSynchronize(so);
      cleanup();
      throw;
    }
    cleanup();
  });
}

qs_status qs_apply_circuit(qs_state_t s, const qs_gate* gates, size_t ngates, const double* theta, size_t ntheta,
                           const qs_plan_opts* opts) {
  return guard([&] {
    check_state(s);
    std::unique_ptr<qs_plan_s> p(create_plan(s->n, s->dt, gates, ngates, opts));
    execute(*p, *s, theta, ntheta);
    CK(cudaStreamSynchronize(s->st));   // the plan's device tables are freed on return
  });
}

qs_status qs_stream_plan(int n, const qs_gate* gates, size_t ngates, int batch_qubits, int pass_qubits,
                         int64_t* npasses, uint64_t* high_masks, int64_t* pass_end, int64_t cap, int32_t* order) {
  return guard([&] {
    require(n >= 1 && n <= kMaxQubits, "n out of range");
    require(batch_qubits >= 1 && batch_qubits <= n && pass_qubits >= 0 && pass_qubits <= n - batch_qubits,
            "batch_qubits / pass_qubits out of range");
    std::vector<HGate> hg;
    resolve_gates(n, gates, ngates, hg);
    const std::vector<StreamPass> ps = plan_stream_passes(n, hg, batch_qubits, pass_qubits);
    if (npasses) *npasses = (int64_t)ps.size();
    int64_t k = 0;
    for (int64_t i = 0; i < (int64_t)ps.size(); ++i) {
      for (int g : ps[i].gates) {
        if (order) order[k] = g;
        ++k;
      }
      if (i < cap) {
        if (high_masks) high_masks[i] = ps[i].high_mask;
        if (pass_end) pass_end[i] = k;
      }
    }
  });
}

qs_status qs_stream_apply(void* host_psi, int n, qs_dtype dt, const qs_gate* gates, size_t ngates, const double* theta,
                          size_t ntheta, const qs_plan_opts* opts, int batch_qubits, int pass_qubits,
                          qs_stream_info* info) {
  return guard([&] {
    require(host_psi != nullptr, "host_psi is NULL");
    require(dt == QS_C64 || dt == QS_C128, "bad dtype");
    require(n >= 1 && n <= kMaxQubits, "n out of range");
    const int l = batch_qubits, h = pass_qubits;
    require(l >= 1 && l <= n && h >= 0 && h <= n - l && l + h <= kMaxQubits, "batch_qubits / pass_qubits out of range");
    std::vector<HGate> hg;
    resolve_gates(n, gates, ngates, hg);
    const std::vector<StreamPass> passes = plan_stream_passes(n, hg, l, h);
    const size_t ab = amp_bytes(dt);
    const size_t batch_bytes = ab << l;
    // one sub-plan per pass over l + |high| qubits: bit j < l stays, high qubit k of the pass -> bit l + k
    std::vector<std::unique_ptr<qs_plan_s>> plans;
    std::vector<std::vector<int>> highs;
    int hmax = 0;
    for (const StreamPass& sp : passes) {
      std::vector<int> hi;
      for (int q = l; q < n; ++q)
        if (sp.high_mask & (1ull << q)) hi.push_back(q);
      auto local = [&](int q) {
        if (q < l) return q;
        return l + (int)(std::find(hi.begin(), hi.end(), q) - hi.begin());
      };
      std::vector<qs_gate> sub;
      for (int g : sp.gates) {
        qs_gate x = gates[g];
        for (int k = 0; k < x.nq; ++k) x.q[k] = local(x.q[k]);
        for (int k = 0; k < x.nctrl; ++k) x.ctrl[k] = local(x.ctrl[k]);
        sub.push_back(x);
      }
      plans.emplace_back(create_plan(l + (int)hi.size(), dt, sub.data(), sub.size(), opts));
      hmax = std::max(hmax, (int)hi.size());
      highs.push_back(hi);
    }
    // three device buffers of 2^(l + hmax) amplitudes; H2D, compute and D2H streams
    DevBuf buf[3];
    for (auto& b : buf) b.ensure(batch_bytes << hmax);
    cudaStream_t sh = nullptr, sc = nullptr, sd = nullptr;
    cudaEvent_t loaded[3] = {}, computed[3] = {}, stored[3] = {}, pass_done = nullptr;
    auto cleanup = [&]() {
      for (int k = 0; k < 3; ++k) {
        if (loaded[k]) cudaEventDestroy(loaded[k]);
        if (computed[k]) cudaEventDestroy(computed[k]);
        if (stored[k]) cudaEventDestroy(stored[k]);
      }
      if (pass_done) cudaEventDestroy(pass_done);
      if (sh) cudaStreamDestroy(sh);
      if (sc) cudaStreamDestroy(sc);
      if (sd) cudaStreamDestroy(sd);
    };
    try {
      CK(cudaStreamCreateWithFlags(&sh, cudaStreamNonBlocking));
      CK(cudaStreamCreateWithFlags(&sc, cudaStreamNonBlocking));
      CK(cudaStreamCreateWithFlags(&sd, cudaStreamNonBlocking));
      for (int k = 0; k < 3; ++k) {
        CK(cudaEventCreateWithFlags(&loaded[k], cudaEventDisableTiming));
        CK(cudaEventCreateWithFlags(&computed[k], cudaEventDisableTiming));
        CK(cudaEventCreateWithFlags(&stored[k], cudaEventDisableTiming));
      }
      CK(cudaEventCreateWithFlags(&pass_done, cudaEventDisableTiming));
      int64_t copies = 0, groups_total = 0;
      for (size_t pi = 0; pi < passes.size(); ++pi) {
        qs_plan_s& p = *plans[pi];
        upload(p);
        resolve_theta(p, theta, ntheta, 1, sc);
        build_device_blocks(p, 1, sc);
        const std::vector<int>& hi = highs[pi];
        const int hh = (int)hi.size();
        std::vector<int> rest;   // batch-index bits (relative to l) the pass does not select
        for (int q = l; q < n; ++q)
          if (std::find(hi.begin(), hi.end(), q) == hi.end()) rest.push_back(q - l);
        const uint64_t ngroups = 1ull << rest.size();
        if (pi > 0) CK(cudaStreamWaitEvent(sh, pass_done, 0));   // the previous pass's results are in host memory
        for (uint64_t gi = 0; gi < ngroups; ++gi) {
          const int k = (int)(gi % 3);
          uint64_t base = 0;
          for (size_t b = 0; b < rest.size(); ++b) base |= ((gi >> b) & 1ull) << rest[b];
          if (gi >= 3 || pi > 0) CK(cudaStreamWaitEvent(sh, stored[k], 0));
          for (uint64_t j = 0; j < (1ull << hh); ++j) {
            uint64_t bi = base;
            for (int b = 0; b < hh; ++b) bi |= ((j >> b) & 1ull) << (hi[b] - l);
            CK(cudaMemcpyAsync((char*)buf[k].p + j * batch_bytes, (const char*)host_psi + bi * batch_bytes, batch_bytes,
                               cudaMemcpyHostToDevice, sh));
          }
          CK(cudaEventRecord(loaded[k], sh));
          CK(cudaStreamWaitEvent(sc, loaded[k], 0));
          issue_circuit(p, buf[k].p, 0, sc);
          CK(cudaEventRecord(computed[k], sc));
          CK(cudaStreamWaitEvent(sd, computed[k], 0));
          for (uint64_t j = 0; j < (1ull << hh); ++j) {
            uint64_t bi = base;
            for (int b = 0; b < hh; ++b) bi |= ((j >> b) & 1ull) << (hi[b] - l);
            CK(cudaMemcpyAsync((char*)host_psi + bi * batch_bytes, (const char*)buf[k].p + j * batch_bytes, batch_bytes,
                               cudaMemcpyDeviceToHost, sd));
          }
          CK(cudaEventRecord(stored[k], sd));
          copies += 2ll << hh;
        }
        groups_total += (int64_t)ngroups;
        CK(cudaEventRecord(pass_done, sd));
      }
      CK(cudaStreamSynchronize(sd));
      CK(cudaStreamSynchronize(sc));
      for (auto& pp : plans)
        if (!pp->tcdesc.empty()) {
          int err = 0;
          CK(cudaMemcpy(&err, pp->d_err.p, sizeof(int), cudaMemcpyDeviceToHost));
          if (err) throw Error(QS_ERR_TIMEOUT, "tensor-core pass: an MMA completion wait timed out");
        }
      if (info) {
        std::memset(info, 0, sizeof(*info));
        info->passes = (int64_t)passes.size();
        info->groups = groups_total;
        info->copies = copies;
        info->bytes_h2d = (double)passes.size() * (double)(ab << n);
        info->bytes_d2h = info->bytes_h2d;
        info->device_bytes = 3.0 * (double)(batch_bytes << hmax);
      }
    } catch (...) {
      cudaStreamSynchronize(sh);
      cudaStreamSynchronize(sc);
      cudaStreamSynchronize(sd);
      cleanup();
      throw;
    }
    cleanup();
  });
}

qs_status qs_norm(qs_state_t s, double* out) {
  return guard([&] {
    check_state(s);
    require(out != nullptr, "out is NULL");
    s->scratch.ensure(partial_bytes(1) + sizeof(double));
    double* d_part = s->scratch.as<double>();
    double* d_out = d_part + reduce_blocks();
    CK(launch_norm(s->d, s->n, s->dt, d_part, d_out, s->st));
    double v = 0;
    CK(cudaMemcpyAsync(&v, d_out, sizeof(double), cudaMemcpyDeviceToHost, s->st));
    CK(cudaStreamSynchronize(s->st));
    *out = v;
  });
}

qs_status qs_inner(qs_state_t a, qs_state_t b, double* re, double* im) {
  return guard([&] {
    check_state(a);
    check_state(b);
    require(a->n == b->n && a->dt == b->dt, "states differ in n or dtype");
    a->scratch.ensure(partial_bytes(2) + 2 * sizeof(double));
    double* d_part = a->scratch.as<double>();
    double* d_out = d_part + 2 * reduce_blocks();
    CK(launch_inner(a->d, b->d, a->n, a->dt, d_part, d_out, a->st));
    double v[2];
    CK(cudaMemcpyAsync(v, d_out, sizeof(v), cudaMemcpyDeviceToHost, a->st));
    CK(cudaStreamSynchronize(a->st));
    if (re) *re = v[0];
    if (im) *im = v[1];
  });
}

qs_status qs_state_diff(qs_state_t a, qs_state_t b, double* max_abs, double* l2) {
  return guard([&] {
    check_state(a);
    check_state(b);
    require(a->n == b->n, "states differ in n");
    const int RB = reduce_blocks();
    a->scratch.ensure(partial_bytes(2));
    CK(cudaStreamSynchronize(b->st));
    CK(launch_diff(a->d, a->dt, b->d, b->dt, a->n, a->scratch.as<double>(), a->st));
    std::vector<double> h(2 * (size_t)RB);
    CK(cudaMemcpyAsync(h.data(), a->scratch.p, sizeof(double) * h.size(), cudaMemcpyDeviceToHost, a->st));
    CK(cudaStreamSynchronize(a->st));
    double m = 0, s2 = 0;
    for (int i = 0; i < RB; ++i) {
      m = std::max(m, h[i]);
      s2 += h[RB + i];
    }
    if (max_abs) *max_abs = m;
    if (l2) *l2 = std::sqrt(s2);
  });
}

qs_status qs_expval_pauli_sum(qs_state_t s, const qs_pauli_term* terms, size_t nterms, double* out) {
  return guard([&] {
    check_state(s);
    require(out != nullptr, "out is NULL");
    *out = expval_sync(*s, terms, nterms);
  });
}

qs_status qs_apply_pauli_sum(qs_state_t s, const qs_pauli_term* terms, size_t nterms, qs_state_t out) {
  return guard([&] {
    check_state(s);
    check_state(out);
    require(s != out && s->d != out->d, "output must not alias the input");
    require(s->n == out->n && s->dt == out->dt, "states differ in n or dtype");
    require(nterms == 0 || terms != nullptr, "terms is NULL");
    group_terms(s->n, terms, nterms);   // validation
    uint64_t *dx, *dz;
    double2* dph;
    std::vector<unsigned char> host;
    upload_pauli_apply(terms, nterms, s->scratch2, s->st, &dx, &dz, &dph, host);
    CK(launch_apply_pauli(s->d, out->d, s->n, s->dt, dx, dz, (const double*)dph, (int)nterms, s->st));
    CK(cudaStreamSynchronize(s->st));
  });
}

qs_status qs_adjoint_grad(qs_state_t s, const qs_gate* gates, size_t ngates, const double* theta, size_t ntheta,
                          const qs_pauli_term* terms, size_t nterms, double* expval_out, double* grad_out) {
  return qs_adjoint_grad_opts(s, gates, ngates, theta, ntheta, terms, nterms, nullptr, expval_out, grad_out);
}

qs_status qs_adjoint_grad_opts(qs_state_t s, const qs_gate* gates, size_t ngates, const double* theta, size_t ntheta,
                               const qs_pauli_term* terms, size_t nterms, const qs_plan_opts* opts,
                               double* expval_out, double* grad_out) {
  return guard([&] {
    check_state(s);
    require(grad_out != nullptr || ntheta == 0, "grad_out is NULL");
    require(nterms == 0 || terms != nullptr, "terms is NULL");
    require(opts == nullptr || opts->mode != QS_MODE_PER_GATE, "the forward plan of the adjoint needs a fused or tensor mode");
    // forward: phi = U psi with a fused plan (tile passes, CUDA cores), or the caller's options
    qs_plan_opts fo;
    std::memset(&fo, 0, sizeof(fo));
    fo.mode = QS_MODE_FUSED;
    if (opts) fo = *opts;
    std::unique_ptr<qs_plan_s> p(create_plan(s->n, s->dt, gates, ngates, &fo));
    // reverse sweep: the reversed circuit, one op per gate, grouped into tile passes
    std::vector<qs_gate> rev(gates, gates + ngates);
    std::reverse(rev.begin(), rev.end());
    qs_plan_opts ro;
    std::memset(&ro, 0, sizeof(ro));
    ro.mode = QS_MODE_FUSED;
    ro.fuse_k = 1;
    ro.reserved[3] = opts ? opts->reserved[3] : 0;   // complex128 arithmetic of the reverse sweep
    std::unique_ptr<qs_plan_s> rp(create_plan(s->n, s->dt, rev.data(), rev.size(), &ro, /*no_merge=*/true));
    upload(*p);
    upload(*rp);
    const size_t bytes = s->bytes();
    DevBuf phi, lam, part, aux, gadj, grow_d;
    phi.ensure(bytes);
    lam.ensure(bytes);
    CK(cudaMemcpyAsync(phi.p, s->d, bytes, cudaMemcpyDeviceToDevice, s->st));
    qs_state_s sphi;   // borrowed view (not owning)
    sphi.n = s->n; sphi.dt = s->dt; sphi.d = phi.p; sphi.st = s->st;
    execute(*p, sphi, theta, ntheta);
    // lam = H phi
    group_terms(s->n, terms, nterms);
    uint64_t *dx, *dz;
    double2* dph;
    std::vector<unsigned char> host;
    upload_pauli_apply(terms, nterms, aux, s->st, &dx, &dz, &dph, host);
    CK(launch_apply_pauli(phi.p, lam.p, s->n, s->dt, dx, dz, (const double*)dph, (int)nterms, s->st));
    // rows: one per parametric gate of the reversed circuit, plus 2 for <phi|lam>
    const int G = (int)rp->gates.size();
    std::vector<int32_t> grow(std::max(1, G), -1);
    std::vector<int> row_gate;
    for (int j = 0; j < G; ++j)
      if (rp->gates[j].parametric) {
        grow[j] = (int32_t)row_gate.size();
        row_gate.push_back(j);
      }
    const int rows = (int)row_gate.size();
    const int RB = reduce_blocks();
    part.ensure(partial_bytes(rows + 2) + sizeof(double) * (rows + 2));
    double* d_part = part.as<double>();
    double* d_sum = d_part + (size_t)RB * (rows + 2);
    CK(cudaMemsetAsync(d_part, 0, partial_bytes(rows), s->st));
    CK(launch_inner(phi.p, lam.p, s->n, s->dt, d_part + (size_t)RB * rows, d_sum + rows, s->st));
    if (G > 0) {
      // G^dagger and dG for every gate of the reversed circuit (theta resolved on the device)
      resolve_theta(*rp, theta, ntheta, 1, s->st);
      gadj.ensure(sizeof(double2) * 16 * (size_t)G);
      CK(launch_adjoint_table(rp->d_gates.as<DevGate>(), G, rp->d_gtab.as<double2>(), gadj.as<double2>(), s->st));
      grow_d.ensure(sizeof(int32_t) * grow.size());
      CK(cudaMemcpyAsync(grow_d.p, grow.data(), sizeof(int32_t) * grow.size(), cudaMemcpyHostToDevice, s->st));
      for (const PassDesc& pd : rp->pdesc) {
        require(adjoint_tile_smem_bytes(pd, s->dt) <= 227 * 1024, "adjoint tile pass does not fit shared memory");
        CK(prepare_adjoint_tile(pd, s->dt));
      }
      for (const auto& stp : rp->steps)
        CK(launch_adjoint_tile(phi.p, lam.p, s->n, s->dt, rp->pdesc[stp.idx], rp->d_ops.as<DevOp>(),
                               gadj.as<double2>(), grow_d.as<int32_t>(), d_part, RB, s->st));
    }
    CK(launch_sum_rows(d_part, rows, RB, d_sum, s->st));
    std::vector<double> sums(rows + 2);
    CK(cudaMemcpyAsync(sums.data(), d_sum, sizeof(double) * (rows + 2), cudaMemcpyDeviceToHost, s->st));
    CK(cudaStreamSynchronize(s->st));
    for (size_t j = 0; j < ntheta; ++j) grad_out[j] = 0;
    for (int r = 0; r < rows; ++r) {
      const HGate& g = rp->gates[row_gate[r]];
      require((size_t)g.param_index < ntheta, "theta shorter than the parameter indices");
      grad_out[g.param_index] += 2.0 * g.scale * sums[r];
    }
    if (expval_out) *expval_out = sums[rows];
  });
}

qs_status qs_plan_execute_batched(qs_plan_t p, qs_state_t* states, int B, const double* theta, size_t ntheta,
                                  const qs_pauli_term* terms, size_t nterms, double* expvals) {
  return guard([&] {
    require(p != nullptr && states != nullptr && B >= 1, "bad arguments");
    for (int b = 0; b < B; ++b) {
      check_state(states[b]);
      require(states[b]->n == p->n && states[b]->dt == p->dt, "plan and state differ in qubit count or dtype");
      require(states[b]->st == states[0]->st, "batched states must share one stream");
    }
    require(terms == nullptr || expvals != nullptr, "expvals is NULL");
    cudaStream_t user_st = states[0]->st;
    if (!p->cap_stream) {
      CK(cudaStreamCreateWithFlags(&p->cap_stream, cudaStreamNonBlocking));
      CK(cudaEventCreateWithFlags(&p->ev_in, cudaEventDisableTiming));
      CK(cudaEventCreateWithFlags(&p->ev_out, cudaEventDisableTiming));
    }
    cudaStream_t st = p->cap_stream;   // capture is not allowed on the legacy default stream
    upload(*p);
    CK(cudaEventRecord(p->ev_in, user_st));
    CK(cudaStreamWaitEvent(st, p->ev_in, 0));
    ensure_gtab_rows(*p, B);
    ensure_block_rows(*p, B);
    // theta upload happens outside the graph; the graph reads p->d_theta
    if (!p->pgates.empty()) {
      require(theta != nullptr && (int64_t)ntheta >= p->nparams, "theta too short");
      p->d_theta.ensure(sizeof(double) * ntheta * B);
      p->theta_stride = (int64_t)ntheta;   // phase passes read row b at b * ntheta (ntheta is in the graph key)
    }
    PreparedTerms P;
    double* d_part = nullptr;
    double* d_out = nullptr;
    const bool one_launch = p->mode != QS_MODE_PER_GATE;   // batched kernels: one launch per pass
    int64_t Z = 0;
    // group table for the batched expectation kernel, after the z list in scratch2:
    // [z: Z u64][x: NL u64][z offset: NL i32][count: NL i32][group order: NL i32,
    // single-string groups first]
    std::vector<unsigned char> gtab_host;
    int NL = 0, NL1 = 0;
    if (terms && nterms) {
      P = prepare_terms(p->n, terms, nterms);
      Z = (int64_t)P.zlist.size();
      NL = (int)P.launches.size();
      qs_state_s& s0 = *states[0];
      const int cols = one_launch ? expval_wave_ctas(expval_wave_states(p->n, p->dt, B)) : reduce_blocks();
      // one launch per wave reuses the partials from offset 0 (each launch reduces
      // its own before the next starts): wave x Z x C(wave) <= Z x reduce_blocks()
      const size_t part = one_launch ? sizeof(double) * (size_t)Z *
                                           std::max<size_t>((size_t)cols * B, (size_t)reduce_blocks())
                                     : sizeof(double) * (size_t)cols * kZPerLaunch;
      s0.scratch.ensure(part + sizeof(double) * P.zlist.size() * B);
      gtab_host.resize(sizeof(uint64_t) * (Z + NL) + sizeof(int32_t) * 3 * NL);
      std::memcpy(gtab_host.data(), P.zlist.data(), sizeof(uint64_t) * Z);
      uint64_t* hx = (uint64_t*)(gtab_host.data() + sizeof(uint64_t) * Z);
      int32_t* hz = (int32_t*)(hx + NL);
      int32_t* hc = hz + NL;
      int32_t* ho = hc + NL;
      for (int l = 0; l < NL; ++l) {
        hx[l] = P.groups[P.launches[l].first].x;
        hz[l] = P.launches[l].second;
        hc[l] = P.counts[l];
        if (hc[l] == 1) ho[NL1++] = l;
      }
      for (int l = 0, r = NL1; l < NL; ++l)
        if (hc[l] != 1) ho[r++] = l;
      s0.scratch2.ensure(gtab_host.size());
      d_part = s0.scratch.as<double>();
      d_out = (double*)((char*)s0.scratch.p + part);
    }
    std::vector<void*> ptrs(B);
    for (int b = 0; b < B; ++b) ptrs[b] = states[b]->d;
    p->d_psis.ensure(sizeof(void*) * B);
    CK(cudaMemcpy(p->d_psis.p, ptrs.data(), sizeof(void*) * B, cudaMemcpyHostToDevice));
    void* const* d_psis = (void* const*)p->d_psis.p;
    std::vector<void*> key = ptrs;
    key.push_back((void*)(uintptr_t)ntheta);
    key.push_back((void*)(uintptr_t)(terms ? nterms : 0));
    key.push_back(p->d_theta.p);
    key.push_back(p->d_psis.p);
    key.push_back(p->d_btab.p);
    key.push_back(p->d_wimg.p);
    key.push_back(p->d_gtab.p);
    key.push_back(states[0]->scratch.p);
    key.push_back(states[0]->scratch2.p);
    if (!p->pgates.empty())
      CK(cudaMemcpyAsync(p->d_theta.p, theta, sizeof(double) * ntheta * B, cudaMemcpyHostToDevice, st));
    if (terms && nterms)
      CK(cudaMemcpyAsync(states[0]->scratch2.p, gtab_host.data(), gtab_host.size(), cudaMemcpyHostToDevice, st));
    // the graph depends on the grouping of the terms (x masks, z order), part of the key
    if (terms && nterms) {
      for (size_t k = 0; k < P.zlist.size(); ++k) key.push_back((void*)(uintptr_t)P.zlist[k]);
      for (auto& L : P.launches) key.push_back((void*)(uintptr_t)P.groups[L.first].x);
    }
    if (!p->graph || p->graph_key != key) {
      if (p->graph) { cudaGraphExecDestroy(p->graph); p->graph = nullptr; }
      cudaGraph_t g = nullptr;
      const int64_t c0 = launch_count();
      CK(cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal));
      try {
        if (!p->pgates.empty()) {
          const size_t G = std::max<size_t>(1, p->gates.size());
          if (p->gtab_rows < B || p->d_theta.bytes < sizeof(double) * ntheta * B)
            throw Error(QS_ERR_CUDA, "internal: gate table or theta smaller than the batch");
          CK(launch_resolve(p->d_gates.as<DevGate>(), p->d_pg.as<int32_t>(), (int)p->pgates.size(),
                            p->d_theta.as<double>(), (int64_t)ntheta, B, p->d_gtab.as<double2>(), (int64_t)16 * G,
                            st));
        }
        build_device_blocks(*p, B, st);
        if (one_launch) {
          // expectation values of each wave right after its passes (the wave is in L2);
          // the partials are reused from offset 0 by every launch
          std::function<void(int, int)> ev;
          if (terms && nterms)
            ev = [&](int w0, int nb) {
              const uint64_t* d_z = states[0]->scratch2.as<uint64_t>();
              const uint64_t* d_gx = d_z + Z;
              const int32_t* d_gz = (const int32_t*)(d_gx + NL);
              CK(launch_expval_groups_batched((const void* const*)(d_psis + w0), nb, p->n, p->dt, d_gx, d_gz, d_gz + NL,
                                              d_gz + 2 * NL, NL1, NL, d_z, (int)Z, d_part, d_out + (size_t)w0 * Z, st));
            };
          issue_circuit_batched(*p, d_psis, B, st, ev);
        } else {
          for (int b = 0; b < B; ++b) {
            issue_circuit(*p, states[b]->d, b, st);
            if (terms && nterms)
              issue_expval(*states[b], P, states[0]->scratch2.as<uint64_t>(), d_part, d_out + (size_t)b * Z, st);
          }
        }
      } catch (...) {
        cudaStreamEndCapture(st, &g);
        if (g) cudaGraphDestroy(g);
        note_launch(-(launch_count() - c0));
        throw;
      }
      CK(cudaStreamEndCapture(st, &g));
      p->graph_launches = launch_count() - c0;   // counted at capture, executed at each replay
      note_launch(-p->graph_launches);
      cudaGraphExec_t ex = nullptr;
      cudaError_t e = cudaGraphInstantiate(&ex, g, 0);
      cudaGraphDestroy(g);
      CK(e);
      p->graph = ex;
      p->graph_key = key;
    }
    CK(cudaGraphLaunch(p->graph, st));
    note_launch(p->graph_launches);
    std::vector<double> vals;
    if (terms && nterms) {
      vals.resize(P.zlist.size() * B);
      CK(cudaMemcpyAsync(vals.data(), d_out, sizeof(double) * vals.size(), cudaMemcpyDeviceToHost, st));
    }
    CK(cudaEventRecord(p->ev_out, st));
    CK(cudaStreamWaitEvent(user_st, p->ev_out, 0));
    if (!p->tcdesc.empty()) {
      int err = 0;
      CK(cudaMemcpyAsync(&err, p->d_err.p, sizeof(int), cudaMemcpyDeviceToHost, st));
      CK(cudaStreamSynchronize(st));
      if (err) throw Error(QS_ERR_TIMEOUT, "tensor-core pass: an MMA completion wait timed out");
    }
    if (terms && nterms) {
      CK(cudaStreamSynchronize(st));
      for (int b = 0; b < B; ++b) expvals[b] = combine_expval(P, terms, vals.data() + (size_t)b * P.zlist.size());
    }
  });
}

}  // extern "C"
