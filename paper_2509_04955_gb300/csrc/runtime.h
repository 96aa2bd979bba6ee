// Host runtime shared by the translation units of the C ABI: error
// handling, device buffers, the state and plan objects, and the plan,
// execution and observable helpers (runtime.cpp). Internal: not installed.
#pragma once

#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <functional>
#include <map>
#include <memory>
#include <mutex>
#include <new>
#include <stdexcept>
#include <string>
#include <vector>

#include "planner.h"
#include "qs_error.h"
#include "qs_internal.h"

namespace qs {
int64_t launch_count();
void set_last_error(const std::string& msg);

namespace rt {

// message of the last failed call on this thread (qs_last_error)
extern thread_local std::string g_err;


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
  } catch (const std::length_error& e) {   // a host container asked for more than it can hold
    g_err = std::string("host allocation too large: ") + e.what();
    return QS_ERR_OOM;
  } catch (const std::exception& e) {
    g_err = e.what();
    return QS_ERR_CUDA;
  }
}

inline void require(bool c, const char* msg) {
  if (!c) throw Error(QS_ERR_ARG, msg);
}

inline void require_device() {
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
    note_device_alloc();
    bytes = b;
  }
  template <class T> T* as() const { return (T*)p; }
};

inline size_t amp_bytes(qs_dtype dt) { return dt == QS_C64 ? 8 : 16; }

// True while `st` is being captured into a CUDA graph by the caller. The
// library's cross-stream events stay out of such captures: a captured wait on
// an event recorded outside the capture is not allowed, and the graph orders
// its own launches.
inline bool capturing(cudaStream_t st) {
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  if (cudaStreamIsCapturing(st, &cs) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return cs != cudaStreamCaptureStatusNone;
}

// Makes later work on `waiter` wait for everything queued on `producer` so far
// (two states on different streams); nothing to do when they are one stream.
inline void stream_after(cudaStream_t waiter, cudaStream_t producer) {
  if (waiter == producer || capturing(waiter) || capturing(producer)) return;
  cudaEvent_t e;
  CK(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
  cudaError_t r = cudaEventRecord(e, producer);
  if (r == cudaSuccess) r = cudaStreamWaitEvent(waiter, e, 0);
  cudaEventDestroy(e);   // released once the wait has been satisfied
  CK(r);
}

}  // namespace rt
}  // namespace qs

using namespace qs;
using namespace qs::rt;

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
  std::vector<TcPassDesc> tcdesc;   // complex64 tensor-core passes
  std::vector<Tc5PassDesc> tc5desc; // complex128 tensor-core passes
  // per TC pass: 16-bit hi image then lo image (64 KiB, complex64) or five digit planes (40 KiB, complex128)
  std::vector<uint16_t> h_wimg;
  int64_t wimg_pass = 32768;       // uint16 elements per pass in h_wimg / d_wimg
  uint32_t tc_spin = 0;            // polls per tensor-core pipeline wait (0 = default bound)
  bool has_tc() const { return !tcdesc.empty() || !tc5desc.empty(); }
  bool has_bulk_tiles() const {
    for (const PassDesc& d : pdesc)
      if (d.bulk) return true;
    return false;
  }
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
  // recorded after each execution's last use of the device tables; the next
  // execution, on whatever stream, waits for it before it rewrites them
  cudaEvent_t ev_done = nullptr;
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
    if (ev_done) cudaEventDestroy(ev_done);
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

namespace qs {
namespace rt {

struct TermGroup {
  uint64_t x;
  std::vector<int> idx;   // term indices
};

struct PreparedTerms {
  std::vector<TermGroup> groups;
  std::vector<uint64_t> zlist;        // group order
  std::vector<int> term_of;           // term index per zlist entry
  std::vector<std::pair<int, int>> launches;   // (group, offset into zlist) per launch, count via chunk
  std::vector<int> counts;
};

constexpr int kZPerLaunch = kExpvalMaxZ;

// ---- device tables of a plan, upload and execution (runtime.cpp)
void fill_fixed_table(const qs_plan_s& p, std::vector<double2>& tab);
void compute_blocks(qs_plan_s& p, const double* theta, bool only_parametric);
void ensure_gtab_rows(qs_plan_s& p, int rows);
void ensure_block_rows(qs_plan_s& p, int rows);
void build_device_blocks(qs_plan_s& p, int rows, cudaStream_t st);
void upload(qs_plan_s& p);
void check_state(const qs_state_s* s);
void plan_wait(qs_plan_s& p, cudaStream_t st);   // st waits for the plan's previous execution
void plan_done(qs_plan_s& p, cudaStream_t st);   // marks the end of this execution on st
void issue_circuit(qs_plan_s& p, void* psi, int row, cudaStream_t st, bool timed = false);
int batched_wave(const qs_plan_s& p, int B);
void issue_circuit_batched(qs_plan_s& p, void* const* d_psis, int B, cudaStream_t st,
                           const std::function<void(int, int)>& after_wave = nullptr);
void resolve_theta(qs_plan_s& p, const double* theta, size_t ntheta, int rows, cudaStream_t st);
void execute(qs_plan_s& p, qs_state_s& s, const double* theta, size_t ntheta);
void check_tc_error(qs_plan_s& p, cudaStream_t st);
// ---- tensor-core W images (16-bit hi / lo split, 128-byte swizzle)
uint16_t bf16_rne(float f);
float bf16_to_float(uint16_t h);
uint16_t f16_rne(float f);
float f16_to_float(uint16_t h);
size_t sw128_offset_host(uint32_t row, uint32_t k);
void build_w_image(const double2* U, uint16_t* img, bool half);
void build_w_digits(const double2* U, uint16_t* img);
double w_digit_value(const uint16_t* img, uint32_t nn, uint32_t k);
float w_to_float(uint16_t v, bool half);
// ---- planning: passes of every kind, options, plan construction
void register_device_block(qs_plan_s& P, const Block& blk, int kind, int64_t out);
void emit_tile_passes(qs_plan_s& P, const std::vector<OpRec>& ops, const std::vector<PassRec>& passes,
                      const std::vector<int>& order, int low_qubits, qs_plan_info& in);
void emit_phase_pass(qs_plan_s& P, const OpRec& r, qs_plan_info& in);
void emit_tc_pass(qs_plan_s& P, const OpRec& r, qs_plan_info& in);
void default_opts(qs_plan_opts& o, qs_dtype dt, int n);
void plan_smgp(qs_plan_s& p);
qs_plan_s* create_plan(int n, qs_dtype dt, const qs_gate* gates, size_t ng, const qs_plan_opts* opts,
                       bool no_merge = false);
// ---- observables: Pauli sums grouped by x mask
std::vector<TermGroup> group_terms(int n, const qs_pauli_term* t, size_t nt);
double term_factor(const qs_pauli_term& t);
PreparedTerms prepare_terms(int n, const qs_pauli_term* t, size_t nt);
void issue_expval(const qs_state_s& s, const PreparedTerms& P, const uint64_t* d_z, double* d_partials,
                  double* d_out, cudaStream_t st);
double combine_expval(const PreparedTerms& P, const qs_pauli_term* t, const double* vals);
size_t partial_bytes(int rows);
double expval_sync(qs_state_s& s, const qs_pauli_term* t, size_t nt);
void upload_pauli_apply(const qs_pauli_term* t, size_t nt, DevBuf& buf, cudaStream_t st, uint64_t** dx,
                        uint64_t** dz, double2** dph, std::vector<unsigned char>& host);

}  // namespace rt
}  // namespace qs
