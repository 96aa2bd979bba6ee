// C ABI of the simulator: state objects, plans, observables, adjoint gradient,
// batched execution, autotuner. Host code only; every arithmetic step on a
// state runs in the CUDA kernels of kernels_*.cu.
#include "runtime.h"

#include <cstdio>

namespace qs {
namespace rt {
thread_local std::string g_err;
}  // namespace rt
void set_last_error(const std::string& msg) { rt::g_err = msg; }
}  // namespace qs

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

// Key of a gate list for the tuning cache: only the fields a gate's kind uses
// (targets up to nq, controls up to nctrl, the angle of rotations, the
// parameter binding, the matrix of U1/U2), so unused fields left unset by a
// caller do not split one circuit into several keys.
uint64_t gate_list_key(const qs_gate* gates, size_t ng) {
  uint64_t h = fnv1a(&ng, sizeof(ng));
  auto mix = [&](const void* d, size_t b) { h = fnv1a(d, b, h); };
  for (size_t i = 0; i < ng; ++i) {
    const qs_gate& g = gates[i];
    mix(&g.kind, sizeof(g.kind));
    const int nq = std::max(0, std::min(g.nq, 2)), nc = std::max(0, std::min(g.nctrl, 2));
    mix(&nq, sizeof(nq));
    mix(g.q, sizeof(int32_t) * nq);
    mix(&nc, sizeof(nc));
    mix(g.ctrl, sizeof(int32_t) * nc);
    const bool angle = g.kind == QS_GATE_RX || g.kind == QS_GATE_RY || g.kind == QS_GATE_RZ || g.kind == QS_GATE_P;
    if (angle) {
      const int32_t pi = g.param_index >= 0 ? g.param_index : -1;
      mix(&pi, sizeof(pi));
      mix(&g.param, sizeof(g.param));
      if (pi >= 0) mix(&g.scale, sizeof(g.scale));
    }
    if (g.kind == QS_GATE_U1) mix(g.mat, sizeof(double) * 8);
    if (g.kind == QS_GATE_U2) mix(g.mat, sizeof(double) * 32);
  }
  return h;
}

std::vector<uint64_t> tune_key(int n, qs_dtype dt, const qs_gate* gates, size_t ng) {
  return {(uint64_t)n, (uint64_t)dt, (uint64_t)ng, gate_list_key(gates, ng)};
}

void check_tune_args(int n, qs_dtype dt, const qs_gate* gates, size_t ng) {
  require(n >= 1 && n <= kMaxQubits, "n out of range");
  require(dt == QS_C64 || dt == QS_C128, "bad dtype");
  require(ng == 0 || gates != nullptr, "gates is NULL");
  require(ng <= kMaxGates, "too many gates (at most 2^30 per circuit)");
}

std::vector<qs_plan_opts> tune_candidates(int n, qs_dtype dt) {
  std::vector<qs_plan_opts> c;
  auto add = [&](int mode, int k, int m, int L, int tcmin, int staging = 0) {
    qs_plan_opts o;
    std::memset(&o, 0, sizeof(o));
    o.mode = mode;
    o.fuse_k = k;
    o.tile_qubits = m;
    o.low_qubits = L;
    o.reserved[0] = tcmin;
    o.reserved[5] = staging;
    c.push_back(o);
  };
  add(QS_MODE_PER_GATE, 0, 0, 0, 0);
  const int ks[] = {1, 2, 3, 4};
  for (int k : ks) {
    if (dt == QS_C64) {
      add(QS_MODE_FUSED, k, 12, 4, 0);
      add(QS_MODE_FUSED, k, 13, 4, 0);
      add(QS_MODE_FUSED, k, 12, 5, 0, 2);   // tiles staged by bulk copies (256-byte runs)
    } else {
      add(QS_MODE_FUSED, k, 11, 3, 0);
      add(QS_MODE_FUSED, k, 12, 4, 0);
    }
  }
  if (dt == QS_C64 && n >= 13) {
    const int tm[] = {2, 4, 8};
    for (int t : tm) add(QS_MODE_TENSOR, 2, 13, 4, t);
    add(QS_MODE_TENSOR, 5, 13, 4, 2);   // 5-qubit contraction, blocks padded to 6
  }
  if (dt == QS_C128 && n >= 12) {   // every block on tensor cores, or only those of >= 2 / 4 gates
    const int tm[] = {1, 2, 4};
    for (int t : tm) add(QS_MODE_TENSOR, 2, 11, 3, t);
    add(QS_MODE_TENSOR, 4, 11, 3, 1);   // 4-qubit contraction, blocks padded to 5
  }
  return c;
}

// =================================================================== C ABI

extern "C" {

const char* qs_last_error(void) { return g_err.c_str(); }

qs_status qs_plan_set_wait_limit(qs_plan_t p, uint32_t polls) {
  return guard([&] {
    require(p != nullptr, "plan is NULL");
    p->tc_spin = polls;
    p->graph_key.clear();   // a captured graph holds the old limit: recapture on the next batch
  });
}

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
      if (blk.rep == OP_TC && p->dt == QS_C128) {
        // digit planes: compare the values they stand for (the FP64 products on the
        // host and the device may differ in their last bits)
        std::vector<uint16_t> img(kTc128WElems);
        build_w_digits(p->h_btab.data() + p->block_off[b], img.data());
        for (size_t st = 0; st < p->steps.size(); ++st)
          if (p->steps[st].kind == 1 && p->exec_ops[p->pass_ops[st].first].block == (int)b) {
            const uint16_t* dv = wdev.data() + (size_t)p->steps[st].idx * p->wimg_pass;
            for (uint32_t nn = 0; nn < 64; ++nn)
              for (uint32_t k = 0; k < 64; ++k)
                worst = std::max(worst, std::fabs(w_digit_value(img.data(), nn, k) - w_digit_value(dv, nn, k)));
          }
      } else if (blk.rep == OP_TC) {
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
int64_t qs_device_alloc_count(void) { return qs::device_alloc_count(); }
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
    note_device_alloc();
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
    stream_after(dst->st, src->st);
    CK(cudaMemcpyAsync(dst->d, src->d, src->bytes(), cudaMemcpyDeviceToDevice, dst->st));
    stream_after(src->st, dst->st);   // later writes of src wait for the copy
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
    check_tune_args(s->n, s->dt, gates, ngates);
    const std::vector<uint64_t> key = tune_key(s->n, s->dt, gates, ngates);
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

qs_status qs_tune_cache_lookup(int n, qs_dtype dtype, const qs_gate* gates, size_t ngates, qs_plan_opts* best,
                               double* best_ms, int* found) {
  return guard([&] {
    check_tune_args(n, dtype, gates, ngates);
    require(found != nullptr, "found is NULL");
    std::lock_guard<std::mutex> lock(g_tune_mu);
    auto it = g_tune_cache.find(tune_key(n, dtype, gates, ngates));
    *found = it != g_tune_cache.end();
    if (*found) {
      if (best) *best = it->second.opts;
      if (best_ms) *best_ms = it->second.ms;
    }
  });
}

qs_status qs_tune_cache_put(int n, qs_dtype dtype, const qs_gate* gates, size_t ngates, const qs_plan_opts* opts,
                            double ms) {
  return guard([&] {
    check_tune_args(n, dtype, gates, ngates);
    require(opts != nullptr, "opts is NULL");
    require(std::isfinite(ms) && ms >= 0, "ms must be finite and >= 0");
    std::unique_ptr<qs_plan_s> p(create_plan(n, dtype, gates, ngates, opts));   // the options must plan this circuit
    std::lock_guard<std::mutex> lock(g_tune_mu);
    g_tune_cache[tune_key(n, dtype, gates, ngates)] = TuneEntry{*opts, ms};
  });
}

qs_status qs_tune_cache_clear(void) {
  return guard([&] {
    std::lock_guard<std::mutex> lock(g_tune_mu);
    g_tune_cache.clear();
  });
}

// Text format: a first line "qsgb300-tune 1", then one entry per line:
// n dtype ngates key(hex) ms mode fuse_k tile_qubits low_qubits paper_mode
// tc_precision threads fuse_parametric reserved[0..7]
qs_status qs_tune_cache_save(const char* path, int64_t* entries) {
  return guard([&] {
    require(path != nullptr, "path is NULL");
    std::string out = "qsgb300-tune 1\n";
    int64_t cnt = 0;
    {
      std::lock_guard<std::mutex> lock(g_tune_mu);
      for (const auto& kv : g_tune_cache) {
        const qs_plan_opts& o = kv.second.opts;
        char line[512];
        std::snprintf(line, sizeof(line), "%llu %llu %llu %016llx %.17g %d %d %d %d %d %d %d %d",
                      (unsigned long long)kv.first[0], (unsigned long long)kv.first[1],
                      (unsigned long long)kv.first[2], (unsigned long long)kv.first[3], kv.second.ms, o.mode,
                      o.fuse_k, o.tile_qubits, o.low_qubits, o.paper_mode, o.tc_precision, o.threads,
                      o.fuse_parametric);
        out += line;
        for (int r = 0; r < 8; ++r) out += " " + std::to_string(o.reserved[r]);
        out += "\n";
        ++cnt;
      }
    }
    FILE* f = std::fopen(path, "w");
    require(f != nullptr, "cannot open the cache file for writing");
    const bool ok = std::fwrite(out.data(), 1, out.size(), f) == out.size();
    const bool closed = std::fclose(f) == 0;
    require(ok && closed, "cannot write the cache file");
    if (entries) *entries = cnt;
  });
}

qs_status qs_tune_cache_load(const char* path, int64_t* entries) {
  return guard([&] {
    require(path != nullptr, "path is NULL");
    FILE* f = std::fopen(path, "r");
    require(f != nullptr, "cannot open the cache file");
    std::string text;
    char buf[4096];
    size_t got;
    while ((got = std::fread(buf, 1, sizeof(buf), f)) > 0) text.append(buf, got);
    std::fclose(f);
    // parse everything first: a malformed file leaves the cache unchanged
    std::vector<std::pair<std::vector<uint64_t>, TuneEntry>> parsed;
    size_t pos = 0;
    int line_no = 0;
    while (pos < text.size()) {
      size_t end = text.find('\n', pos);
      if (end == std::string::npos) end = text.size();
      const std::string line = text.substr(pos, end - pos);
      pos = end + 1;
      ++line_no;
      if (line_no == 1) {
        require(line == "qsgb300-tune 1", "not a tuning cache file (bad first line)");
        continue;
      }
      if (line.empty()) continue;
      unsigned long long n, dt, ng, key;
      double ms;
      qs_plan_opts o;
      std::memset(&o, 0, sizeof(o));
      int used = 0;
      const int k = std::sscanf(line.c_str(), "%llu %llu %llu %llx %lg %d %d %d %d %d %d %d %d %d %d %d %d %d %d %d %d%n",
                                &n, &dt, &ng, &key, &ms, &o.mode, &o.fuse_k, &o.tile_qubits, &o.low_qubits,
                                &o.paper_mode, &o.tc_precision, &o.threads, &o.fuse_parametric, &o.reserved[0],
                                &o.reserved[1], &o.reserved[2], &o.reserved[3], &o.reserved[4], &o.reserved[5],
                                &o.reserved[6], &o.reserved[7], &used);
      const std::string where = "cache file line " + std::to_string(line_no);
      if (k != 21 || line.find_first_not_of(" \t\r", (size_t)used) != std::string::npos)
        throw Error(QS_ERR_ARG, where + ": malformed entry");
      if (n < 1 || n > (unsigned long long)kMaxQubits || (dt != QS_C64 && dt != QS_C128) || ng > kMaxGates ||
          !std::isfinite(ms) || ms < 0 || o.mode < QS_MODE_PER_GATE || o.mode > QS_MODE_SMGP)
        throw Error(QS_ERR_ARG, where + ": value out of range");
      parsed.push_back({{n, dt, ng, key}, TuneEntry{o, ms}});
    }
    require(line_no >= 1, "not a tuning cache file (empty)");
    {
      std::lock_guard<std::mutex> lock(g_tune_mu);
      for (auto& e : parsed) g_tune_cache[e.first] = e.second;
    }
    if (entries) *entries = (int64_t)parsed.size();
  });
}

qs_status qs_plan_execute(qs_plan_t p, qs_state_t s, const double* theta, size_t ntheta) {
  return guard([&] {
    require(p != nullptr, "plan is NULL");
    check_state(s);
    execute(*p, *s, theta, ntheta);
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
    stream_after(a->st, b->st);
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
    stream_after(s->st, out->st);
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
    std::vector<double> grad(ntheta, 0.0);   // outputs are written only on success
    for (int r = 0; r < rows; ++r) {
      const HGate& g = rp->gates[row_gate[r]];
      require((size_t)g.param_index < ntheta, "theta shorter than the parameter indices");
      grad[g.param_index] += 2.0 * g.scale * sums[r];
    }
    std::copy(grad.begin(), grad.end(), grad_out);
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
    plan_wait(*p, st);
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
    // ordered on the plan's stream: a replay still running there reads the previous table
    CK(cudaMemcpyAsync(p->d_psis.p, ptrs.data(), sizeof(void*) * B, cudaMemcpyHostToDevice, st));
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
    plan_done(*p, st);
    check_tc_error(*p, st);
    if (terms && nterms) {
      CK(cudaStreamSynchronize(st));
      for (int b = 0; b < B; ++b) expvals[b] = combine_expval(P, terms, vals.data() + (size_t)b * P.zlist.size());
    }
  });
}

qs_status qs_apply_circuit_batched(qs_state_t* states, int B, const qs_gate* gates, size_t ngates,
                                   const double* theta, size_t ntheta, const qs_plan_opts* opts) {
  return guard([&] {
    require(states != nullptr && B >= 1, "bad arguments");
    check_state(states[0]);
    std::unique_ptr<qs_plan_s> p(create_plan(states[0]->n, states[0]->dt, gates, ngates, opts));
    const qs_status st = qs_plan_execute_batched(p.get(), states, B, theta, ntheta, nullptr, 0, nullptr);
    if (st != QS_OK) throw Error(st, g_err);
    CK(cudaStreamSynchronize(states[0]->st));   // the plan's device tables are freed on return
  });
}

}  // extern "C"
