// Host-resident states streamed through device buffers (Section 3.2's
// batches) and the host pipeline of independent inputs. Host code only.
#include "runtime.h"

// ---------------------------------------------------------------- host-resident states (Section 3.2)

// Streamed passes: the tile-pass scheduler with the l low qubits always in the
// "tile" and at most h batch-index qubits (>= l) beside them; gates move ahead
// of the gates they commute with, so a pass gathers every gate that fits.
// Each pass moves the state once through the host link in each direction.
static std::vector<StreamPass> plan_stream_passes(int n, const std::vector<HGate>& gates, int l, int h) {
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

extern "C" {

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
      for (auto& pp : plans) check_tc_error(*pp, sd);
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
    DevBuf dnorm;   // outlives the streams' work (freed after the synchronisations below)
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
      plan_wait(*p, sc);
      resolve_theta(*p, theta, ntheta, 1, sc);
      build_device_blocks(*p, 1, sc);
      // norms land in a device array read once at the end: a per-step copy into the
      // caller's (pageable) array would block this loop until that step's circuit ends
      if (norms) dnorm.ensure(sizeof(double) * std::max(1, count));
      for (int i = 0; i < count; ++i) {
        const int b = i % nwork;
        qs_state_s& w = *work[b];
        CK(cudaStreamWaitEvent(si, stored[b], 0));
        CK(cudaMemcpyAsync(w.d, host_in[i], bytes, cudaMemcpyHostToDevice, si));
        CK(cudaEventRecord(loaded[b], si));
        CK(cudaStreamWaitEvent(sc, loaded[b], 0));
        issue_circuit(*p, w.d, 0, sc);
        if (norms) CK(launch_norm(w.d, w.n, w.dt, w.scratch.as<double>(), dnorm.as<double>() + i, sc));
        CK(cudaEventRecord(computed[b], sc));
        CK(cudaStreamWaitEvent(so, computed[b], 0));
        if (host_out && host_out[i]) CK(cudaMemcpyAsync(host_out[i], w.d, bytes, cudaMemcpyDeviceToHost, so));
        CK(cudaEventRecord(stored[b], so));
      }
      CK(cudaStreamSynchronize(so));
      CK(cudaStreamSynchronize(sc));
      CK(cudaStreamSynchronize(si));
      if (norms && count > 0) CK(cudaMemcpy(norms, dnorm.p, sizeof(double) * count, cudaMemcpyDeviceToHost));
      for (int b = 0; b < nwork; ++b) CK(cudaStreamWaitEvent(work[b]->st, stored[b], 0));
      check_tc_error(*p, sc);
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

}  // extern "C"
