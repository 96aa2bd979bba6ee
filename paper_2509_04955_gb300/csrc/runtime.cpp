// Plans (contraction, pass scheduling, tile / tensor-core / phase passes,
// staggered groups), their upload and execution, and the observable helpers.
// Host code only; every arithmetic step on a state runs in kernels_*.cu.
#include "runtime.h"

namespace qs {
namespace rt {
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
  if (p.has_tc() && want > p.wimg_rows) {
    p.d_wimg.release();
    p.d_wimg.ensure(sizeof(uint16_t) * p.h_wimg.size() * want);
    CK(cudaMemcpy(p.d_wimg.p, p.h_wimg.data(), sizeof(uint16_t) * p.h_wimg.size(), cudaMemcpyHostToDevice));
    p.wimg_rows = want;
  }
}

void build_device_blocks(qs_plan_s& p, int rows, cudaStream_t st) {
  if (p.h_dblocks.empty()) return;
  if (p.gtab_rows < rows || p.btab_rows < rows || (p.has_tc() && p.wimg_rows < rows))
    throw Error(QS_ERR_CUDA, "internal: block tables have fewer rows than the batch");
  const size_t G = std::max<size_t>(1, p.gates.size());
  CK(launch_build_blocks(p.d_dblocks.as<DevBlock>(), (int)p.h_dblocks.size(), p.d_dmem.as<DevMember>(),
                         p.d_gtab.as<double2>(), (int64_t)(16 * G), rows, p.d_btab.as<double2>(), p.btab_elems,
                         p.d_wimg.as<uint16_t>(), (int64_t)p.h_wimg.size(),
                         p.dt == QS_C128 ? 2 : (p.tc_prec == 4 ? 1 : 0), p.wimg_pass, st));
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
  if (!p.tc5desc.empty()) CK(prepare_tc128_pass());
  if (!p.h_dblocks.empty()) CK(prepare_build_blocks());
  p.uploaded = true;
}

void check_state(const qs_state_s* s) { require(s != nullptr && s->d != nullptr, "null state"); }

// An event (not the previous stream itself, which the caller may have destroyed
// since) orders executions of one plan on different streams. Inside a caller's
// stream capture the event is left alone (see capturing()).

void plan_wait(qs_plan_s& p, cudaStream_t st) {
  if (p.ev_done && !capturing(st)) CK(cudaStreamWaitEvent(st, p.ev_done, 0));
}

void plan_done(qs_plan_s& p, cudaStream_t st) {
  if (capturing(st)) return;
  if (!p.ev_done) CK(cudaEventCreateWithFlags(&p.ev_done, cudaEventDisableTiming));
  CK(cudaEventRecord(p.ev_done, st));
}

// Issues the kernels of one circuit execution on `st` for batch row `row` of
// the gate table (theta already resolved into it).
void issue_circuit(qs_plan_s& p, void* psi, int row, cudaStream_t st, bool timed) {
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
      PassDesc pd = p.pdesc[p.steps[i].idx];
      pd.err = p.d_err.as<int>();
      pd.spin = p.tc_spin;
      CK(launch_tile_pass(psi, p.n, p.dt, pd, p.d_ops.as<DevOp>(), gtab, p.d_btab.as<double2>(), 0, st));
    } else if (p.steps[i].kind == 2) {
      const double* th = p.theta_needed ? p.d_theta.as<double>() + (size_t)row * p.theta_stride : nullptr;
      CK(launch_phase_pass(psi, nullptr, 1, p.n, p.dt, p.d_pterms.as<DevPhaseTerm>(), p.phdesc[p.steps[i].idx], th,
                           p.theta_stride, st));
    } else {
      const int t = p.steps[i].idx;
      const uint16_t* w = p.d_wimg.as<uint16_t>() + (size_t)t * p.wimg_pass;
      if (p.dt == QS_C128)
        CK(launch_tc128_pass(psi, nullptr, 1, 0, p.n, p.tc5desc[t], w, p.d_err.as<int>(), st, p.tc_spin));
      else
        CK(launch_tc_pass(psi, p.n, p.tcdesc[t], w, p.tc_prec, p.tc_pipe, p.d_err.as<int>(), st, p.tc_spin));
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
                           const std::function<void(int, int)>& after_wave) {
  const size_t G = std::max<size_t>(1, p.gates.size());
  if (p.gtab_rows < B || (!p.h_dblocks.empty() && (p.btab_rows < B || (p.has_tc() && p.wimg_rows < B))))
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
        PassDesc pd = p.pdesc[stp.idx];
        pd.err = p.d_err.as<int>();
        pd.spin = p.tc_spin;
        CK(launch_tile_pass_batched(nullptr, ps, nb, (int64_t)(16 * G), p.btab_elems, w0, p.n, p.dt, pd,
                                    p.d_ops.as<DevOp>(), p.d_gtab.as<double2>() + (size_t)w0 * 16 * G,
                                    p.d_btab.as<double2>(), st));
      } else {
        const int64_t wstride = p.tc_param[stp.idx] ? (int64_t)p.h_wimg.size() : 0;
        const uint16_t* w = p.d_wimg.as<uint16_t>() + (size_t)stp.idx * p.wimg_pass + (size_t)w0 * wstride;
        if (p.dt == QS_C128)
          CK(launch_tc128_pass(nullptr, ps, nb, wstride, p.n, p.tc5desc[stp.idx], w, p.d_err.as<int>(), st,
                               p.tc_spin));
        else
          CK(launch_tc_pass_batched(nullptr, ps, nb, wstride, p.n, p.tcdesc[stp.idx], w, p.tc_prec, p.tc_pipe,
                                    p.d_err.as<int>(), st, p.tc_spin));
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
  plan_wait(p, s.st);
  resolve_theta(p, theta, ntheta, 1, s.st);
  build_device_blocks(p, 1, s.st);
  issue_circuit(p, s.d, 0, s.st, p.timing);
  plan_done(p, s.st);
  check_tc_error(p, s.st);
}

// Reads the tensor-core passes' error flag after the work queued on `st`,
// clears it for the next execution and reports a timeout.
void check_tc_error(qs_plan_s& p, cudaStream_t st) {
  if (!p.has_tc() && !p.has_bulk_tiles()) return;
  int err = 0;
  CK(cudaMemcpyAsync(&err, p.d_err.p, sizeof(int), cudaMemcpyDeviceToHost, st));
  CK(cudaStreamSynchronize(st));
  if (err) {
    CK(cudaMemsetAsync(p.d_err.p, 0, sizeof(int), st));
    CK(cudaStreamSynchronize(st));
    throw Error(QS_ERR_TIMEOUT, "tensor-core or bulk-staged tile pass: a pipeline wait ran out of polls");
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

// Digit planes of a 32x32 complex block U for the complex128 tensor-core pass:
// entry (nn, k) of the N x K = 64 x 64 operand is W[k][nn] of the real
// embedding, w = 2^-8 sum_{j<6} g_j 2^(-9 j) with balanced integer digits
// (|g_j| <= 256; X = rint(w 2^53) split from the bottom), plane j (j < 6)
// stored as fp16 integers in the K-major 128-byte-swizzled layout (8 KiB per
// plane). The device builder (kernels_build.cu) follows the same steps.
void build_w_digits(const double2* U, uint16_t* img) {
  for (uint32_t nn = 0; nn < 64; ++nn)
    for (uint32_t k = 0; k < 64; ++k) {
      const uint32_t co = nn >> 1, b = nn & 1, ci = k >> 1, a = k & 1;
      const double ur = U[co * 32 + ci].x, ui = U[co * 32 + ci].y;
      const double w = (a == 0) ? (b == 0 ? ur : ui) : (b == 0 ? -ui : ur);
      long long X = std::llrint(std::ldexp(w, 53));
      int g[6];
      for (int j = 5; j >= 1; --j) {
        g[j] = (int)(((X + 256) & 511) - 256);
        X = (X - g[j]) / 512;
      }
      g[0] = (int)X;
      const size_t off = (nn * 128 + (((k >> 3) ^ (nn & 7)) << 4) + (k & 7) * 2) / 2;
      for (int j = 0; j < 6; ++j) img[(size_t)j * 4096 + off] = f16_rne((float)g[j]);
    }
}

// The value an entry (nn, k) of a digit image stands for: 2^-8 sum_{j<6} g_j 2^(-9 j).
double w_digit_value(const uint16_t* img, uint32_t nn, uint32_t k) {
  const size_t off = (nn * 128 + (((k >> 3) ^ (nn & 7)) << 4) + (k & 7) * 2) / 2;
  double v = (double)f16_to_float(img[(size_t)5 * 4096 + off]);
  for (int j = 4; j >= 0; --j) v = v / 512.0 + (double)f16_to_float(img[(size_t)j * 4096 + off]);
  return std::ldexp(v, -8);
}

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
    // reserved[5] = 2: runs of at least 16 bytes moved by bulk copies into two
    // tile buffers, where both fit (FP32-pair tiles keep the register path)
    const size_t amp = dt == QS_C64 ? 8 : 16;
    pd.bulk = (P.opts.reserved[5] == 2 && !pd.df && ((amp << pd.L) % 16) == 0) ? 1 : 0;
    if (pd.bulk && tile_pass_smem_bytes(pd, dt) > 227 * 1024) pd.bulk = 0;
    in.reserved[0] += pd.bulk;
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

// A complex128 tensor-core pass: one dense 5-qubit block over tiles of the
// block's qubits and the 7 lowest other qubits; W as five digit planes.
static void emit_tc128_pass(qs_plan_s& P, const OpRec& r, qs_plan_info& in) {
  const Block& blk = P.blocks[r.block];
  Tc5PassDesc t;
  std::memset(&t, 0, sizeof(t));
  require(blk.qubits.size() == 5, "internal: complex128 tensor-core block needs 5 qubits");
  for (int j = 0; j < 5; ++j) t.col[j] = blk.qubits[j];
  int nr = 0;
  for (int q = 0; q < P.n && nr < 7; ++q)
    if (std::find(blk.qubits.begin(), blk.qubits.end(), q) == blk.qubits.end()) t.row[nr++] = q;
  require(nr == 7, "internal: tensor-core tile needs 7 row qubits");
  std::vector<int> tile(t.row, t.row + 7);
  tile.insert(tile.end(), t.col, t.col + 5);
  std::sort(tile.begin(), tile.end());
  for (int j = 0; j < 12; ++j) t.tile[j] = tile[j];
  const size_t w0 = P.h_wimg.size();
  P.h_wimg.resize(w0 + kTc128WElems);
  if (blk.parametric)
    register_device_block(P, blk, 2, (int64_t)P.tc5desc.size());   // digit planes rebuilt per row on the device
  else
    build_w_digits(P.h_btab.data() + P.block_off[r.block], P.h_wimg.data() + w0);
  P.tc_param.push_back(blk.parametric ? 1 : 0);
  DevOp d;
  std::memset(&d, 0, sizeof(d));
  d.type = OP_TC;
  d.k = 5;
  const int b = (int)P.dops.size();
  P.dops.push_back(d);
  P.exec_ops.push_back(r);
  P.steps.push_back({1, (int)P.tc5desc.size()});
  P.tc5desc.push_back(t);
  P.pass_tiles.push_back(tile);
  P.pass_ops.push_back({b, b + 1});
  in.flops_per_amp += 8.0 * 32;
  in.max_block_qubits = std::max(in.max_block_qubits, 5);
}

void emit_tc_pass(qs_plan_s& P, const OpRec& r, qs_plan_info& in) {
  if (P.dt == QS_C128) {
    emit_tc128_pass(P, r, in);
    return;
  }
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
                       bool no_merge) {
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
  if (tensor && dt == QS_C128) {
    // complex128: 5-qubit blocks as exact fp16 digit products (one arithmetic only)
    require(o.tc_precision == 0, "complex128 tensor-core passes take tc_precision 0 (exact digit products)");
    require(o.reserved[1] == 0, "complex128 tensor-core passes have one pipeline (reserved[1] = 0)");
    p->tc_prec = 0;
    p->wimg_pass = kTc128WElems;
    if (n < 12) tensor = false;   // a tile needs 12 qubits; smaller states use CUDA-core blocks
  } else if (tensor) {
    require(o.tc_precision == 0 || o.tc_precision == 1 || o.tc_precision == 3 || o.tc_precision == 4,
            "tc_precision must be 1, 3 or 4");
    p->tc_prec = o.tc_precision == 0 ? 4 : o.tc_precision;
    require(o.reserved[1] == 0 || o.reserved[1] == 1, "tensor-core pipeline (reserved[1]) must be 0 or 1");
    p->tc_pipe = o.reserved[1];
    if (n < 13) tensor = false;   // a tensor-core tile needs 13 qubits; smaller states use CUDA-core blocks
  }
  const int tc_width = dt == QS_C128 ? 5 : 6;
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
  // tensor mode: contraction width fuse_k = 4 or 5 (complex64) / 4 (complex128), else the pass's
  // own width; narrower blocks are padded to the pass width below
  po.k = o.paper_mode ? 2
                      : (tensor ? ((user_k == 4 || (user_k == 5 && dt == QS_C64)) ? user_k : tc_width) : o.fuse_k);
  po.paper = o.paper_mode != 0;
  po.amp_bytes = (int)amp_bytes(dt);
  // GB300: FP32 FMA 128 lanes/clk/SM, FP64 about 1/59 of that (measured),
  // shared memory 128 B/clk/SM -> one byte costs one FP32 FMA slot.
  // complex128 CUDA-core passes in FP32 pairs (reserved[3] 0 or 1, the
  // default) cost about 15 FP32 instructions per FMA (a pair product and a
  // pair sum); reserved[3] = 2 keeps them in FP64
  require(o.reserved[3] >= 0 && o.reserved[3] <= 2, "complex128 arithmetic (reserved[3]) must be 0, 1 or 2");
  require(o.reserved[5] >= 0 && o.reserved[5] <= 2, "tile staging (reserved[5]) must be 0, 1 or 2");
  p->df = dt == QS_C128 && o.reserved[3] != 2;
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
    // A block worth a tensor-core pass (one HBM sweep) carries many gates in
    // complex64, where CUDA-core tile passes are cheap; in complex128 (FP64 or
    // FP32-pair tile passes) every block is. It is padded to the pass's width
    // (6 qubits complex64, 5 complex128) with the highest qubits it does not touch.
    const int tc_min_gates = o.reserved[0] > 0 ? o.reserved[0] : (dt == QS_C128 ? 1 : 10);
    for (Block& blk : p->blocks) {
      if ((int)blk.gates.size() >= tc_min_gates) {
        blk.rep = OP_TC;
        blk.diag = false;
        for (int q = n - 1; q >= 0 && (int)blk.qubits.size() < tc_width; --q)
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
  // Consecutive complex128 tensor-core passes hand the state over as FP32
  // pairs (about 48 significant bits, the same 16 bytes per amplitude): only
  // the first of a run reads complex128 and only the last writes it.
  if (dt == QS_C128)
    for (size_t i = 0; i < p->steps.size(); ++i)
      if (p->steps[i].kind == 1) {
        Tc5PassDesc& t = p->tc5desc[p->steps[i].idx];
        t.in_pairs = i > 0 && p->steps[i - 1].kind == 1;
        t.out_pairs = i + 1 < p->steps.size() && p->steps[i + 1].kind == 1;
      }
  in.passes = (int64_t)p->steps.size();
  in.launches = in.passes;
  in.sweeps = (double)in.passes;
  in.tile_qubits = o.tile_qubits;
  in.low_qubits = o.low_qubits;
  return p.release();
}

// ---------------------------------------------------------------- observables


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

}  // namespace rt
}  // namespace qs
