// Per-gate kernels (one launch per gate): the GB300 form of Algorithms 1-4.
//
// One thread per amplitude pair (the one-dimensional mapping of Section 3.3,
// Fig. 8), with the pair found by inserting zero bits at the sorted target and
// control positions of a pair counter instead of the mask test of Algorithm 1
// or the grouped loops of Algorithms 3-4: the same pairs, no idle iterations,
// and valid for controls on either side of the target (Eq. 4 for any c, t).
// Structured gates touch only the amplitudes they change:
//   DENSE1 / ANTI1: pairs (i, i | 2^t) with controls set            (Eq. 3, Eq. 4)
//   PHASE1: amplitudes with target and controls set (Z, S, T, P, CZ, CP)
//   DIAG1:  amplitudes with controls set (RZ)
//   SWAP2:  pairs (..0_a..1_b.., ..1_a..0_b..) with controls set
//   DENSE2: quads of Eq. 6 with local bit 0 = first target.
#include <cuda_runtime.h>
#include <math.h>

#include <atomic>

#include "cplx.cuh"
#include "qs_internal.h"

namespace qs {

static std::atomic<int64_t> g_launches{0};
static thread_local bool g_count_suspended = false;
void note_launch(int64_t k) {
  if (!g_count_suspended) g_launches += k;
}
void suspend_launch_count(bool on) { g_count_suspended = on; }
int64_t launch_count() { return g_launches.load(); }
static std::atomic<int64_t> g_allocs{0};
void note_device_alloc() { ++g_allocs; }
int64_t device_alloc_count() { return g_allocs.load(); }

int device_sm_count() {
  static std::atomic<int> sms{0};
  int v = sms.load();
  if (v > 0) return v;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
      v <= 0) {
    cudaGetLastError();
    return 152;   // not cached: asked again on the next call
  }
  sms.store(v);
  return v;
}

static int grid_for(uint64_t work, int threads) {
  // Enough CTAs to fill every SM several times over; the kernels stride.
  uint64_t want = (work + threads - 1) / threads;
  const uint64_t cap = (uint64_t)device_sm_count() * 16;
  if (want > cap) want = cap;
  if (want < 1) want = 1;
  return (int)want;
}

// ---------------------------------------------------------------- basis state

template <typename C>
__global__ void k_set_basis(C* __restrict__ psi, uint64_t dim, uint64_t x) {
  const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
  for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < dim; i += stride) {
    C v; v.x = (i == x) ? 1 : 0; v.y = 0;
    psi[i] = v;
  }
}

template <typename C>
__global__ void k_gather(const C* __restrict__ psi, const uint64_t* __restrict__ idx, uint64_t count,
                         C* __restrict__ out) {
  const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
  for (uint64_t k = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; k < count; k += stride) out[k] = psi[idx[k]];
}

cudaError_t launch_gather(const void* psi, qs_dtype dt, const uint64_t* idx, uint64_t count, void* out,
                          cudaStream_t st) {
  if (count == 0) return cudaSuccess;
  const int th = 256, gr = grid_for(count, th);
  if (dt == QS_C64) k_gather<float2><<<gr, th, 0, st>>>((const float2*)psi, idx, count, (float2*)out);
  else k_gather<double2><<<gr, th, 0, st>>>((const double2*)psi, idx, count, (double2*)out);
  note_launch();
  return cudaGetLastError();
}

cudaError_t launch_set_basis(void* psi, int n, qs_dtype dt, uint64_t x, cudaStream_t st) {
  const uint64_t dim = 1ull << n;
  const int th = 256, gr = grid_for(dim, th);
  if (dt == QS_C64) k_set_basis<float2><<<gr, th, 0, st>>>((float2*)psi, dim, x);
  else k_set_basis<double2><<<gr, th, 0, st>>>((double2*)psi, dim, x);
  note_launch();
  return cudaGetLastError();
}

// ---------------------------------------------------------------- resolve

// Fills the 2x2 matrix (slots 0..3) and its angle derivative (slots 4..7) of
// every parametric gate for every batch row from theta on the device.
// R_P(a) = exp(-i a P / 2), P(a) = diag(1, e^{ia}).
__global__ void k_resolve(const DevGate* __restrict__ gates, const int32_t* __restrict__ pg, int npg,
                          const double* __restrict__ theta, int64_t ntheta, int batch,
                          double2* __restrict__ table, int64_t stride) {
  const int total = npg * batch;
  for (int w = blockIdx.x * blockDim.x + threadIdx.x; w < total; w += gridDim.x * blockDim.x) {
    const int b = w / npg, j = w % npg;
    const int gi = pg[j];
    const DevGate g = gates[gi];
    const double a = g.param + g.scale * theta[(int64_t)b * ntheta + g.param_index];
    double s, c;
    sincos(0.5 * a, &s, &c);
    double2* m = table + (int64_t)b * stride + (int64_t)gi * 16;
    const double2 z = make_double2(0, 0);
    switch (g.kind) {
      case QS_GATE_RX:
        m[0] = make_double2(c, 0); m[1] = make_double2(0, -s); m[2] = make_double2(0, -s); m[3] = make_double2(c, 0);
        m[4] = make_double2(-0.5 * s, 0); m[5] = make_double2(0, -0.5 * c);
        m[6] = make_double2(0, -0.5 * c); m[7] = make_double2(-0.5 * s, 0);
        break;
      case QS_GATE_RY:
        m[0] = make_double2(c, 0); m[1] = make_double2(-s, 0); m[2] = make_double2(s, 0); m[3] = make_double2(c, 0);
        m[4] = make_double2(-0.5 * s, 0); m[5] = make_double2(-0.5 * c, 0);
        m[6] = make_double2(0.5 * c, 0); m[7] = make_double2(-0.5 * s, 0);
        break;
      case QS_GATE_RZ:  // diag(c - is, c + is); derivative diag(-i/2 e^{-ia/2}, i/2 e^{ia/2})
        m[0] = make_double2(c, -s); m[1] = z; m[2] = z; m[3] = make_double2(c, s);
        m[4] = make_double2(-0.5 * s, -0.5 * c); m[5] = z; m[6] = z; m[7] = make_double2(-0.5 * s, 0.5 * c);
        break;
      default: {  // QS_GATE_P: diag(1, e^{ia}); derivative diag(0, i e^{ia})
        double sa, ca;
        sincos(a, &sa, &ca);
        m[0] = make_double2(1, 0); m[1] = z; m[2] = z; m[3] = make_double2(ca, sa);
        m[4] = z; m[5] = z; m[6] = z; m[7] = make_double2(-sa, ca);
      }
    }
  }
}

cudaError_t launch_resolve(const DevGate* gates, const int32_t* pg, int npg, const double* theta,
                           int64_t ntheta, int batch, double2* table, int64_t stride,
                           cudaStream_t st) {
  if (npg == 0 || batch == 0) return cudaSuccess;
  const int th = 128, gr = (npg * batch + th - 1) / th;
  k_resolve<<<gr, th, 0, st>>>(gates, pg, npg, theta, ntheta, batch, table, stride);
  note_launch();
  return cudaGetLastError();
}

// ---------------------------------------------------------------- per-gate

template <typename R>
struct Mat2 { typename V2<R>::T m00, m01, m10, m11; };

template <typename R>
__device__ __forceinline__ Mat2<R> load_mat2(const double2* __restrict__ mat, bool adjoint) {
  Mat2<R> u;
  double2 a = mat[0], b = mat[1], c = mat[2], d = mat[3];
  if (adjoint) {  // conjugate transpose
    double2 t = b;
    b = make_double2(c.x, -c.y); c = make_double2(t.x, -t.y);
    a.y = -a.y; d.y = -d.y;
  }
  u.m00 = from_d<R>(a); u.m01 = from_d<R>(b); u.m10 = from_d<R>(c); u.m11 = from_d<R>(d);
  return u;
}

template <typename R, int FORM>
__global__ void __launch_bounds__(256) k_gate1(typename V2<R>::T* __restrict__ psi, uint64_t count,
                                               DevGate g, const double2* __restrict__ mat, bool adjoint) {
  using C = typename V2<R>::T;
  const Mat2<R> u = load_mat2<R>(mat, adjoint);
  const uint64_t tb = 1ull << g.t0;
  const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
  for (uint64_t p = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; p < count; p += stride) {
    const uint64_t base = insert_zero_bits_u<4>(p, g.ins, g.nins) | g.cmask;
    if (FORM == FORM_DENSE1 || FORM == FORM_ANTI1 || FORM == FORM_REAL1 || FORM == FORM_RXLIKE1 ||
        FORM == FORM_X1) {
      const C a0 = psi[base], a1 = psi[base | tb];
      C r0, r1;
      if (FORM == FORM_DENSE1) {
        r0 = cfma(u.m01, a1, cmul(u.m00, a0));
        r1 = cfma(u.m11, a1, cmul(u.m10, a0));
      } else if (FORM == FORM_REAL1) {
        r0 = rmix<R>(u.m00.x, a0, u.m01.x, a1);
        r1 = rmix<R>(u.m10.x, a0, u.m11.x, a1);
      } else if (FORM == FORM_RXLIKE1) {
        r0 = ixmix<R>(u.m00.x, a0, u.m01.y, a1);
        r1 = ixmix<R>(u.m11.x, a1, u.m10.y, a0);
      } else if (FORM == FORM_X1) {
        r0 = a1;
        r1 = a0;
      } else {
        r0 = cmul(u.m01, a1);
        r1 = cmul(u.m10, a0);
      }
      psi[base] = r0;
      psi[base | tb] = r1;
    } else if (FORM == FORM_PHASE1) {
      const uint64_t i = base | tb;
      psi[i] = cmul(u.m11, psi[i]);
    } else {  // DIAG1: every amplitude with controls set
      const C a = psi[base];
      psi[base] = cmul((base & tb) ? u.m11 : u.m00, a);
    }
  }
}

template <typename R>
__global__ void __launch_bounds__(256) k_swap2(typename V2<R>::T* __restrict__ psi, uint64_t count, DevGate g) {
  using C = typename V2<R>::T;
  const uint64_t ta = 1ull << g.t0, tb = 1ull << g.t1;
  const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
  for (uint64_t p = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; p < count; p += stride) {
    const uint64_t base = insert_zero_bits_u<4>(p, g.ins, g.nins) | g.cmask;
    const C a = psi[base | ta], b = psi[base | tb];
    psi[base | ta] = b;
    psi[base | tb] = a;
  }
}

template <typename R>
__global__ void __launch_bounds__(256) k_dense2(typename V2<R>::T* __restrict__ psi, uint64_t count, DevGate g,
                                                const double2* __restrict__ mat, bool adjoint) {
  using C = typename V2<R>::T;
  __shared__ C m[16];
  if (threadIdx.x < 16) {
    const int r = threadIdx.x >> 2, c = threadIdx.x & 3;
    double2 v = adjoint ? mat[c * 4 + r] : mat[r * 4 + c];
    if (adjoint) v.y = -v.y;
    m[threadIdx.x] = from_d<R>(v);
  }
  __syncthreads();
  const uint64_t ta = 1ull << g.t0, tb = 1ull << g.t1;
  const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
  for (uint64_t p = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; p < count; p += stride) {
    const uint64_t base = insert_zero_bits_u<4>(p, g.ins, g.nins) | g.cmask;
    const uint64_t idx[4] = {base, base | ta, base | tb, base | ta | tb};
    C a[4];
#pragma unroll
    for (int j = 0; j < 4; ++j) a[j] = psi[idx[j]];
#pragma unroll
    for (int r = 0; r < 4; ++r) {
      C acc = cmul(m[4 * r], a[0]);
#pragma unroll
      for (int j = 1; j < 4; ++j) acc = cfma(m[4 * r + j], a[j], acc);
      psi[idx[r]] = acc;
    }
  }
}

template <typename R>
static cudaError_t launch_gate_t(void* psi_, int n, const DevGate& g, const double2* mat, bool adjoint,
                                 cudaStream_t st) {
  using C = typename V2<R>::T;
  C* psi = (C*)psi_;
  const uint64_t count = 1ull << (n - g.nins);
  const int th = 256, gr = grid_for(count, th);
  switch (g.form) {
    case FORM_DENSE1: k_gate1<R, FORM_DENSE1><<<gr, th, 0, st>>>(psi, count, g, mat, adjoint); break;
    case FORM_ANTI1: k_gate1<R, FORM_ANTI1><<<gr, th, 0, st>>>(psi, count, g, mat, adjoint); break;
    case FORM_REAL1: k_gate1<R, FORM_REAL1><<<gr, th, 0, st>>>(psi, count, g, mat, adjoint); break;
    case FORM_RXLIKE1: k_gate1<R, FORM_RXLIKE1><<<gr, th, 0, st>>>(psi, count, g, mat, adjoint); break;
    case FORM_X1: k_gate1<R, FORM_X1><<<gr, th, 0, st>>>(psi, count, g, mat, adjoint); break;
    case FORM_PHASE1: k_gate1<R, FORM_PHASE1><<<gr, th, 0, st>>>(psi, count, g, mat, adjoint); break;
    case FORM_DIAG1: k_gate1<R, FORM_DIAG1><<<gr, th, 0, st>>>(psi, count, g, mat, adjoint); break;
    case FORM_SWAP2: k_swap2<R><<<gr, th, 0, st>>>(psi, count, g); break;
    case FORM_DENSE2: k_dense2<R><<<gr, th, 0, st>>>(psi, count, g, mat, adjoint); break;
    default: return cudaErrorInvalidValue;
  }
  note_launch();
  return cudaGetLastError();
}

cudaError_t launch_gate(void* psi, int n, qs_dtype dt, const DevGate& g, const double2* mat, bool adjoint,
                        cudaStream_t st) {
  return dt == QS_C64 ? launch_gate_t<float>(psi, n, g, mat, adjoint, st)
                      : launch_gate_t<double>(psi, n, g, mat, adjoint, st);
}

// ---------------------------------------------------------------- staggered multi-gate parallelism

// Section 3.3's two-dimensional block: threadIdx.y selects the member gate,
// threadIdx.x the amplitude pair, and at time step T member j works on
// segment (T + j) mod S (the cyclic timeline of Tab. 3), so the S gates of a
// launch never touch the same amplitudes. S launches apply every member to
// every segment; the members act on distinct qubits and commute, so the
// order in which a segment meets them does not matter. Each launch is one
// sweep of the state (S segments, one gate each).
template <typename R>
__global__ void __launch_bounds__(256) k_smgp_step(typename V2<R>::T* __restrict__ psi, uint64_t count,
                                                   const SmgpDesc* __restrict__ d, int T,
                                                   const double2* __restrict__ gtab) {
  using C = typename V2<R>::T;
  const int j = threadIdx.y;
  const int S = d->S, lg1 = d->lgS + 1;
  const int s = (T + j) & (S - 1);
  const Mat2<R> u = load_mat2<R>(gtab + (int64_t)d->gate[j] * 16, false);
  const int form = d->form[j];
  const uint64_t tb = 1ull << d->t[j], so = d->seg_or[s];
  int32_t pos[4];
#pragma unroll
  for (int k = 0; k < 4; ++k) pos[k] = d->pos[j][k];
  const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
  for (uint64_t p = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; p < count; p += stride) {
    const uint64_t base = insert_zero_bits_u<4>(p, pos, lg1) | so;
    const C a0 = psi[base], a1 = psi[base | tb];
    C r0, r1;
    switch (form) {   // uniform per warp: blockDim.x >= 32
      case FORM_REAL1:
        r0 = rmix<R>(u.m00.x, a0, u.m01.x, a1);
        r1 = rmix<R>(u.m10.x, a0, u.m11.x, a1);
        break;
      case FORM_RXLIKE1:
        r0 = ixmix<R>(u.m00.x, a0, u.m01.y, a1);
        r1 = ixmix<R>(u.m11.x, a1, u.m10.y, a0);
        break;
      case FORM_X1:
        r0 = a1;
        r1 = a0;
        break;
      case FORM_ANTI1:
        r0 = cmul(u.m01, a1);
        r1 = cmul(u.m10, a0);
        break;
      case FORM_PHASE1:
        r0 = a0;
        r1 = cmul(u.m11, a1);
        break;
      case FORM_DIAG1:
        r0 = cmul(u.m00, a0);
        r1 = cmul(u.m11, a1);
        break;
      default:
        r0 = cfma(u.m01, a1, cmul(u.m00, a0));
        r1 = cfma(u.m11, a1, cmul(u.m10, a0));
    }
    psi[base] = r0;
    psi[base | tb] = r1;
  }
}

cudaError_t launch_smgp_step(void* psi, int n, qs_dtype dt, const SmgpDesc* d_desc, const SmgpDesc& h, int T,
                             const double2* gtab, cudaStream_t st) {
  if (h.S < 2 || h.S > kSmgpMax || (1 << h.lgS) != h.S || n < h.S + h.lgS) return cudaErrorInvalidValue;
  const uint64_t count = 1ull << (n - h.lgS - 1);   // pairs per segment
  const dim3 block(256 / h.S, h.S);
  const int gr = grid_for(count, 256 / h.S);
  if (dt == QS_C64) k_smgp_step<float><<<gr, block, 0, st>>>((float2*)psi, count, d_desc, T, gtab);
  else k_smgp_step<double><<<gr, block, 0, st>>>((double2*)psi, count, d_desc, T, gtab);
  note_launch();
  return cudaGetLastError();
}

}  // namespace qs
