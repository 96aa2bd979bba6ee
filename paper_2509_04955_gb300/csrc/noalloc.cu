// Pauli-sum expectation value that allocates no device memory.
//
// Some callers cannot call cudaMalloc while they evaluate an observable: a
// host application that hands this library a fixed slice of device memory
// and forbids any other allocation (an embedded solver, a real-time control
// loop, an inference server with a pre-reserved memory budget), or code that
// runs where allocation is not allowed or would stall the device (inside
// another framework's caching allocator, between the steps of a hot loop).
// For them, qs_expval_pauli_sum_noalloc works on a state given as a raw
// device pointer and keeps every temporary in one fixed array compiled into
// the library: g_noalloc_scratch below, NOALLOC_SCRATCH_BYTES (80 KiB)
// of device memory that every GPU loading the library holds until the process
// exits. The kernels it launches are the same ones qs_expval_pauli_sum uses.
#include <cuda_runtime.h>

#include <algorithm>
#include <string>   // error messages only

#include "qs_internal.h"

namespace qs {
void set_last_error(const std::string& msg);
int reduce_blocks();
}  // namespace qs

using namespace qs;

namespace {

constexpr int kNoAllocMaxTerms = 1024;      // largest Pauli sum accepted
constexpr int kNoAllocZPerLaunch = kExpvalMaxZ;   // strings per expectation launch (the kernel's limit)
constexpr int kNoAllocPartialRows = kNoAllocZPerLaunch;   // rows of per-CTA partial sums per launch
constexpr int kNoAllocPartialCols = 1024;   // >= the reduction grid
static_assert(kNoAllocZPerLaunch == 8, "scratch layout sized for 8 strings per expectation launch");
constexpr size_t kPartialBytes = sizeof(double) * kNoAllocPartialRows * kNoAllocPartialCols;
constexpr size_t kOutBytes = sizeof(double) * kNoAllocMaxTerms;
constexpr size_t kZBytes = sizeof(uint64_t) * kNoAllocMaxTerms;
constexpr size_t NOALLOC_SCRATCH_BYTES = kPartialBytes + kOutBytes + kZBytes;

// Layout: [partials: 8 x 1024 doubles][per-string results: 1024 doubles][z masks: 1024 uint64].
// Every launch writes each slot it later reads, so nothing needs clearing
// between calls; stale contents from an earlier call are never read.
static __device__ __align__(256) unsigned char g_noalloc_scratch[NOALLOC_SCRATCH_BYTES];

// Device address of the scratch array in the current CUDA context. In host
// code g_noalloc_scratch names a host-side stand-in, never the device array,
// so the address is asked for on every call: the module holding the array is
// loaded per context, and a cached address would go stale after
// cudaDeviceReset or when the caller makes another context current. The
// lookup is cheap once the module is loaded in that context.
cudaError_t scratch_address(void** out) {
  void* p = nullptr;
  const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
  if (e != cudaSuccess) return e;
  *out = p;
  return cudaSuccess;
}

qs_status fail(qs_status code, const std::string& msg) {
  set_last_error(msg);
  return code;
}

}  // namespace

extern "C" qs_status qs_expval_pauli_sum_noalloc(const void* dev_state, int n, qs_dtype dtype, void* stream,
                                                 const qs_pauli_term* terms, size_t nterms, double* out) {
  if (out == nullptr) return fail(QS_ERR_ARG, "out is NULL");
  if (dev_state == nullptr || ((uintptr_t)dev_state & 15) != 0)
    return fail(QS_ERR_ARG, "state pointer must be a 16-byte aligned device pointer");
  if (n < 1 || n > kMaxQubits) return fail(QS_ERR_ARG, "n out of range (1..40)");
  if (dtype != QS_C64 && dtype != QS_C128) return fail(QS_ERR_ARG, "bad dtype");
  if (nterms > (size_t)kNoAllocMaxTerms)
    return fail(QS_ERR_ARG, "nterms exceeds the 1024-term limit of qs_expval_pauli_sum_noalloc");
  if (nterms > 0 && terms == nullptr) return fail(QS_ERR_ARG, "terms is NULL");
  if (reduce_blocks() > kNoAllocPartialCols) return fail(QS_ERR_UNSUPPORTED, "reduction grid larger than scratch");
  const uint64_t valid = (1ull << n) - 1;
  for (size_t j = 0; j < nterms; ++j)
    if ((terms[j].xmask | terms[j].zmask) & ~valid) return fail(QS_ERR_ARG, "Pauli term acts on a qubit >= n");
  if (nterms == 0) {
    *out = 0.0;
    return QS_OK;
  }
  void* base = nullptr;
  cudaError_t e = scratch_address(&base);
  if (e != cudaSuccess) return fail(QS_ERR_CUDA, std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(e));
  double* d_part = (double*)base;
  double* d_out = (double*)((unsigned char*)base + kPartialBytes);
  uint64_t* d_z = (uint64_t*)((unsigned char*)base + kPartialBytes + kOutBytes);
  cudaStream_t st = (cudaStream_t)stream;

  // Strings sorted by (x mask, index) in stack arrays (std::sort works in
  // place): strings sharing x share a sweep.
  int order[kNoAllocMaxTerms];
  uint64_t zl[kNoAllocMaxTerms];
  double vals[kNoAllocMaxTerms];
  for (size_t j = 0; j < nterms; ++j) order[j] = (int)j;
  std::sort(order, order + nterms, [&](int a, int b) {
    return terms[a].xmask != terms[b].xmask ? terms[a].xmask < terms[b].xmask : a < b;
  });
  for (size_t j = 0; j < nterms; ++j) zl[j] = terms[order[j]].zmask;
  e = cudaMemcpyAsync(d_z, zl, sizeof(uint64_t) * nterms, cudaMemcpyHostToDevice, st);
  if (e != cudaSuccess) return fail(QS_ERR_CUDA, std::string("cudaMemcpyAsync: ") + cudaGetErrorString(e));
  size_t j = 0;
  while (j < nterms) {
    const uint64_t x = terms[order[j]].xmask;
    size_t end = j;
    while (end < nterms && end - j < (size_t)kNoAllocZPerLaunch && terms[order[end]].xmask == x) ++end;
    e = launch_expval_x(dev_state, n, dtype, x, d_z + j, nullptr, (int)(end - j), d_part, d_out + j, st);
    if (e != cudaSuccess) return fail(QS_ERR_CUDA, std::string("expectation launch: ") + cudaGetErrorString(e));
    j = end;
  }
  e = cudaMemcpyAsync(vals, d_out, sizeof(double) * nterms, cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return fail(QS_ERR_CUDA, std::string("result copy: ") + cudaGetErrorString(e));
  double total = 0;
  for (size_t k = 0; k < nterms; ++k) {
    const qs_pauli_term& t = terms[order[k]];
    total += t.coeff * rt::term_factor(t) * vals[k];
  }
  *out = total;
  return QS_OK;
}
