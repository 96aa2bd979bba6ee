// Tile-pass kernels for complex128 (FP64), blocks of up to 5 qubits: instances of kernels_tile.cuh (the
// dispatcher is in kernels_tile.cu).
#include "kernels_tile.cuh"

namespace qs {

cudaError_t launch_tile_f64(int kmax, void* psi, void* const* psis, int nstates, int64_t gstride, int64_t bstride,
                          int64_t brow0, int n, const PassDesc& p, const DevOp* ops, const double2* gtab,
                          const double2* btab, cudaStream_t st, size_t smem) {
  return launch_tile_range<double, 2, 5>(kmax, psi, psis, nstates, gstride, bstride, brow0, n, p, ops, gtab, btab, st, smem);
}

cudaError_t prepare_tile_f64(int kmax, bool bulk, size_t smem) {
  return prepare_tile_range<double, 2, 5>(kmax, bulk, smem);
}

}  // namespace qs
