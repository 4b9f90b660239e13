// Row and RK4 pass instantiations, double.
#include "kernels.cuh"

namespace sbi {
template <> cudaError_t launch_row<double>(int nx, const RowParams& p, cudaStream_t st) {
  return launch_row_impl<double>(nx, p, st);
}
template <> cudaError_t launch_rk<double>(int nx, const RkParams& p, cudaStream_t st) {
  return launch_rk_impl<double>(nx, p, st);
}
template <> cudaError_t prepare_row_kernels<double>(int nx) { return prepare_row_impl<double>(nx); }
template <> size_t row_smem_bytes<double>(int nx, int nslots) {
  return row_smem_impl<double>(nx, nslots);
}
}  // namespace sbi
