// Column pass instantiations and kernel preparation, double.
#include "kernels.cuh"

namespace sbi {
template <> cudaError_t launch_col<double>(int ny, const ColParams& p, cudaStream_t st) {
  return launch_col_impl<double>(ny, p, st);
}
template <> cudaError_t prepare_col_kernels<double>(int ny) { return prepare_col_impl<double>(ny); }
}  // namespace sbi
