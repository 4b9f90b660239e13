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
template <> int row_rpc<double>(int nx, int W, int nslots) { return row_rpc_impl<double>(nx, W, nslots); }
template <> int row_tpr<double>(int nx) { return row_tpr_impl<double>(nx); }
template <> cudaError_t state_convert<double>(const void* src, void* dst, long long n, bool to_double,
                                          cudaStream_t st) {
  return state_convert_impl<double>(src, dst, n, to_double, st);
}
}  // namespace sbi
