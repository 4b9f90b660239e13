// Row and RK4 pass instantiations, float.
#include "kernels.cuh"

namespace sbi {
template <> cudaError_t launch_row<float>(int nx, const RowParams& p, cudaStream_t st) {
  return launch_row_impl<float>(nx, p, st);
}
template <> cudaError_t launch_rk<float>(int nx, const RkParams& p, cudaStream_t st) {
  return launch_rk_impl<float>(nx, p, st);
}
template <> cudaError_t prepare_row_kernels<float>(int nx) { return prepare_row_impl<float>(nx); }
template <> int row_rpc<float>(int nx, int W, int nslots) { return row_rpc_impl<float>(nx, W, nslots); }
template <> int row_tpr<float>(int nx) { return row_tpr_impl<float>(nx); }
template <> cudaError_t state_convert<float>(const void* src, void* dst, long long n, bool to_double,
                                          cudaStream_t st) {
  return state_convert_impl<float>(src, dst, n, to_double, st);
}
}  // namespace sbi
