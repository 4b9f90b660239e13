// Column pass instantiations and kernel preparation, float.
#include "kernels.cuh"

namespace sbi {
template <> cudaError_t launch_col<float>(int ny, const ColParams& p, cudaStream_t st) {
  return launch_col_impl<float>(ny, p, st);
}
template <> cudaError_t prepare_col_kernels<float>(int ny) { return prepare_col_impl<float>(ny); }
template <> int col_geometry<float>(int ny, int* tpc) { return col_geometry_impl<float>(ny, tpc); }
template <> bool col_stageable<float>(int ny) { return col_stageable_impl<float>(ny); }
template <> cudaError_t launch_coef_table<float>(void* out, const TableSpec& s, cudaStream_t st) {
  return launch_coef_table_impl<float>(out, s, st);
}
}  // namespace sbi
