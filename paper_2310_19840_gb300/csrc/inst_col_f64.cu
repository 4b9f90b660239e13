// Column pass instantiations and kernel preparation, double.
#include "kernels.cuh"

namespace sbi {
template <> cudaError_t launch_col<double>(int ny, const ColParams& p, cudaStream_t st) {
  return launch_col_impl<double>(ny, p, st);
}
template <> cudaError_t prepare_col_kernels<double>(int ny) { return prepare_col_impl<double>(ny); }
template <> int col_geometry<double>(int ny, int* tpc) { return col_geometry_impl<double>(ny, tpc); }
template <> bool col_stageable<double>(int ny) { return col_stageable_impl<double>(ny); }
template <> cudaError_t launch_coef_table<double>(void* out, const TableSpec& s, cudaStream_t st) {
  return launch_coef_table_impl<double>(out, s, st);
}
}  // namespace sbi
