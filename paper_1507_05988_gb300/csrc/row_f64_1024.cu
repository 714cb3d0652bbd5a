// row_f64_1024.cu -- double row-stage kernels for Nt = 1024
// (see row_kernel.cuh); split by Nt so the build compiles them in parallel.
#include "row_kernel.cuh"

namespace fcn {
namespace rowimpl {
template cudaError_t launch_nt<double, 1024>(const RowArgs<double> &, cudaStream_t);
template cudaError_t launch_nt_multi<double, 1024>(const RowMultiArgs<double> &, int, cudaStream_t);
template cudaError_t prepare_nt<double, 1024>();
}  // namespace rowimpl
}  // namespace fcn
