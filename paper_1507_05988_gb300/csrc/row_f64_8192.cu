// row_f64_8192.cu -- double row-stage kernels for Nt = 8192
// (see row_kernel.cuh); split by Nt so the build compiles them in parallel.
#include "row_kernel.cuh"

namespace fcn {
namespace rowimpl {
template cudaError_t launch_nt<double, 8192>(const RowArgs<double> &, cudaStream_t);
template cudaError_t launch_nt_multi<double, 8192>(const RowMultiArgs<double> &, int, cudaStream_t);
template cudaError_t prepare_nt<double, 8192>();
}  // namespace rowimpl
}  // namespace fcn
