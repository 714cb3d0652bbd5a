// row_f64_4096.cu -- double row-stage kernels for Nt = 4096
// (see row_kernel.cuh); split by Nt so the build compiles them in parallel.
#include "row_kernel.cuh"

namespace fcn {
namespace rowimpl {
template cudaError_t launch_nt<double, 4096>(const RowArgs<double> &, cudaStream_t);
template cudaError_t launch_nt_multi<double, 4096>(const RowMultiArgs<double> &, int, cudaStream_t);
template cudaError_t prepare_nt<double, 4096>();
}  // namespace rowimpl
}  // namespace fcn
