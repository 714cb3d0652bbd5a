// row_f64_small.cu -- double row-stage kernels for Nt = 64, 128, 256
// (see row_kernel.cuh); split by Nt so the build compiles them in parallel.
#include "row_kernel.cuh"

namespace fcn {
namespace rowimpl {
template cudaError_t launch_nt<double, 64>(const RowArgs<double> &, cudaStream_t);
template cudaError_t launch_nt_multi<double, 64>(const RowMultiArgs<double> &, int, cudaStream_t);
template cudaError_t prepare_nt<double, 64>();
template cudaError_t launch_nt<double, 128>(const RowArgs<double> &, cudaStream_t);
template cudaError_t launch_nt_multi<double, 128>(const RowMultiArgs<double> &, int, cudaStream_t);
template cudaError_t prepare_nt<double, 128>();
template cudaError_t launch_nt<double, 256>(const RowArgs<double> &, cudaStream_t);
template cudaError_t launch_nt_multi<double, 256>(const RowMultiArgs<double> &, int, cudaStream_t);
template cudaError_t prepare_nt<double, 256>();
}  // namespace rowimpl
}  // namespace fcn
