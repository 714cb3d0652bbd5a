// row_f64_tiny.cu -- double row-stage kernels for Nt = 2, 4, 8, 16, 32
// (see row_kernel.cuh); split by Nt so the build compiles them in parallel.
#include "row_kernel.cuh"

namespace fcn {
namespace rowimpl {
template cudaError_t launch_nt<double, 2>(const RowArgs<double> &, cudaStream_t);
template cudaError_t launch_nt_multi<double, 2>(const RowMultiArgs<double> &, int, cudaStream_t);
template cudaError_t prepare_nt<double, 2>();
template cudaError_t launch_nt<double, 4>(const RowArgs<double> &, cudaStream_t);
template cudaError_t launch_nt_multi<double, 4>(const RowMultiArgs<double> &, int, cudaStream_t);
template cudaError_t prepare_nt<double, 4>();
template cudaError_t launch_nt<double, 8>(const RowArgs<double> &, cudaStream_t);
template cudaError_t launch_nt_multi<double, 8>(const RowMultiArgs<double> &, int, cudaStream_t);
template cudaError_t prepare_nt<double, 8>();
template cudaError_t launch_nt<double, 16>(const RowArgs<double> &, cudaStream_t);
template cudaError_t launch_nt_multi<double, 16>(const RowMultiArgs<double> &, int, cudaStream_t);
template cudaError_t prepare_nt<double, 16>();
template cudaError_t launch_nt<double, 32>(const RowArgs<double> &, cudaStream_t);
template cudaError_t launch_nt_multi<double, 32>(const RowMultiArgs<double> &, int, cudaStream_t);
template cudaError_t prepare_nt<double, 32>();
}  // namespace rowimpl
}  // namespace fcn
