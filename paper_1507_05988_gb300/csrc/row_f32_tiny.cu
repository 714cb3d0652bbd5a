// row_f32_tiny.cu -- float row-stage kernels for Nt = 2, 4, 8, 16, 32
// (see row_kernel.cuh); split by Nt so the build compiles them in parallel.
#include "row_kernel.cuh"

namespace fcn {
namespace rowimpl {
template cudaError_t launch_nt<float, 2>(const RowArgs<float> &, cudaStream_t);
template cudaError_t launch_nt_multi<float, 2>(const RowMultiArgs<float> &, int, cudaStream_t);
template cudaError_t prepare_nt<float, 2>();
template cudaError_t launch_nt<float, 4>(const RowArgs<float> &, cudaStream_t);
template cudaError_t launch_nt_multi<float, 4>(const RowMultiArgs<float> &, int, cudaStream_t);
template cudaError_t prepare_nt<float, 4>();
template cudaError_t launch_nt<float, 8>(const RowArgs<float> &, cudaStream_t);
template cudaError_t launch_nt_multi<float, 8>(const RowMultiArgs<float> &, int, cudaStream_t);
template cudaError_t prepare_nt<float, 8>();
template cudaError_t launch_nt<float, 16>(const RowArgs<float> &, cudaStream_t);
template cudaError_t launch_nt_multi<float, 16>(const RowMultiArgs<float> &, int, cudaStream_t);
template cudaError_t prepare_nt<float, 16>();
template cudaError_t launch_nt<float, 32>(const RowArgs<float> &, cudaStream_t);
template cudaError_t launch_nt_multi<float, 32>(const RowMultiArgs<float> &, int, cudaStream_t);
template cudaError_t prepare_nt<float, 32>();
}  // namespace rowimpl
}  // namespace fcn
