// row_f32_1024.cu -- float row-stage kernels for Nt = 1024
// (see row_kernel.cuh); split by Nt so the build compiles them in parallel.
#include "row_kernel.cuh"

namespace fcn {
namespace rowimpl {
template cudaError_t launch_nt<float, 1024>(const RowArgs<float> &, cudaStream_t);
template cudaError_t launch_nt_multi<float, 1024>(const RowMultiArgs<float> &, int, cudaStream_t);
template cudaError_t prepare_nt<float, 1024>();
}  // namespace rowimpl
}  // namespace fcn
