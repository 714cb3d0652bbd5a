// row_f32_small.cu -- float row-stage kernels for Nt = 64, 128, 256
// (see row_kernel.cuh); split by Nt so the build compiles them in parallel.
#include "row_kernel.cuh"

namespace fcn {
namespace rowimpl {
template cudaError_t launch_nt<float, 64>(const RowArgs<float> &, cudaStream_t);
template cudaError_t launch_nt_multi<float, 64>(const RowMultiArgs<float> &, int, cudaStream_t);
template cudaError_t prepare_nt<float, 64>();
template cudaError_t launch_nt<float, 128>(const RowArgs<float> &, cudaStream_t);
template cudaError_t launch_nt_multi<float, 128>(const RowMultiArgs<float> &, int, cudaStream_t);
template cudaError_t prepare_nt<float, 128>();
template cudaError_t launch_nt<float, 256>(const RowArgs<float> &, cudaStream_t);
template cudaError_t launch_nt_multi<float, 256>(const RowMultiArgs<float> &, int, cudaStream_t);
template cudaError_t prepare_nt<float, 256>();
}  // namespace rowimpl
}  // namespace fcn
