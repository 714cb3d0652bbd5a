// row_f32.cu -- float instantiation of the row stage (row_kernel.cuh); one
// translation unit per precision so the two compile in parallel.
#include "row_kernel.cuh"

namespace fcn {
template cudaError_t launch_rows<float>(const RowArgs<float> &, int, cudaStream_t);
template cudaError_t prepare_rows<float>(int);
}  // namespace fcn
