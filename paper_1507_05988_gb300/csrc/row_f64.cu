// row_f64.cu -- double instantiation of the row stage (row_kernel.cuh); one
// translation unit per precision so the two compile in parallel.
#include "row_kernel.cuh"

namespace fcn {
template cudaError_t launch_rows<double>(const RowArgs<double> &, int, cudaStream_t);
template cudaError_t prepare_rows<double>(int);
}  // namespace fcn
