// row_batch.cu -- the batched (work-list) row stage: pulses of uneven grids
// (Nt = 512 ... 8192) in one persistent launch per stage.  FP32 with K = 8,
// the form the batched path runs in (see row_kernel.cuh for the row body).
#include "row_kernel.cuh"

namespace fcn {

size_t row_batch_smem(int nt, int bytes_per_complex) {
    // 512 threads hold 512 / (Nt/16) rows of Nt + Nt/16 padded values and
    // as many real u values
    const int tpr = nt / 16;
    const int rpc = 512 / tpr;
    return (size_t)(bytes_per_complex + bytes_per_complex / 2) * rpc * (nt + nt / 16) + sizeof(double) * kRowScratch;
}

template <>
cudaError_t prepare_rows_batch<float>(size_t smem) {
    return cudaFuncSetAttribute(row_batch_kernel<float, 8>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)smem);
}

template <>
cudaError_t launch_rows_batch<float>(const RowArgs<float> *pulses, const int2 *items, int nitems, int ops,
                                     unsigned *counter, size_t smem, int grid, cudaStream_t st) {
    row_batch_kernel<float, 8><<<grid, 512, smem, st>>>(pulses, items, nitems, ops, counter);
    return cudaGetLastError();
}

}  // namespace fcn
