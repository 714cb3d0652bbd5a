// row_dispatch.cu -- run-time dispatch of the row stage on Nt.  The kernels
// themselves are instantiated in row_<precision>_<Nt>.cu (one translation
// unit per precision and Nt group, so that they compile in parallel).
#include "row_kernel.cuh"

namespace fcn {
namespace rowimpl {
extern template cudaError_t launch_nt<float, 2>(const RowArgs<float> &, cudaStream_t);
extern template cudaError_t launch_nt_multi<float, 2>(const RowMultiArgs<float> &, int, cudaStream_t);
extern template cudaError_t prepare_nt<float, 2>();
extern template cudaError_t launch_nt<float, 4>(const RowArgs<float> &, cudaStream_t);
extern template cudaError_t launch_nt_multi<float, 4>(const RowMultiArgs<float> &, int, cudaStream_t);
extern template cudaError_t prepare_nt<float, 4>();
extern template cudaError_t launch_nt<float, 8>(const RowArgs<float> &, cudaStream_t);
extern template cudaError_t launch_nt_multi<float, 8>(const RowMultiArgs<float> &, int, cudaStream_t);
extern template cudaError_t prepare_nt<float, 8>();
extern template cudaError_t launch_nt<float, 16>(const RowArgs<float> &, cudaStream_t);
extern template cudaError_t launch_nt_multi<float, 16>(const RowMultiArgs<float> &, int, cudaStream_t);
extern template cudaError_t prepare_nt<float, 16>();
extern template cudaError_t launch_nt<float, 32>(const RowArgs<float> &, cudaStream_t);
extern template cudaError_t launch_nt_multi<float, 32>(const RowMultiArgs<float> &, int, cudaStream_t);
extern template cudaError_t prepare_nt<float, 32>();
extern template cudaError_t launch_nt<float, 64>(const RowArgs<float> &, cudaStream_t);
extern template cudaError_t launch_nt_multi<float, 64>(const RowMultiArgs<float> &, int, cudaStream_t);
extern template cudaError_t prepare_nt<float, 64>();
extern template cudaError_t launch_nt<float, 128>(const RowArgs<float> &, cudaStream_t);
extern template cudaError_t launch_nt_multi<float, 128>(const RowMultiArgs<float> &, int, cudaStream_t);
extern template cudaError_t prepare_nt<float, 128>();
extern template cudaError_t launch_nt<float, 256>(const RowArgs<float> &, cudaStream_t);
extern template cudaError_t launch_nt_multi<float, 256>(const RowMultiArgs<float> &, int, cudaStream_t);
extern template cudaError_t prepare_nt<float, 256>();
extern template cudaError_t launch_nt<float, 512>(const RowArgs<float> &, cudaStream_t);
extern template cudaError_t launch_nt_multi<float, 512>(const RowMultiArgs<float> &, int, cudaStream_t);
extern template cudaError_t prepare_nt<float, 512>();
extern template cudaError_t launch_nt<float, 1024>(const RowArgs<float> &, cudaStream_t);
extern template cudaError_t launch_nt_multi<float, 1024>(const RowMultiArgs<float> &, int, cudaStream_t);
extern template cudaError_t prepare_nt<float, 1024>();
extern template cudaError_t launch_nt<float, 2048>(const RowArgs<float> &, cudaStream_t);
extern template cudaError_t launch_nt_multi<float, 2048>(const RowMultiArgs<float> &, int, cudaStream_t);
extern template cudaError_t prepare_nt<float, 2048>();
extern template cudaError_t launch_nt<float, 4096>(const RowArgs<float> &, cudaStream_t);
extern template cudaError_t launch_nt_multi<float, 4096>(const RowMultiArgs<float> &, int, cudaStream_t);
extern template cudaError_t prepare_nt<float, 4096>();
extern template cudaError_t launch_nt<float, 8192>(const RowArgs<float> &, cudaStream_t);
extern template cudaError_t launch_nt_multi<float, 8192>(const RowMultiArgs<float> &, int, cudaStream_t);
extern template cudaError_t prepare_nt<float, 8192>();
extern template cudaError_t launch_nt<double, 2>(const RowArgs<double> &, cudaStream_t);
extern template cudaError_t launch_nt_multi<double, 2>(const RowMultiArgs<double> &, int, cudaStream_t);
extern template cudaError_t prepare_nt<double, 2>();
extern template cudaError_t launch_nt<double, 4>(const RowArgs<double> &, cudaStream_t);
extern template cudaError_t launch_nt_multi<double, 4>(const RowMultiArgs<double> &, int, cudaStream_t);
extern template cudaError_t prepare_nt<double, 4>();
extern template cudaError_t launch_nt<double, 8>(const RowArgs<double> &, cudaStream_t);
extern template cudaError_t launch_nt_multi<double, 8>(const RowMultiArgs<double> &, int, cudaStream_t);
extern template cudaError_t prepare_nt<double, 8>();
extern template cudaError_t launch_nt<double, 16>(const RowArgs<double> &, cudaStream_t);
extern template cudaError_t launch_nt_multi<double, 16>(const RowMultiArgs<double> &, int, cudaStream_t);
extern template cudaError_t prepare_nt<double, 16>();
extern template cudaError_t launch_nt<double, 32>(const RowArgs<double> &, cudaStream_t);
extern template cudaError_t launch_nt_multi<double, 32>(const RowMultiArgs<double> &, int, cudaStream_t);
extern template cudaError_t prepare_nt<double, 32>();
extern template cudaError_t launch_nt<double, 64>(const RowArgs<double> &, cudaStream_t);
extern template cudaError_t launch_nt_multi<double, 64>(const RowMultiArgs<double> &, int, cudaStream_t);
extern template cudaError_t prepare_nt<double, 64>();
extern template cudaError_t launch_nt<double, 128>(const RowArgs<double> &, cudaStream_t);
extern template cudaError_t launch_nt_multi<double, 128>(const RowMultiArgs<double> &, int, cudaStream_t);
extern template cudaError_t prepare_nt<double, 128>();
extern template cudaError_t launch_nt<double, 256>(const RowArgs<double> &, cudaStream_t);
extern template cudaError_t launch_nt_multi<double, 256>(const RowMultiArgs<double> &, int, cudaStream_t);
extern template cudaError_t prepare_nt<double, 256>();
extern template cudaError_t launch_nt<double, 512>(const RowArgs<double> &, cudaStream_t);
extern template cudaError_t launch_nt_multi<double, 512>(const RowMultiArgs<double> &, int, cudaStream_t);
extern template cudaError_t prepare_nt<double, 512>();
extern template cudaError_t launch_nt<double, 1024>(const RowArgs<double> &, cudaStream_t);
extern template cudaError_t launch_nt_multi<double, 1024>(const RowMultiArgs<double> &, int, cudaStream_t);
extern template cudaError_t prepare_nt<double, 1024>();
extern template cudaError_t launch_nt<double, 2048>(const RowArgs<double> &, cudaStream_t);
extern template cudaError_t launch_nt_multi<double, 2048>(const RowMultiArgs<double> &, int, cudaStream_t);
extern template cudaError_t prepare_nt<double, 2048>();
extern template cudaError_t launch_nt<double, 4096>(const RowArgs<double> &, cudaStream_t);
extern template cudaError_t launch_nt_multi<double, 4096>(const RowMultiArgs<double> &, int, cudaStream_t);
extern template cudaError_t prepare_nt<double, 4096>();
extern template cudaError_t launch_nt<double, 8192>(const RowArgs<double> &, cudaStream_t);
extern template cudaError_t launch_nt_multi<double, 8192>(const RowMultiArgs<double> &, int, cudaStream_t);
extern template cudaError_t prepare_nt<double, 8192>();
}  // namespace rowimpl

template <typename T>
cudaError_t prepare_rows(int nt) {
    switch (nt) {
        case 2: return rowimpl::prepare_nt<T, 2>();
        case 4: return rowimpl::prepare_nt<T, 4>();
        case 8: return rowimpl::prepare_nt<T, 8>();
        case 16: return rowimpl::prepare_nt<T, 16>();
        case 32: return rowimpl::prepare_nt<T, 32>();
        case 64: return rowimpl::prepare_nt<T, 64>();
        case 128: return rowimpl::prepare_nt<T, 128>();
        case 256: return rowimpl::prepare_nt<T, 256>();
        case 512: return rowimpl::prepare_nt<T, 512>();
        case 1024: return rowimpl::prepare_nt<T, 1024>();
        case 2048: return rowimpl::prepare_nt<T, 2048>();
        case 4096: return rowimpl::prepare_nt<T, 4096>();
        case 8192: return rowimpl::prepare_nt<T, 8192>();
        default: return cudaErrorInvalidValue;
    }
}

// Dispatch on Nt (one compiled kernel per power of two).
template <typename T>
cudaError_t launch_rows(const RowArgs<T> &a, int nt, cudaStream_t st) {
    switch (nt) {
        case 2: return rowimpl::launch_nt<T, 2>(a, st);
        case 4: return rowimpl::launch_nt<T, 4>(a, st);
        case 8: return rowimpl::launch_nt<T, 8>(a, st);
        case 16: return rowimpl::launch_nt<T, 16>(a, st);
        case 32: return rowimpl::launch_nt<T, 32>(a, st);
        case 64: return rowimpl::launch_nt<T, 64>(a, st);
        case 128: return rowimpl::launch_nt<T, 128>(a, st);
        case 256: return rowimpl::launch_nt<T, 256>(a, st);
        case 512: return rowimpl::launch_nt<T, 512>(a, st);
        case 1024: return rowimpl::launch_nt<T, 1024>(a, st);
        case 2048: return rowimpl::launch_nt<T, 2048>(a, st);
        case 4096: return rowimpl::launch_nt<T, 4096>(a, st);
        case 8192: return rowimpl::launch_nt<T, 8192>(a, st);
        default: return cudaErrorInvalidValue;
    }
}

// The same for several pulses of one grid (RowMultiArgs, npulse <= kRowMulti).
template <typename T>
cudaError_t launch_rows_multi(const RowMultiArgs<T> &m, int npulse, int nt, cudaStream_t st) {
    switch (nt) {
        case 2: return rowimpl::launch_nt_multi<T, 2>(m, npulse, st);
        case 4: return rowimpl::launch_nt_multi<T, 4>(m, npulse, st);
        case 8: return rowimpl::launch_nt_multi<T, 8>(m, npulse, st);
        case 16: return rowimpl::launch_nt_multi<T, 16>(m, npulse, st);
        case 32: return rowimpl::launch_nt_multi<T, 32>(m, npulse, st);
        case 64: return rowimpl::launch_nt_multi<T, 64>(m, npulse, st);
        case 128: return rowimpl::launch_nt_multi<T, 128>(m, npulse, st);
        case 256: return rowimpl::launch_nt_multi<T, 256>(m, npulse, st);
        case 512: return rowimpl::launch_nt_multi<T, 512>(m, npulse, st);
        case 1024: return rowimpl::launch_nt_multi<T, 1024>(m, npulse, st);
        case 2048: return rowimpl::launch_nt_multi<T, 2048>(m, npulse, st);
        case 4096: return rowimpl::launch_nt_multi<T, 4096>(m, npulse, st);
        case 8192: return rowimpl::launch_nt_multi<T, 8192>(m, npulse, st);
        default: return cudaErrorInvalidValue;
    }
}

template cudaError_t launch_rows<float>(const RowArgs<float> &, int, cudaStream_t);
template cudaError_t launch_rows_multi<float>(const RowMultiArgs<float> &, int, int, cudaStream_t);
template cudaError_t launch_rows_multi<double>(const RowMultiArgs<double> &, int, int, cudaStream_t);
template cudaError_t launch_rows<double>(const RowArgs<double> &, int, cudaStream_t);
template cudaError_t prepare_rows<float>(int);
template cudaError_t prepare_rows<double>(int);

}  // namespace fcn
