// reduce.cu -- FP64 reductions (diagnostics, step-doubling error norm, power
// and fluence profiles) and precision conversions of the FCN library.
// All reductions use fixed trees without atomics, so repeated runs give
// bit-identical results.
#include "fcn_device.cuh"

namespace fcn {
namespace {

constexpr int RT = 256;   // threads of the reduction CTAs


template <typename T>
__global__ void widen_kernel(const cx<T> *src, double *dst, int64_t n) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        const cx<T> v = src[i];
        reinterpret_cast<double2 *>(dst)[i] = make_double2(double(v.x), double(v.y));
    }
}

template <typename T>
__global__ void narrow_kernel(const double *src, cx<T> *dst, int64_t n) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        const double2 v = reinterpret_cast<const double2 *>(src)[i];
        dst[i] = mk(T(v.x), T(v.y));
    }
}

template <typename T>
__global__ void widen_real_kernel(const T *src, double *dst, int64_t n) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x)
        dst[i] = double(src[i]);
}

// out: [energy_sum, max I, max u, onaxis max I, S0, S1, S2, nonfinite];
// FLAT: every row weighs 1 (Cartesian grid) and the on-axis row is axis_row.
template <bool FLAT>
__global__ void reduce_stats_kernel(const double *st, int nr, int axis_row, double *out) {
    __shared__ double sh[32];
    double e = 0, mi = 0, mu = 0, s0 = 0, s1 = 0, s2 = 0, bad = 0;
    for (int m = threadIdx.x; m < nr; m += blockDim.x) {
        const double *r = st + (size_t)m * NSTAT;
        const double w = FLAT ? 1.0 : radial_weight(m);
        e += w * r[ST_SUM_I];
        mi = fmax(mi, r[ST_MAX_I]);
        mu = fmax(mu, r[ST_MAX_U]);
        s0 += w * r[ST_S0];
        s1 += w * r[ST_S1];
        s2 += w * r[ST_S2];
        bad += r[ST_NONFINITE];
        if (!isfinite(r[ST_SUM_I])) bad += 1.0;
    }
    e = block_sum(e, sh);
    if (threadIdx.x == 0) out[0] = e;
    mi = block_max(mi, sh);
    if (threadIdx.x == 0) out[1] = mi;
    mu = block_max(mu, sh);
    if (threadIdx.x == 0) out[2] = mu;
    if (threadIdx.x == 0) out[3] = st[(size_t)axis_row * NSTAT + ST_MAX_I];
    s0 = block_sum(s0, sh);
    if (threadIdx.x == 0) out[4] = s0;
    s1 = block_sum(s1, sh);
    if (threadIdx.x == 0) out[5] = s1;
    s2 = block_sum(s2, sh);
    if (threadIdx.x == 0) out[6] = s2;
    bad = block_sum(bad, sh);
    if (threadIdx.x == 0) out[7] = bad;
}

__global__ void diff_final_kernel(const double *rows, int nr, double *out) {
    __shared__ double sh[32];
    double d2 = 0.0, b2 = 0.0;
    for (int m = threadIdx.x; m < nr; m += blockDim.x) {
        d2 += rows[2 * m];
        b2 += rows[2 * m + 1];
    }
    d2 = block_sum(d2, sh);
    if (threadIdx.x == 0) out[0] = d2;
    b2 = block_sum(b2, sh);
    if (threadIdx.x == 0) out[1] = b2;
}

// power[p] = sum_m W_m |A_mp|^2 (one thread per p, coalesced over p)
template <typename T>
__global__ void power_kernel(const cx<T> *f, int nr, int nt, double *power) {
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= nt) return;
    double s = 0.0;
    for (int m = 0; m < nr; ++m) {
        const cx<T> v = f[(size_t)m * nt + p];
        s += radial_weight(m) * (double(v.x) * double(v.x) + double(v.y) * double(v.y));
    }
    power[p] = s;
}

template <typename T>
__global__ void rowsum_kernel(const cx<T> *f, int nt, double *rowsum) {
    __shared__ double sh[32];
    const int m = blockIdx.x;
    double s = 0.0;
    for (int p = threadIdx.x; p < nt; p += blockDim.x) {
        const cx<T> v = f[(size_t)m * nt + p];
        s += double(v.x) * double(v.x) + double(v.y) * double(v.y);
    }
    s = block_sum(s, sh);
    if (threadIdx.x == 0) rowsum[m] = s;
}

int grid_for(int64_t n) {
    int64_t g = (n + RT - 1) / RT;
    return (int)(g > 4096 ? 4096 : (g < 1 ? 1 : g));
}

}  // namespace

template <typename T>
cudaError_t launch_widen(const cx<T> *src, double *dst, int64_t n, cudaStream_t st) {
    widen_kernel<T><<<grid_for(n), RT, 0, st>>>(src, dst, n);
    return cudaGetLastError();
}
template <typename T>
cudaError_t launch_narrow(const double *src, cx<T> *dst, int64_t n, cudaStream_t st) {
    narrow_kernel<T><<<grid_for(n), RT, 0, st>>>(src, dst, n);
    return cudaGetLastError();
}
template <typename T>
cudaError_t launch_widen_real(const T *src, double *dst, int64_t n, cudaStream_t st) {
    widen_real_kernel<T><<<grid_for(n), RT, 0, st>>>(src, dst, n);
    return cudaGetLastError();
}
cudaError_t launch_reduce_stats(const double *stats, int nr, double *out, cudaStream_t st) {
    reduce_stats_kernel<false><<<1, RT, 0, st>>>(stats, nr, 0, out);
    return cudaGetLastError();
}
cudaError_t launch_reduce_stats_flat(const double *stats, int nrows, int axis_row, double *out,
                                     cudaStream_t st) {
    if (axis_row < 0 || axis_row >= nrows) return cudaErrorInvalidValue;
    reduce_stats_kernel<true><<<1, 1024, 0, st>>>(stats, nrows, axis_row, out);
    return cudaGetLastError();
}
cudaError_t launch_diff_final(const double *rows, int nr, double *out, cudaStream_t st) {
    diff_final_kernel<<<1, RT, 0, st>>>(rows, nr, out);
    return cudaGetLastError();
}
template <typename T>
cudaError_t launch_profiles(const cx<T> *f, int nr, int nt, double *power, double *rowsum,
                            cudaStream_t st) {
    if (power) power_kernel<T><<<(nt + RT - 1) / RT, RT, 0, st>>>(f, nr, nt, power);
    if (rowsum) rowsum_kernel<T><<<nr, RT, 0, st>>>(f, nt, rowsum);
    return cudaGetLastError();
}

#define FCN_INST(T)                                                                       \
    template cudaError_t launch_widen<T>(const cx<T> *, double *, int64_t, cudaStream_t);  \
    template cudaError_t launch_narrow<T>(const double *, cx<T> *, int64_t, cudaStream_t); \
    template cudaError_t launch_widen_real<T>(const T *, double *, int64_t, cudaStream_t); \
    template cudaError_t launch_profiles<T>(const cx<T> *, int, int, double *, double *,   \
                                            cudaStream_t);
FCN_INST(float)
FCN_INST(double)
#undef FCN_INST

}  // namespace fcn
