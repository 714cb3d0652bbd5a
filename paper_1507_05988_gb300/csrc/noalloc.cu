// noalloc.cu -- the Crank-Nicolson column stage for callers that cannot
// allocate device memory (fcn_op_cn_noalloc in include/fcn.h).
//
// The column stage needs scratch beyond its input/output field: the table of
// inverse Thomas pivots for the given dz and the radial ratio tables.  The
// regular entry points keep those in cudaMalloc'ed buffers.  This variant
// keeps them in one file-scope device array of fixed size instead, so a call
// allocates nothing: no cudaMalloc, no cudaFree, no allocating library call.
//
// The array lives in every GPU that loads the library, until the process
// exits.  Host code cannot use the array's name as a device address, so the
// first call on each device (with that device current) looks the address up
// with cudaGetSymbolAddress and caches it.  All calls share the array and it
// keeps the last call's contents; every call rewrites everything it reads, so
// nothing has to be cleared, but calls whose kernels overlap on the GPU (two
// streams, or two host threads) race on it.
#include <cuda_runtime.h>

#include <cmath>
#include <mutex>
#include <string>

#include "../../include/fcn.h"
#include "fcn_device.cuh"
#include "fcn_host.h"

using namespace fcn;

namespace {

constexpr size_t kScratchBytes = size_t(FCN_NOALLOC_SCRATCH_BYTES);
static __device__ __align__(256) unsigned char g_cn_scratch[kScratchBytes];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
void *g_scratch_ptr[kMaxDevices] = {nullptr};

// Device address of g_cn_scratch on the current device (looked up once per
// device, with that device current).
int scratch_address(void **out) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return FCN_ERR_CUDA;
    if (dev < 0 || dev >= kMaxDevices) return FCN_ERR_UNSUPPORTED;
    std::lock_guard<std::mutex> lk(g_mu);
    if (!g_scratch_ptr[dev]) {
        void *p = nullptr;
        e = cudaGetSymbolAddress(&p, g_cn_scratch);
        if (e != cudaSuccess) return FCN_ERR_CUDA;
        g_scratch_ptr[dev] = p;
    }
    *out = g_scratch_ptr[dev];
    return FCN_OK;
}

// lo_j = 1 - 1/(2j), hi_j = 1 + 1/(2j) for j >= 1, 0 at j = 0, in FP64 and in
// the working precision (the same expression the host tables use).
template <typename T>
__global__ void lohi_kernel(int nr, double *lo64, double *hi64, T *lo, T *hi) {
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= nr) return;
    const double l = j ? 1.0 - 1.0 / (2.0 * j) : 0.0;
    const double h = j ? 1.0 + 1.0 / (2.0 * j) : 0.0;
    lo64[j] = l;
    hi64[j] = h;
    lo[j] = T(l);
    hi[j] = T(h);
}

size_t align256(size_t n) { return (n + 255) & ~size_t(255); }

template <typename T>
int run(const fcn_grid &g, const fcn_params &p, double dz, void *field, cudaStream_t st) {
    const size_t entries = (size_t)g.nr * (g.nt / 2 + 1);
    const size_t tab_bytes = align256(entries * sizeof(cx<T>));
    const size_t r64_bytes = align256(sizeof(double) * g.nr);
    const size_t rt_bytes = align256(sizeof(T) * g.nr);
    const size_t need = tab_bytes + 2 * r64_bytes + 2 * rt_bytes;
    // the table (Nr*(Nt/2+1) complex values) and 4 radial tables must fit
    if (need > kScratchBytes) return FCN_ERR_UNSUPPORTED;
    void *base = nullptr;
    int rc = scratch_address(&base);
    if (rc) return rc;
    unsigned char *b = static_cast<unsigned char *>(base);
    cx<T> *table = reinterpret_cast<cx<T> *>(b);
    double *lo64 = reinterpret_cast<double *>(b + tab_bytes);
    double *hi64 = reinterpret_cast<double *>(b + tab_bytes + r64_bytes);
    T *lo = reinterpret_cast<T *>(b + tab_bytes + 2 * r64_bytes);
    T *hi = reinterpret_cast<T *>(b + tab_bytes + 2 * r64_bytes + rt_bytes);

    // the same coefficients as the regular column stage (one host routine)
    double s, dk, disp;
    hostx::cn_coefs(g, p, dz, &s, &dk, &disp);

    lohi_kernel<T><<<(g.nr + 127) / 128, 128, 0, st>>>(g.nr, lo64, hi64, lo, hi);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return FCN_ERR_CUDA;
    TableArgs ta;
    ta.nr = g.nr;
    ta.nt = g.nt;
    ta.s = s;
    ta.dk = dk;
    ta.lo = lo64;
    ta.hi = hi64;
    e = launch_cn_table<T>(ta, table, st);
    if (e != cudaSuccess) return FCN_ERR_CUDA;
    ColArgs<T> ca;
    ca.field = static_cast<cx<T> *>(field);
    ca.invden = table;
    ca.lo = lo;
    ca.hi = hi;
    ca.nr = g.nr;
    ca.nt = g.nt;
    ca.s = T(s);
    ca.dk = T(dk);
    ca.disp = disp;
    ca.variant = 0;
    e = launch_cn<T>(ca, st);
    if (e != cudaSuccess) return FCN_ERR_CUDA;
    return FCN_OK;
}

}  // namespace

extern "C" {

int fcn_op_cn_noalloc(const fcn_grid *grid, const fcn_params *params, int32_t precision, double dz,
                      void *field, void *stream) {
    // the same argument checks as every other entry point (grid range,
    // precision, physics parameters and flags), then the field and dz
    std::string why;
    const int rc = hostx::check_params(precision, grid, params, &why);
    if (rc) return rc;
    if (!field || !(dz > 0) || !std::isfinite(dz)) return FCN_ERR_ARG;
    const cudaStream_t st = static_cast<cudaStream_t>(stream);
    return precision == FCN_FP64 ? run<double>(*grid, *params, dz, field, st)
                                 : run<float>(*grid, *params, dz, field, st);
}

}  // extern "C"
