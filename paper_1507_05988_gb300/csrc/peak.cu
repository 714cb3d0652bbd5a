// peak.cu -- arithmetic peaks of the GPU the library runs on, measured by
// this library's own microkernel: the denominators of the ALU rooflines of
// the FP64 path (FP64 FMA) and of the row stage (FP32 FMA, scalar and packed
// f32x2).  Not an operation of the method.
//
// Each thread runs CH independent FMA chains a <- a * b + c for `iters`
// iterations (CH hides the FMA latency), over a grid of 8 CTAs of 256 threads
// per SM; the rate is 2 CH iters threads / time, best of three launches
// timed with CUDA events after one warm-up launch.  Clocks are whatever the
// GPU runs at (nothing here changes them).
#include <cuda_runtime.h>

#include <algorithm>

#include "../../include/fcn.h"

namespace {

constexpr int kCh = 8;

__global__ void __launch_bounds__(256) fma64_kernel(double *out, int iters, double b, double c) {
    double a[kCh];
#pragma unroll
    for (int k = 0; k < kCh; ++k) a[k] = 1e-3 * threadIdx.x + k;
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int k = 0; k < kCh; ++k) a[k] = fma(a[k], b, c);
    }
    double s = 0.0;
#pragma unroll
    for (int k = 0; k < kCh; ++k) s += a[k];
    out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

__global__ void __launch_bounds__(256) fma32_kernel(float *out, int iters, float b, float c) {
    float a[kCh];
#pragma unroll
    for (int k = 0; k < kCh; ++k) a[k] = 1e-3f * threadIdx.x + k;
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int k = 0; k < kCh; ++k) a[k] = fmaf(a[k], b, c);
    }
    float s = 0.f;
#pragma unroll
    for (int k = 0; k < kCh; ++k) s += a[k];
    out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

// Packed pairs: one fma.rn.f32x2 instruction does two IEEE single FMAs.
__global__ void __launch_bounds__(256) fma32x2_kernel(float *out, int iters, float b, float c) {
    unsigned long long a[kCh];
    const float2 bb = make_float2(b, b), cc = make_float2(c, c);
    const unsigned long long pb = *reinterpret_cast<const unsigned long long *>(&bb);
    const unsigned long long pc = *reinterpret_cast<const unsigned long long *>(&cc);
#pragma unroll
    for (int k = 0; k < kCh; ++k) {
        const float2 v = make_float2(1e-3f * threadIdx.x + k, 2e-3f * threadIdx.x - k);
        a[k] = *reinterpret_cast<const unsigned long long *>(&v);
    }
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int k = 0; k < kCh; ++k)
            asm volatile("fma.rn.f32x2 %0, %0, %1, %2;" : "+l"(a[k]) : "l"(pb), "l"(pc));
    }
    float s = 0.f;
#pragma unroll
    for (int k = 0; k < kCh; ++k) {
        const float2 v = *reinterpret_cast<const float2 *>(&a[k]);
        s += v.x + v.y;
    }
    out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

}  // namespace

extern "C" int fcn_alu_peak(int32_t kind, double *flop_per_s, void *stream) {
    if (!flop_per_s || kind < 0 || kind > 2) return FCN_ERR_ARG;
    const cudaStream_t st = static_cast<cudaStream_t>(stream);
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
        return FCN_ERR_CUDA;
    const int threads = 256, ctas = 8 * sms;
    // about 10 ms per launch at the nominal rates (FP64 is ~1/50 of FP32)
    const int iters = kind == 0 ? 2048 : 65536;
    void *buf = nullptr;
    if (cudaMalloc(&buf, sizeof(double) * (size_t)threads * ctas) != cudaSuccess) return FCN_ERR_NOMEM;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    int rc = FCN_OK;
    float best = 1e30f;
    if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) rc = FCN_ERR_CUDA;
    for (int r = 0; r < 4 && rc == FCN_OK; ++r) {     // launch 0 warms up
        cudaEventRecord(e0, st);
        if (kind == 0)
            fma64_kernel<<<ctas, threads, 0, st>>>((double *)buf, iters, 0.999999, 1e-7);
        else if (kind == 1)
            fma32_kernel<<<ctas, threads, 0, st>>>((float *)buf, iters, 0.9999f, 1e-4f);
        else
            fma32x2_kernel<<<ctas, threads, 0, st>>>((float *)buf, iters, 0.9999f, 1e-4f);
        cudaEventRecord(e1, st);
        float ms = 0.f;
        if (cudaGetLastError() != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess ||
            cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess) {
            rc = FCN_ERR_CUDA;
            break;
        }
        if (r > 0) best = std::min(best, ms);
    }
    if (rc == FCN_OK) {
        const double fmas = double(kCh) * iters * threads * ctas * (kind == 2 ? 2.0 : 1.0);
        *flop_per_s = 2.0 * fmas / (best * 1e-3);
    }
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    cudaFree(buf);
    return rc;
}
