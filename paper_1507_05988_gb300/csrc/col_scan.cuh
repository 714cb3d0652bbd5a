// col_scan.cuh -- device helpers shared by the column stages (the radial
// Crank-Nicolson solve in col_kernel.cu and the Cartesian line solves in
// xy_kernel.cu): complex reciprocal, warp shuffles of complex values, the
// chunked affine-map scan that evaluates a Thomas sweep in parallel, and the
// exact dispersion factor of one frequency column.
#pragma once

#include "fcn_device.cuh"

namespace fcn {
namespace colscan {

template <typename T>
__device__ __forceinline__ cx<T> czero() { return mk(T(0), T(0)); }

// 1/z in FP64
__device__ __forceinline__ cx<double> crecip(cx<double> z) {
    const double d = z.x * z.x + z.y * z.y;
    return mk(z.x / d, -z.y / d);
}

__device__ __forceinline__ cx<float> crecip(cx<float> z) {
    const float d = 1.0f / (z.x * z.x + z.y * z.y);
    return mk(z.x * d, -z.y * d);
}

template <typename T>
__device__ __forceinline__ cx<T> shfl_up_cx(cx<T> v, int d) {
    return mk(__shfl_up_sync(0xffffffffu, v.x, d), __shfl_up_sync(0xffffffffu, v.y, d));
}
template <typename T>
__device__ __forceinline__ cx<T> shfl_down_cx(cx<T> v, int d) {
    return mk(__shfl_down_sync(0xffffffffu, v.x, d), __shfl_down_sync(0xffffffffu, v.y, d));
}

// Value entering this thread's chunk when the chunk maps x -> A x + B of one
// column are composed in chunk order (REV = false: from chunk 0, value 0
// entering it) or in reverse chunk order (REV = true: from the last chunk).
// Lanes of one column sit C apart in a warp, so the in-warp part is a
// shuffle scan; warp totals are combined by one thread per column.
template <typename T, bool REV>
__device__ __forceinline__ cx<T> chunk_scan(cx<T> A, cx<T> B, int C, int col, cx<T> *smA,
                                            cx<T> *smB, cx<T> *smC) {
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int cpw = 32 / C;
    const int ciw = lane / C;
    for (int d = 1; d < cpw; d <<= 1) {
        const cx<T> Ao = REV ? shfl_down_cx(A, d * C) : shfl_up_cx(A, d * C);
        const cx<T> Bo = REV ? shfl_down_cx(B, d * C) : shfl_up_cx(B, d * C);
        const bool take = REV ? (ciw + d < cpw) : (ciw >= d);
        if (take) {
            B = cmul(A, Bo) + B;
            A = cmul(A, Ao);
        }
    }
    cx<T> Ae = REV ? shfl_down_cx(A, C) : shfl_up_cx(A, C);
    cx<T> Be = REV ? shfl_down_cx(B, C) : shfl_up_cx(B, C);
    if (REV ? (ciw == cpw - 1) : (ciw == 0)) {
        Ae = mk(T(1), T(0));
        Be = czero<T>();
    }
    const int nw = blockDim.x >> 5;
    cx<T> wc = czero<T>();
    if (nw > 1) {
        if (REV ? (ciw == 0) : (ciw == cpw - 1)) {
            smA[FCN_IDX(w * C + col, nw * C, 38)] = A;
            smB[FCN_IDX(w * C + col, nw * C, 39)] = B;
        }
        __syncthreads();
        if (nw * C <= 32) {
            // one warp scans the warp totals of all C columns at once:
            // lane l holds warp l / C of column l % C
            if (threadIdx.x < 32) {
                const int kw = lane / C, c0 = lane % C;
                const bool on = kw < nw;
                cx<T> A2 = mk(T(1), T(0)), B2 = czero<T>();
                if (on) {
                    A2 = smA[FCN_IDX(kw * C + c0, nw * C, 48)];
                    B2 = smB[FCN_IDX(kw * C + c0, nw * C, 49)];
                }
                for (int d = 1; d < nw; d <<= 1) {
                    const cx<T> Ao = REV ? shfl_down_cx(A2, d * C) : shfl_up_cx(A2, d * C);
                    const cx<T> Bo = REV ? shfl_down_cx(B2, d * C) : shfl_up_cx(B2, d * C);
                    if (REV ? (kw + d < nw) : (kw >= d)) {
                        B2 = cmul(A2, Bo) + B2;
                        A2 = cmul(A2, Ao);
                    }
                }
                cx<T> ex = REV ? shfl_down_cx(B2, C) : shfl_up_cx(B2, C);
                if (REV ? (kw == nw - 1) : (kw == 0)) ex = czero<T>();
                if (on) smC[FCN_IDX(kw * C + c0, nw * C, 50)] = ex;
            }
        } else if ((int)threadIdx.x < C) {
            const int c0 = threadIdx.x;
            cx<T> c = czero<T>();
            if (!REV) {
                for (int k = 0; k < nw; ++k) {
                    smC[FCN_IDX(k * C + c0, nw * C, 40)] = c;
                    c = cmul(smA[FCN_IDX(k * C + c0, nw * C, 41)], c) + smB[FCN_IDX(k * C + c0, nw * C, 42)];
                }
            } else {
                for (int k = nw - 1; k >= 0; --k) {
                    smC[FCN_IDX(k * C + c0, nw * C, 40)] = c;
                    c = cmul(smA[FCN_IDX(k * C + c0, nw * C, 41)], c) + smB[FCN_IDX(k * C + c0, nw * C, 42)];
                }
            }
        }
        __syncthreads();
        wc = smC[FCN_IDX(w * C + col, nw * C, 43)];
    }
    return cmul(Ae, wc) + Be;
}

// Exact dispersion factor exp(2 i disp qq^2) of column q (FCN_EXACT_DISPERSION;
// disp = 0: none).  Computed in FP64 once per thread; in FP32 applied as a
// two-float pair (hi + lo) inside the FMAs, so that its rounding does not
// act identically at every step.
template <typename T>
struct DispPhase {
    cx<T> hi, lo;
    bool on;
};
template <typename T>
__device__ __forceinline__ DispPhase<T> disp_phase(double disp, int qq) {
    DispPhase<T> p;
    p.on = disp != 0.0;
    p.hi = mk(T(1), T(0));
    p.lo = czero<T>();
    if (p.on) {
        double sn, cs;
        sincos(2.0 * disp * (double)qq * (double)qq, &sn, &cs);
        p.hi = mk(T(cs), T(sn));
        p.lo = mk(T(cs - (double)p.hi.x), T(sn - (double)p.hi.y));
    }
    return p;
}
template <typename T>
__device__ __forceinline__ cx<T> disp_apply(cx<T> x, const DispPhase<T> &p) {
    if (!p.on) return x;
    if constexpr (sizeof(T) == 4) {
        const float lre = fmaf(x.x, p.lo.x, -x.y * p.lo.y);
        const float lim = fmaf(x.x, p.lo.y, x.y * p.lo.x);
        return mk(fmaf(x.x, p.hi.x, fmaf(-x.y, p.hi.y, lre)), fmaf(x.x, p.hi.y, fmaf(x.y, p.hi.x, lim)));
    } else {
        return cmul(x, p.hi);
    }
}

// chunk_scan for NP right-hand sides sharing one A: returns the value entering
// this thread's chunk for each of them.  smB, smC hold NP * nwarp * C values.
template <typename T, bool REV, int NP>
__device__ __forceinline__ void chunk_scan_n(cx<T> A, cx<T> (&B)[NP], int C, int col, cx<T> *smA,
                                             cx<T> *smB, cx<T> *smC, cx<T> (&out)[NP]) {
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int cpw = 32 / C;
    const int ciw = lane / C;
    for (int d = 1; d < cpw; d <<= 1) {
        const cx<T> Ao = REV ? shfl_down_cx(A, d * C) : shfl_up_cx(A, d * C);
        cx<T> Bo[NP];
#pragma unroll
        for (int i = 0; i < NP; ++i) Bo[i] = REV ? shfl_down_cx(B[i], d * C) : shfl_up_cx(B[i], d * C);
        const bool take = REV ? (ciw + d < cpw) : (ciw >= d);
        if (take) {
#pragma unroll
            for (int i = 0; i < NP; ++i) B[i] = cmul(A, Bo[i]) + B[i];
            A = cmul(A, Ao);
        }
    }
    cx<T> Ae = REV ? shfl_down_cx(A, C) : shfl_up_cx(A, C);
    cx<T> Be[NP];
#pragma unroll
    for (int i = 0; i < NP; ++i) Be[i] = REV ? shfl_down_cx(B[i], C) : shfl_up_cx(B[i], C);
    if (REV ? (ciw == cpw - 1) : (ciw == 0)) {
        Ae = mk(T(1), T(0));
#pragma unroll
        for (int i = 0; i < NP; ++i) Be[i] = czero<T>();
    }
    const int nw = blockDim.x >> 5;
    const int nwc = nw * C;
#pragma unroll
    for (int i = 0; i < NP; ++i) out[i] = Be[i];
    if (nw > 1) {
        if (REV ? (ciw == 0) : (ciw == cpw - 1)) {
            smA[FCN_IDX(w * C + col, nwc, 54)] = A;
#pragma unroll
            for (int i = 0; i < NP; ++i) smB[FCN_IDX(i * nwc + w * C + col, NP * nwc, 55)] = B[i];
        }
        __syncthreads();
        if ((int)threadIdx.x < C) {
            const int c0 = threadIdx.x;
            cx<T> c[NP];
#pragma unroll
            for (int i = 0; i < NP; ++i) c[i] = czero<T>();
            for (int kk = 0; kk < nw; ++kk) {
                const int k = REV ? nw - 1 - kk : kk;
                const cx<T> Ak = smA[FCN_IDX(k * C + c0, nwc, 56)];
#pragma unroll
                for (int i = 0; i < NP; ++i) {
                    smC[FCN_IDX(i * nwc + k * C + c0, NP * nwc, 57)] = c[i];
                    c[i] = cmul(Ak, c[i]) + smB[FCN_IDX(i * nwc + k * C + c0, NP * nwc, 58)];
                }
            }
        }
        __syncthreads();
#pragma unroll
        for (int i = 0; i < NP; ++i)
            out[i] = cmul(Ae, smC[FCN_IDX(i * nwc + w * C + col, NP * nwc, 59)]) + Be[i];
    }
}

}  // namespace colscan
}  // namespace fcn
