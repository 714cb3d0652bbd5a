// xy_kernel.cu -- transverse stage of the FCN z-step on a Cartesian grid
// (Ma & Lin, arXiv:1507.05988, Sec. 2: Delta_perp = d^2/dx^2 + d^2/dy^2 for
// beams without cylindrical symmetry).
//
// Each axis takes the Crank-Nicolson step of Eqs. (diff1)-(diff2) with the
// walls held at A = 0 (Eq. (bound) at r = max, on all four sides); the
// two-dimensional system is not tridiagonal, so the stage applies the x and
// the y factor one after the other (Peaceman-Rachford alternating
// directions; the factors commute, and the product differs from the unsplit
// two-dimensional step by O(dz^3) per step, the order of the Strang split).
// On a line of n nodes, spacing h, s = dz/(4 k0 h^2):
//   walls (j = 0, n-1) : b = 1, everything else 0
//   1..n-2             : a = c = -is, b = 1 + i(2s - delta_q)
//                        d = f =  is, e = 1 - i(2s - delta_q)
// with delta_q = k'' omega_q^2 dz/4 in the y factor and 0 in the x factor.
//
// The matrix depends on (j, |q|, dz) only; its Thomas pivots are computed
// once per dz (xy_table_kernel, FP64, stored as 1/pivot in the working
// precision), and the two sweeps run as the chunked parallel scan of affine
// maps that the radial column stage uses (colscan::chunk_scan_n): a thread
// owns L consecutive nodes of one line (or of NP lines of the same
// frequency bin, which share the pivots) in registers.  In FP32 the
// pivots, the sweep factors and the explicit side's coefficients are
// two-float pairs (see xy_table_kernel).  The lines of one
// launch are addressed as b * bstride + j * pitch + c (see XYLine), so the x
// lines (stride ny*nt) and the y lines (stride nt) use the same kernel, with
// C adjacent frequency columns per CTA for whole-sector row accesses.
#include "col_scan.cuh"

namespace fcn {
namespace {

using namespace colscan;

// One thread per |q| = 0..nt/2: piv_0 = 1 (wall), piv_1 = b,
// piv_j = b - a c / piv_{j-1} = b + s^2 / piv_{j-1} (2 <= j <= n-2),
// piv_{n-1} = 1 (wall); the table holds 1/piv_j, row j at j * (nt/2+1):
// in FP64 one complex double per entry, in FP32 a two-float pair (hi, lo;
// xy_table_entries complex floats per entry).  On a line the coefficients do
// not depend on j, so the pivots settle to one value within a few nodes and
// their FP32 roundings are the same at almost every node: rounded once they
// made the discrete factor non-unitary coherently along the line, which
// showed as an energy drift of -2e-8 per line factor and step (an FP32
// emulation of one line; -3e-10 with the pivots and sweep factors two-float).
template <typename T>
__global__ void xy_table_kernel(int n, int nt, double s, double dk, cx<T> *table) {
    const int nq = nt / 2 + 1;
    const int q = blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= nq) return;
    const double delta = dk * double(q) * double(q);
    const cx<double> b = mk(1.0, 2.0 * s - delta);
    cx<double> inv = mk(1.0, 0.0);
    for (int j = 0; j < n; ++j) {
        cx<double> piv;
        if (j == 0 || j == n - 1) piv = mk(1.0, 0.0);
        else if (j == 1) piv = b;
        else piv = b + mk(s * s * inv.x, s * s * inv.y);
        inv = crecip(piv);
        const size_t e = FCN_IDX((size_t)j * nq + q, (size_t)n * nq, 70);
        if constexpr (sizeof(T) == 4) {
            const float hx = float(inv.x), hy = float(inv.y);
            reinterpret_cast<float4 *>(table)[e] =
                make_float4(hx, hy, float(inv.x - double(hx)), float(inv.y - double(hy)));
        } else {
            table[e] = mk(T(inv.x), T(inv.y));
        }
    }
}

// Two-float pivots and sweep factors of the FP32 line sweeps (FP64: the lo
// parts are zero and drop out at compile time).
template <typename T>
struct Piv2 {
    cx<T> h, l;
};
template <typename T>
__device__ __forceinline__ Piv2<T> load_piv(const cx<T> *tab, size_t e) {
    Piv2<T> p;
    if constexpr (sizeof(T) == 4) {
        const float4 w = __ldg(reinterpret_cast<const float4 *>(tab) + e);
        p.h = mk(w.x, w.y);
        p.l = mk(w.z, w.w);
    } else {
        p.h = ldg_cx(tab + e);
        p.l = czero<T>();
    }
    return p;
}
// alpha = i s / piv as a two-float pair from s = sh + sl and 1/piv = h + l:
// hi the rounded product i sh h, lo its rounding error (exact by FMA) plus
// i (sh l + sl h).
template <typename T>
__device__ __forceinline__ Piv2<T> sweep_factor(const Piv2<T> &v, T sh, T sl) {
    Piv2<T> a;
    if constexpr (sizeof(T) == 4) {
        const float hx = -sh * v.h.y, hy = sh * v.h.x;
        const float ex = fmaf(-sh, v.h.y, -hx), ey = fmaf(sh, v.h.x, -hy);
        a.h = mk(hx, hy);
        a.l = mk(fmaf(-sh, v.l.y, fmaf(-sl, v.h.y, ex)), fmaf(sh, v.l.x, fmaf(sl, v.h.x, ey)));
    } else {
        a.h = cmul_i(v.h, sh);
        a.l = czero<T>();
    }
    return a;
}
// a x + b with a two-float: the lo product first, then the hi one fused.
template <typename T>
__device__ __forceinline__ cx<T> cmadd2(const Piv2<T> &a, cx<T> x, cx<T> b) {
    if constexpr (sizeof(T) == 4) {
        const float tx = fmaf(a.l.x, x.x, fmaf(-a.l.y, x.y, b.x));
        const float ty = fmaf(a.l.x, x.y, fmaf(a.l.y, x.x, b.y));
        return mk(fmaf(a.h.x, x.x, fmaf(-a.h.y, x.y, tx)), fmaf(a.h.x, x.y, fmaf(a.h.y, x.x, ty)));
    } else {
        return cmul(a.h, x) + b;
    }
}

// NP lines per thread: batch items b = NP blockIdx.y + i (i < NP) at the
// same column c share the frequency bin, hence the pivots and the A part of
// every affine map; their recurrences run side by side (independent chains).
template <typename T, int L, int NP, int MAXT = 512, int MINB = 1>
__global__ void __launch_bounds__(MAXT, MINB)
xy_line_kernel(XYLine<T> a, int C) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int nwarp = blockDim.x >> 5;
    cx<T> *smA = reinterpret_cast<cx<T> *>(smem_raw);
    cx<T> *smB = smA + nwarp * C;
    cx<T> *smC = smB + NP * nwarp * C;

    const int tid = threadIdx.x;
    const int col = tid % C;
    const int chunk = tid / C;
    const int c = blockIdx.x * C + col;               // < width (width % C == 0)
    const int nt = a.nt, n = a.n;
    const int q = c & (nt - 1);
    const int nq = nt / 2 + 1;
    const int qq = (q <= nt / 2) ? q : nt - q;
    // interior: e = 1 - i g1, g1 = 2s - delta_q; in FP32 s and g1 are
    // two-float pairs (lo = rounding error of the FP64 value), on the
    // explicit side as in the radial stage and in the sweep factors with the
    // two-float pivots, so that the rounding of the coefficients does not
    // perturb the discrete operator the same way at every step
    const T s = a.s;
    const double g1d = 2.0 * a.s64 - a.dk64 * double(qq) * double(qq);
    const T g1 = T(g1d);
    const T sl = T(a.s64 - double(s)), g1l = T(g1d - double(g1));
    const int j0 = chunk * L;
    cx<T> *line[NP];
    bool on[NP];
#pragma unroll
    for (int i = 0; i < NP; ++i) {
        const int b = blockIdx.y * NP + i;
        on[i] = b < a.batch;
        line[i] = a.field + (size_t)(on[i] ? b : 0) * (size_t)a.bstride + c;
    }

    cx<T> x[NP][L + 2];
#pragma unroll
    for (int i = 0; i < NP; ++i)
#pragma unroll
        for (int k = 0; k < L + 2; ++k) {
            const int j = j0 - 1 + k;
            x[i][k] = (on[i] && j >= 0 && j < n)
                          ? a.field[FCN_IDX(line[i] - a.field + (size_t)j * a.pitch, a.total, 71)]
                          : czero<T>();
        }
    Piv2<T> inv[L];
#pragma unroll
    for (int k = 0; k < L; ++k) {
        const int j = j0 + k;
        if (j < n) {
            inv[k] = load_piv(a.invden, FCN_IDX((size_t)j * nq + qq, (size_t)n * nq, 72));
        } else {
            inv[k].h = inv[k].l = czero<T>();
        }
    }

    // forward sweep, pass 1: y_j = alpha_j y_{j-1} + beta_j per node, and the
    // chunk's composed map y_end = PA y_in + PB
    cx<T> y[NP][L];
    cx<T> PA = mk(T(1), T(0)), PB[NP];
#pragma unroll
    for (int i = 0; i < NP; ++i) PB[i] = czero<T>();
#pragma unroll
    for (int k = 0; k < L; ++k) {
        const int j = j0 + k;
        if (j >= 1 && j < n - 1) {
            const Piv2<T> alpha = sweep_factor(inv[k], s, sl);
#pragma unroll
            for (int i = 0; i < NP; ++i) {
                const cx<T> sum = x[i][k] + x[i][k + 2];
                cx<T> w;
                if constexpr (sizeof(T) == 4) {
                    w.x = fmaf(-g1, x[i][k + 1].x, fmaf(s, sum.x, fmaf(-g1l, x[i][k + 1].x, sl * sum.x)));
                    w.y = fmaf(-g1, x[i][k + 1].y, fmaf(s, sum.y, fmaf(-g1l, x[i][k + 1].y, sl * sum.y)));
                } else {
                    w = mk(s * sum.x - g1 * x[i][k + 1].x, s * sum.y - g1 * x[i][k + 1].y);
                }
                const cx<T> rhs = mk(x[i][k + 1].x - w.y, x[i][k + 1].y + w.x);
                y[i][k] = cmadd2(inv[k], rhs, czero<T>());
                PB[i] = cmadd2(alpha, PB[i], y[i][k]);
            }
            PA = cmadd2(alpha, PA, czero<T>());
        } else {
            // walls: y = 0 and the map sends everything to 0; nodes past the
            // end of the line: identity
#pragma unroll
            for (int i = 0; i < NP; ++i) {
                y[i][k] = czero<T>();
                if (j < n) PB[i] = czero<T>();
            }
            if (j < n) PA = czero<T>();
        }
    }
    // forward sweep, pass 2: exact y from the carry entering the chunk
    {
        cx<T> yp[NP];
        chunk_scan_n<T, false, NP>(PA, PB, C, col, smA, smB, smC, yp);
#pragma unroll
        for (int k = 0; k < L; ++k) {
            const int j = j0 + k;
            const bool inner = j >= 1 && j < n - 1;
            const Piv2<T> alpha = sweep_factor(inv[k], s, sl);
#pragma unroll
            for (int i = 0; i < NP; ++i) {
                if (inner) {
                    y[i][k] = cmadd2(alpha, yp[i], y[i][k]);
                    yp[i] = y[i][k];
                } else if (j < n) {
                    yp[i] = czero<T>();
                }
            }
        }
    }
    // backward sweep, pass 1: chunk map x_first = QA x_next + QB, with
    // x_j = gamma_j x_{j+1} + y_j, gamma_j = is / piv_j inside, 0 at walls
    cx<T> QA = mk(T(1), T(0)), QB[NP];
#pragma unroll
    for (int i = 0; i < NP; ++i) QB[i] = czero<T>();
#pragma unroll
    for (int k = L - 1; k >= 0; --k) {
        const int j = j0 + k;
        if (j < n) {
            Piv2<T> gamma;
            if (j >= 1 && j < n - 1) gamma = sweep_factor(inv[k], s, sl);
            else gamma.h = gamma.l = czero<T>();
#pragma unroll
            for (int i = 0; i < NP; ++i) QB[i] = cmadd2(gamma, QB[i], y[i][k]);
            QA = cmadd2(gamma, QA, czero<T>());
        }
    }
    // backward sweep, pass 2 and store
    {
        cx<T> xn[NP];
        chunk_scan_n<T, true, NP>(QA, QB, C, col, smA, smB, smC, xn);
        const DispPhase<T> ph = disp_phase<T>(a.disp, qq);
#pragma unroll
        for (int k = L - 1; k >= 0; --k) {
            const int j = j0 + k;
            if (j < n) {
                Piv2<T> gamma;
                if (j >= 1 && j < n - 1) gamma = sweep_factor(inv[k], s, sl);
                else gamma.h = gamma.l = czero<T>();
#pragma unroll
                for (int i = 0; i < NP; ++i) {
                    xn[i] = cmadd2(gamma, xn[i], y[i][k]);
                    if (on[i])
                        a.field[FCN_IDX(line[i] - a.field + (size_t)j * a.pitch, a.total, 73)] =
                            disp_apply(xn[i], ph);
                }
            }
        }
    }
}

// C columns per CTA: at least one 32-byte sector, doubled while the CTA
// stays within `target` threads; whole warps (chunks past the line's end
// are identity maps).
template <typename T, int L, int NP, int MAXT = 512, int MINB = 1>
cudaError_t launch_xy_l(const XYLine<T> &a, int target, cudaStream_t st) {
    constexpr int CMIN = 32 / int(sizeof(cx<T>));
    const int P = (a.n + L - 1) / L;
    int C = CMIN;
    while (C * 2 * P <= target && C * 2 <= 32) C *= 2;
    if (C > a.nt) C = a.nt;
    const int threads = ((C * P + 31) / 32) * 32;
    if (threads > MAXT) return cudaErrorInvalidConfiguration;
    if (a.width % C != 0) return cudaErrorInvalidValue;
    const size_t smem = sizeof(cx<T>) * (1 + 2 * NP) * (size_t)(threads / 32) * C;
    const dim3 grid(a.width / C, (a.batch + NP - 1) / NP);
    return launch_k(xy_line_kernel<T, L, NP, MAXT, MINB>, grid, dim3(threads), smem, st, a, C);
}

}  // namespace

template <typename T>
cudaError_t launch_xy_table(int n, int nt, double s, double dk, cx<T> *table, cudaStream_t st) {
    const int nq = nt / 2 + 1;
    xy_table_kernel<T><<<(nq + 127) / 128, 128, 0, st>>>(n, nt, s, dk, table);
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_xy_line(const XYLine<T> &a, cudaStream_t st) {
    if (a.n < 3 || a.nt < 1 || (a.nt & (a.nt - 1)) || a.width < 1 || (a.width % a.nt) || a.batch < 1)
        return cudaErrorInvalidValue;
    constexpr int LL = sizeof(T) == 4 ? 16 : 8;   // long chunk
    constexpr int LS = LL / 2;                     // short chunk
    cudaError_t e = cudaErrorInvalidConfiguration;
    switch (a.variant) {
        case 1: e = launch_xy_l<T, LS, 1>(a, 512, st); break;
        case 2: e = launch_xy_l<T, LS, 2>(a, 512, st); break;
        case 3: e = launch_xy_l<T, LS, 2>(a, 256, st); break;
        case 4: e = launch_xy_l<T, LL, 1>(a, 256, st); break;
        case 5: e = launch_xy_l<T, LS, 1>(a, 256, st); break;
        case 6: e = launch_xy_l<T, LS, 2, 256, 3>(a, 256, st); break;
        case 7: e = launch_xy_l<T, LS, 1, 256, 4>(a, 256, st); break;
        default: break;
    }
    if (e == cudaErrorInvalidConfiguration) e = launch_xy_l<T, LL, 1>(a, 512, st);
    return e;
}

template cudaError_t launch_xy_table<float>(int, int, double, double, cx<float> *, cudaStream_t);
template cudaError_t launch_xy_table<double>(int, int, double, double, cx<double> *, cudaStream_t);
template cudaError_t launch_xy_line<float>(const XYLine<float> &, cudaStream_t);
template cudaError_t launch_xy_line<double>(const XYLine<double> &, cudaStream_t);

}  // namespace fcn
