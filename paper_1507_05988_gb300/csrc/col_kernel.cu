// col_kernel.cu -- the column stage of the FCN z-step: for every frequency
// bin q the Crank-Nicolson system M_abc^q A~^{n+1} = M_def^q A~^n of Eq. (matrix)
// (Ma & Lin, arXiv:1507.05988, Sec. 3.1, Eqs. (diff1)-(diff3), (bound),
// (matrix1) and the coefficients after it; reading: c_j and f_j carry
// (1 + 1/(2j)), the value Eqs. (diff2)-(diff3) give).
//
// With s = dz/(4 k0 dr^2) and delta_q = k'' omega_q^2 dz/4:
//   row 0      : b = 1 + i(4s - delta), c = -4is ; e = 1 - i(4s - delta), f = 4is
//   1..Nr-2    : a = -is lo_j, b = 1 + i(2s - delta), c = -is hi_j
//                d =  is lo_j, e = 1 - i(2s - delta), f =  is hi_j
//   row Nr-1   : b = 1, everything else 0 (A = 0 at r = R)
// with lo_j = 1 - 1/(2j), hi_j = 1 + 1/(2j).
//
// The matrix depends on (j, |q|, dz) only, never on the field, so its Thomas
// factorisation (the pivots) is computed once per dz by cn_table_kernel and
// kept in HBM as 1/pivot_j for q = 0..Nt/2 (bins q and Nt-q share omega^2).
// Given the pivots, the two Thomas sweeps are first-order linear recurrences
//   y_j = alpha_j y_{j-1} + beta_j        (alpha = -a/piv, beta = rhs/piv)
//   x_j = gamma_j x_{j+1} + y_j           (gamma = -c/piv)
// i.e. compositions of affine maps, which the column kernel evaluates as a
// chunked parallel scan: a thread owns L consecutive rows of one column
// (values in registers), composes its chunk's map, the chunk maps of a
// column are scanned with warp shuffles (one short pass over the warp
// totals in shared memory), and each thread then replays its recurrence
// from the exact carry.  The result equals the sequential Thomas
// sweep up to rounding.
//
// Layout: the field is [Nr][Nt] with Nt contiguous.  A CTA takes C adjacent
// columns (C complex = 32 B, one DRAM sector, at least) and all Nr rows, so
// each row access of a warp covers whole sectors.  CTAs for the bins q and
// Nt-q are launched next to each other so that the second reads the shared
// pivot rows from L2.
#include "col_scan.cuh"

#include <mutex>

namespace fcn {
namespace {

using namespace colscan;

// One thread per |q| = 0..Nt/2 runs the Thomas pivot recurrence down the
// radial index, piv_j = b_j - a_j c_{j-1}/piv_{j-1}, in FP64 (FP64 tables;
// FP32 tables use cn_table_kernel_f32 below with the same accuracy: pivots
// computed in plain FP32 carry ~1e-7 relative errors that make the discrete
// Crank-Nicolson step slightly non-unitary, the same way at every z-step,
// which showed as an energy drift of ~1e-8 per step).  The radial ratio
// tables are staged in shared memory first, so the serial recurrence waits
// on no global load.
template <typename T>
__global__ void cn_table_kernel(TableArgs a, cx<T> *table) {
    extern __shared__ double sh_lohi[];    // lo[nr], hi[nr]
    for (int j = threadIdx.x; j < a.nr; j += blockDim.x) {
        sh_lohi[j] = a.lo[FCN_IDX(j, a.nr, 31)];
        sh_lohi[a.nr + j] = a.hi[FCN_IDX(j, a.nr, 32)];
    }
    __syncthreads();
    const int nq = a.nt / 2 + 1;
    const int tp = a.tp ? a.tp : nq;
    const int q = blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= nq) return;
    const double delta = a.dk * double(q) * double(q);
    const double s = a.s;
    cx<double> cp = mk(0.0, 0.0);
    for (int j = 0; j < a.nr; ++j) {
        cx<double> b, aa, c;
        if (j == 0) {
            aa = mk(0.0, 0.0);
            b = mk(1.0, 4.0 * s - delta);
            c = mk(0.0, -4.0 * s);
        } else if (j < a.nr - 1) {
            aa = mk(0.0, -s * sh_lohi[j]);
            b = mk(1.0, 2.0 * s - delta);
            c = mk(0.0, -s * sh_lohi[a.nr + j]);
        } else {
            aa = mk(0.0, 0.0);
            b = mk(1.0, 0.0);
            c = mk(0.0, 0.0);
        }
        const cx<double> den = b - cmul(aa, cp);
        const cx<double> inv = crecip(den);
        cp = cmul(c, inv);
        table[FCN_IDX((size_t)j * tp + q, (size_t)a.nr * tp, 30)] = mk(T(inv.x), T(inv.y));
    }
}

// ---- FP32 tables in double-float arithmetic --------------------------------
// A value h + l (two floats, |l| <= ulp(h)/2) carries ~48 significant bits
// with FP32 latencies (Dekker / Knuth error-free transformations; products
// through fmaf).  With aa_j c_{j-1} = -s^2 lo_j hi'_{j-1} (hi'_0 = 4 from
// the axis row, hi'_j = hi_j otherwise) the pivot recurrence is
//   1/piv_j = 1 / (b_j + kappa_j / piv_{j-1}),   kappa_j = s^2 lo_j hi'_{j-1},
// evaluated here in double-float and rounded to float once.
struct f2 {
    float h, l;
};
__device__ __forceinline__ f2 fast_two_sum(float a, float b) {   // |a| >= |b|
    const float s = a + b;
    return {s, b - (s - a)};
}
__device__ __forceinline__ f2 two_sum(float a, float b) {
    const float s = a + b;
    const float bb = s - a;
    return {s, (a - (s - bb)) + (b - bb)};
}
__device__ __forceinline__ f2 df_add(f2 a, f2 b) {
    const f2 s = two_sum(a.h, b.h);
    return fast_two_sum(s.h, s.l + (a.l + b.l));
}
__device__ __forceinline__ f2 df_mul(f2 a, f2 b) {
    const float p = a.h * b.h;
    float e = fmaf(a.h, b.h, -p);
    e = fmaf(a.h, b.l, e);
    e = fmaf(a.l, b.h, e);
    return fast_two_sum(p, e);
}
__device__ __forceinline__ f2 df_recip(f2 a) {
    const float r0 = __frcp_rn(a.h);
    // e = 1 - a r0 (exact leading part by Sterbenz), then r = r0 + r0 e
    const float p = a.h * r0;
    const float pe = fmaf(a.h, r0, -p);
    const float e = ((1.0f - p) - pe) - a.l * r0;
    return fast_two_sum(r0, r0 * e);
}
__device__ __forceinline__ f2 to_f2(double x) {
    const float h = float(x);
    return {h, float(x - double(h))};
}

__global__ void cn_table_kernel_f32(TableArgs a, cx<float> *table) {
    extern __shared__ double sh_kappa[];     // kappa_j as double-float pairs (2 floats)
    f2 *kap = reinterpret_cast<f2 *>(sh_kappa);
    const double s2 = a.s * a.s;
    for (int j = threadIdx.x; j < a.nr; j += blockDim.x) {
        double k = 0.0;
        if (j == 1) k = s2 * a.lo[FCN_IDX(1, a.nr, 31)] * 4.0;
        else if (j >= 2 && j < a.nr - 1) k = s2 * a.lo[FCN_IDX(j, a.nr, 31)] * a.hi[FCN_IDX(j - 1, a.nr, 32)];
        kap[j] = to_f2(k);
    }
    __syncthreads();
    const int nq = a.nt / 2 + 1;
    const int tp = a.tp ? a.tp : nq;
    const int q = blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= nq) return;
    const double delta = a.dk * double(q) * double(q);
    const cx<double> lim = (a.cc || a.pivlim) ? piv_limit(a.s, a.dk, q) : cx<double>{0.0, 0.0};
    if (a.cc) {
        const CdCol<float> c = cd_col<float>(a.s, a.dk, q);
        const float hx = float(lim.x), hy = float(lim.y);
        a.cc[q].lim = make_float4(hx, hy, float(lim.x - double(hx)), float(lim.y - double(hy)));
        a.cc[q].cd = make_float4(c.ah, c.al, c.ih, c.il);
    }
    const f2 by0 = to_f2(4.0 * a.s - delta), by1 = to_f2(2.0 * a.s - delta);
    // the column's pivot limit as double-float pairs (FP64 once per thread:
    // the loop below stays in FP32 arithmetic)
    f2 lx = {0.f, 0.f}, ly = {0.f, 0.f};
    if (a.pivlim) {
        lx = to_f2(lim.x);
        ly = to_f2(lim.y);
    }
    f2 ix = {0.f, 0.f}, iy = {0.f, 0.f};
    const f2 one = {1.f, 0.f};
    for (int j = 0; j < a.nr; ++j) {
        const f2 kp = kap[j];
        const f2 by = (j == 0) ? by0 : ((j < a.nr - 1) ? by1 : f2{0.f, 0.f});
        const f2 wx = df_add(df_mul(kp, ix), one);
        const f2 wy = df_add(df_mul(kp, iy), by);
        const f2 rn = df_recip(df_add(df_mul(wx, wx), df_mul(wy, wy)));
        ix = df_mul(wx, rn);
        iy = df_mul(wy, rn);
        iy = {-iy.h, -iy.l};
        // relative to the column's limit (piv_limit): the hi parts differ
        // exactly where the pivot has settled (Sterbenz), then the lo parts
        const cx<float> e = a.pivlim ? mk((ix.h - lx.h) + (ix.l - lx.l), (iy.h - ly.h) + (iy.l - ly.l))
                                     : mk(ix.h + ix.l, iy.h + iy.l);
        table[FCN_IDX((size_t)j * tp + q, (size_t)a.nr * tp, 30)] = e;
    }
}

// The same table with the rows split into kTabChunks chunks, so that a
// column's recurrence no longer runs down all Nr rows in one thread.  The
// step 1/piv_j = 1/(b_j + kappa_j / piv_{j-1}) is a Moebius map of
// z = 1/piv_{j-1}: z -> (0 z + 1)/(kappa_j z + b_j), i.e. the matrix
// F_j = [[0, 1], [kappa_j, b_j]] acting on (num, den), z = num/den.
//   1. warp c composes its chunk's matrices, G_c = F_{j1-1} ... F_{j0}
//      (double-float complex entries, rescaled by powers of two now and
//      then: z is a ratio, so the common scale is free);
//   2. warp 0 walks the chunks from (num, den) = (0, 1) (1/piv_{-1} = 0),
//      giving each chunk the z that enters it;
//   3. warp c runs the recurrence of cn_table_kernel_f32 over its rows from
//      that z and stores the table.
// The entering z comes from the matrix products instead of the recurrence
// itself, so the two kernels agree to double-float precision (~1e-14), not
// bit for bit.  Lane = frequency bin (32 per CTA).
constexpr int kTabChunks = 16;
struct c2 {
    f2 re, im;
};
__device__ __forceinline__ f2 df_neg(f2 a) { return {-a.h, -a.l}; }
__device__ __forceinline__ f2 df_scale(f2 a, float p2) { return {a.h * p2, a.l * p2}; }   // p2 a power of 2
__device__ __forceinline__ c2 c2_add(c2 a, c2 b) { return {df_add(a.re, b.re), df_add(a.im, b.im)}; }
__device__ __forceinline__ c2 c2_real(f2 k, c2 a) { return {df_mul(k, a.re), df_mul(k, a.im)}; }
// (1 + i by) a
__device__ __forceinline__ c2 c2_b(f2 by, c2 a) {
    return {df_add(a.re, df_neg(df_mul(by, a.im))), df_add(a.im, df_mul(by, a.re))};
}
__device__ __forceinline__ c2 c2_mul(c2 a, c2 b) {
    return {df_add(df_mul(a.re, b.re), df_neg(df_mul(a.im, b.im))), df_add(df_mul(a.re, b.im), df_mul(a.im, b.re))};
}
__device__ __forceinline__ c2 c2_scale(c2 a, float p2) { return {df_scale(a.re, p2), df_scale(a.im, p2)}; }
__device__ __forceinline__ int c2_exp(c2 a) {
    int e = 0;
    frexpf(fmaxf(fabsf(a.re.h), fabsf(a.im.h)), &e);
    return e;
}
// rescales the entries by a common power of two so that the largest is O(1)
__device__ __forceinline__ void c2_norm(c2 *v, int n) {
    int e = -1000;
    for (int k = 0; k < n; ++k)
        if (v[k].re.h != 0.f || v[k].im.h != 0.f) e = max(e, c2_exp(v[k]));
    if (e == -1000 || e == 0) return;
    const float p2 = ldexpf(1.f, -e);
    for (int k = 0; k < n; ++k) v[k] = c2_scale(v[k], p2);
}

__global__ void __launch_bounds__(32 * kTabChunks) cn_table_kernel_f32_chunked(TableArgs a, cx<float> *table) {
    extern __shared__ double sh_tab[];
    f2 *kap = reinterpret_cast<f2 *>(sh_tab);                         // [nr]
    c2 *G = reinterpret_cast<c2 *>(kap + a.nr);                      // [kTabChunks][32][4]
    c2 *Z = G + kTabChunks * 32 * 4;                                 // [kTabChunks][32]
    const double s2 = a.s * a.s;
    for (int j = threadIdx.x; j < a.nr; j += blockDim.x) {
        double k = 0.0;
        if (j == 1) k = s2 * a.lo[FCN_IDX(1, a.nr, 31)] * 4.0;
        else if (j >= 2 && j < a.nr - 1) k = s2 * a.lo[FCN_IDX(j, a.nr, 31)] * a.hi[FCN_IDX(j - 1, a.nr, 32)];
        kap[j] = to_f2(k);
    }
    const int lane = threadIdx.x & 31, c = threadIdx.x >> 5;
    const int nq = a.nt / 2 + 1;
    const int tp = a.tp ? a.tp : nq;
    const int q = blockIdx.x * 32 + lane;
    const bool on = q < nq;
    const int qc = on ? q : nq - 1;             // lanes past the last bin compute bin nq-1, store nothing
    const double delta = a.dk * double(qc) * double(qc);
    const cx<double> lim = (a.cc || a.pivlim) ? piv_limit(a.s, a.dk, qc) : cx<double>{0.0, 0.0};
    if (a.cc && on && c == 0) {
        const CdCol<float> cd = cd_col<float>(a.s, a.dk, q);
        const float hx = float(lim.x), hy = float(lim.y);
        a.cc[q].lim = make_float4(hx, hy, float(lim.x - double(hx)), float(lim.y - double(hy)));
        a.cc[q].cd = make_float4(cd.ah, cd.al, cd.ih, cd.il);
    }
    const f2 by0 = to_f2(4.0 * a.s - delta), by1 = to_f2(2.0 * a.s - delta);
    const f2 zero = {0.f, 0.f}, one = {1.f, 0.f};
    const int L = (a.nr + kTabChunks - 1) / kTabChunks;
    const int j0 = min(a.nr, c * L), j1 = min(a.nr, j0 + L);
    auto by_of = [&](int j) { return (j == 0) ? by0 : ((j < a.nr - 1) ? by1 : zero); };
    __syncthreads();
    {
        // 1. this chunk's matrix
        c2 g[4] = {{one, zero}, {zero, zero}, {zero, zero}, {one, zero}};   // g00 g01 g10 g11
        for (int j = j0; j < j1; ++j) {
            const f2 kp = kap[j], by = by_of(j);
            const c2 n10 = c2_add(c2_real(kp, g[0]), c2_b(by, g[2]));
            const c2 n11 = c2_add(c2_real(kp, g[1]), c2_b(by, g[3]));
            g[0] = g[2];
            g[1] = g[3];
            g[2] = n10;
            g[3] = n11;
            if (((j - j0) & 7) == 7) c2_norm(g, 4);
        }
        c2_norm(g, 4);
        for (int k = 0; k < 4; ++k) G[(c * 32 + lane) * 4 + k] = g[k];
    }
    __syncthreads();
    if (c == 0) {
        // 2. the z entering every chunk
        c2 v[2] = {{zero, zero}, {one, zero}};                                // (num, den)
        for (int k = 0; k < kTabChunks; ++k) {
            const c2 n = v[0], d = v[1];
            const f2 rn = df_recip(df_add(df_mul(d.re, d.re), df_mul(d.im, d.im)));
            const c2 z = c2_mul(n, c2{d.re, df_neg(d.im)});
            Z[k * 32 + lane] = c2{df_mul(z.re, rn), df_mul(z.im, rn)};
            const c2 *gk = G + (k * 32 + lane) * 4;
            v[0] = c2_add(c2_mul(gk[0], n), c2_mul(gk[1], d));
            v[1] = c2_add(c2_mul(gk[2], n), c2_mul(gk[3], d));
            c2_norm(v, 2);
        }
    }
    __syncthreads();
    // 3. the rows of this chunk
    f2 lx = zero, ly = zero;
    if (a.pivlim) {
        lx = to_f2(lim.x);
        ly = to_f2(lim.y);
    }
    const c2 z = Z[c * 32 + lane];
    f2 ix = z.re, iy = z.im;
    for (int j = j0; j < j1; ++j) {
        const f2 kp = kap[j];
        const f2 by = by_of(j);
        const f2 wx = df_add(df_mul(kp, ix), one);
        const f2 wy = df_add(df_mul(kp, iy), by);
        const f2 rn = df_recip(df_add(df_mul(wx, wx), df_mul(wy, wy)));
        ix = df_mul(wx, rn);
        iy = df_mul(wy, rn);
        iy = {-iy.h, -iy.l};
        const cx<float> e = a.pivlim ? mk((ix.h - lx.h) + (ix.l - lx.l), (iy.h - ly.h) + (iy.l - ly.l))
                                     : mk(ix.h + ix.l, iy.h + iy.l);
        if (on) table[FCN_IDX((size_t)j * tp + q, (size_t)a.nr * tp, 30)] = e;
    }
}

// Coefficients of row j in the form rhs_j = d x_j + i (sl x_{j-1} + sh x_{j+1}
// - cd x_j), alpha_j = i sl / piv_j, gamma_j = i sh / piv_j: from the CnCoef
// rows when the launch has them (context tables), else from s and the ratio
// tables (stateless operations).
// With CnCoef rows the FP32 explicit side is two-float (see CnCoef); the
// stateless path forms single-rounded coefficients from s and the tables.
template <typename T>
__device__ __forceinline__ ExRow<T> row_co(const ColArgs<T> &a, int j, T delta, const CdCol<T> &cdc) {
    ExRow<T> r;
    r.sll = r.shl = r.cdl = T(0);
    const int nr = a.nr;
    if (a.coef) {
        const CnCoef<T> cf = j < nr - 1 ? a.coef[FCN_IDX(j, nr, 35)] : CnCoef<T>{};
        r = ex_row(cf, j == 0, cdc);
    } else if (j == 0) {
        r.sl = T(0); r.sh = T(4) * a.s; r.d = T(1); r.cd = T(4) * a.s - delta;
    } else if (j < nr - 1) {
        r.sl = a.s * a.lo[FCN_IDX(j, nr, 35)]; r.sh = a.s * a.hi[FCN_IDX(j, nr, 36)];
        r.d = T(1); r.cd = T(2) * a.s - delta;
    } else {
        r.sl = T(0); r.sh = T(0); r.d = T(0); r.cd = T(0);
    }
    return r;
}

// One CTA solves columns [g C, g C + C) of one pulse; blockDim.x >= C P
// (P = chunks per column), threads beyond C P hold empty chunks.  Every
// thread of the CTA must call it (barriers inside).
template <typename T, int L>
__device__ __forceinline__ void cn_body(const ColArgs<T> &a, int C, int g, unsigned char *smem_raw) {
    const int nwarp = blockDim.x >> 5;
    cx<T> *smA = reinterpret_cast<cx<T> *>(smem_raw);
    cx<T> *smB = smA + nwarp * C;
    cx<T> *smC = smB + nwarp * C;

    const int tid = threadIdx.x;
    const int col = tid % C;
    const int chunk = tid / C;
    const int q = g * C + col;
    const int nt = a.nt, nr = a.nr;
    const int nq = a.tp;
    const int qq = (q <= nt / 2) ? q : nt - q;
    const T delta = a.dk * T(qq) * T(qq);
    CdCol<T> cdc;
    PivLim<T> plim;
    col_consts<T>(a.cc, a.pivlim, a.s64, a.dk64, qq, &cdc, &plim);
    const int j0 = chunk * L;

    cx<T> x[L + 2];
#pragma unroll
    for (int k = 0; k < L + 2; ++k) {
        const int j = j0 - 1 + k;
        x[k] = (j >= 0 && j < nr) ? a.field[FCN_IDX((size_t)j * nt + q, (size_t)nr * nt, 33)] : czero<T>();
    }
    cx<T> inv[L];       // table entries (rhs / pivot by piv_apply)
    cx<T> ivf[L];       // 1/pivot rounded, for the sweep factors
#pragma unroll
    for (int k = 0; k < L; ++k) {
        const int j = j0 + k;
        inv[k] = (j < nr) ? ldg_cx(&a.invden[FCN_IDX((size_t)j * nq + qq, (size_t)nr * nq, 34)]) : czero<T>();
        ivf[k] = (j < nr) ? piv_full(inv[k], plim) : czero<T>();
    }

    // forward sweep, pass 1: beta_j and the chunk map y_end = PA y_in + PB
    cx<T> y[L];
    cx<T> PA = mk(T(1), T(0)), PB = czero<T>();
#pragma unroll
    for (int k = 0; k < L; ++k) {
        const int j = j0 + k;
        if (j < nr) {
            const ExRow<T> c = row_co(a, j, delta, cdc);
            const cx<T> rhs = ex_rhs(c, x[k], x[k + 1], x[k + 2]);
            const cx<T> alpha = cmul_i(ivf[k], c.sl);
            y[k] = piv_apply(rhs, inv[k], plim);
            PB = cmul(alpha, PB) + y[k];
            PA = cmul(alpha, PA);
        } else {
            y[k] = czero<T>();
        }
    }
    // forward sweep, pass 2: exact y from the carry entering the chunk
    {
        cx<T> yp = chunk_scan<T, false>(PA, PB, C, col, smA, smB, smC);
#pragma unroll
        for (int k = 0; k < L; ++k) {
            const int j = j0 + k;
            if (j < nr) {
                const cx<T> alpha = cmul_i(ivf[k], row_co(a, j, delta, cdc).sl);
                y[k] = cmul(alpha, yp) + y[k];
                yp = y[k];
            }
        }
    }
    // backward sweep, pass 1: chunk map x_first = QA x_next + QB
    cx<T> QA = mk(T(1), T(0)), QB = czero<T>();
#pragma unroll
    for (int k = L - 1; k >= 0; --k) {
        const int j = j0 + k;
        if (j < nr) {
            const cx<T> gamma = cmul_i(ivf[k], row_co(a, j, delta, cdc).sh);
            QB = cmul(gamma, QB) + y[k];
            QA = cmul(gamma, QA);
        }
    }
    // backward sweep, pass 2 and store
    {
        cx<T> xn = chunk_scan<T, true>(QA, QB, C, col, smA, smB, smC);
        const DispPhase<T> ph = disp_phase<T>(a.disp, qq);
#pragma unroll
        for (int k = L - 1; k >= 0; --k) {
            const int j = j0 + k;
            if (j < nr) {
                const cx<T> gamma = cmul_i(ivf[k], row_co(a, j, delta, cdc).sh);
                xn = cmul(gamma, xn) + y[k];
                a.field[FCN_IDX((size_t)j * nt + q, (size_t)nr * nt, 37)] = disp_apply(xn, ph);
            }
        }
    }
}

template <typename T, int L>
__global__ void __launch_bounds__(512)
cn_kernel(ColArgs<T> a, int C) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    pdl_enter();
    // CTAs for bins q and Nt - q are launched next to each other
    const int ngroups = a.nt / C;
    const int b = blockIdx.x;
    const int g = (b & 1) ? (ngroups - 1 - (b >> 1)) : (b >> 1);
    cn_body<T, L>(a, C, g, smem_raw);
}

// Batched work list: item = (pulse, column group, C); 512-thread CTAs; a
// persistent grid pulls items from a global counter.
template <typename T, int L>
__global__ void __launch_bounds__(512)
cn_batch_kernel(const ColArgs<T> *__restrict__ pulses, const int4 *__restrict__ items, int nitems,
                unsigned *counter) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ int next;
    for (;;) {
        if (threadIdx.x == 0) next = (int)atomicAdd(counter, 1u);
        __syncthreads();
        const int it = next;
        __syncthreads();
        if (it >= nitems) break;
        const int4 w = items[it];
        const ColArgs<T> a = pulses[w.x];
        cn_body<T, L>(a, w.z, w.y, smem_raw);
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        const unsigned done = atomicAdd(counter + 1, 1u) + 1;
        if (done == gridDim.x) {
            counter[0] = 0;
            counter[1] = 0;
        }
    }
}

// ---------------------------------------------------------------------------
// Staged variant.  Same chunked scan, but each thread first copies its chunk
// (rows j0-1 .. j0+L of its column, and the L pivots) into private
// shared-memory slots with cp.async, so no registers are held by loads in
// flight, and the per-row coefficients come from one CnCoef row instead of
// index tests.  The first sweep turns each slot into what the later sweeps
// need (x_j -> alpha_j, 1/piv_j -> gamma_j), so every later pass is one
// shared-memory load and one complex multiply-add per row.  Slot k of thread
// t sits at k * blockDim + t: consecutive lanes, consecutive words.
// ---------------------------------------------------------------------------

// One complex value global -> shared, asynchronously; valid = false writes
// zeros without reading the source.
template <typename T>
__device__ __forceinline__ void cp_async_cx(cx<T> *dst, const cx<T> *src, bool valid) {
    const unsigned d = (unsigned)__cvta_generic_to_shared(dst);
    const int n = valid ? int(sizeof(cx<T>)) : 0;
    if constexpr (sizeof(cx<T>) == 16)
        asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;\n" ::"r"(d), "l"(src), "r"(n) : "memory");
    else
        asm volatile("cp.async.ca.shared.global [%0], [%1], 8, %2;\n" ::"r"(d), "l"(src), "r"(n) : "memory");
}

template <typename T>
__device__ __forceinline__ void cp_async_cx_full(cx<T> *dst, const cx<T> *src) {
    const unsigned d = (unsigned)__cvta_generic_to_shared(dst);
    if constexpr (sizeof(cx<T>) == 16)
        asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(d), "l"(src) : "memory");
    else
        asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(d), "l"(src) : "memory");
}

__device__ __forceinline__ void cp_async_wait_all() {
    asm volatile("cp.async.commit_group;\ncp.async.wait_group 0;\n" ::: "memory");
}

constexpr size_t kCnStagedSmemMax = 227 * 1024;

// Forward sweep, pass 1, of the register-fed staged variant: x and 1/piv
// are read from global memory straight into registers (the compiler
// hoists the loads of the unrolled loop), alpha_j and gamma_j go to the
// thread's shared-memory slots.  EDGE: the chunk touches row -1 or row nr.
template <typename T, int L, bool EDGE, int NTC>
__device__ __forceinline__ void cn_f1_reg(const ColArgs<T> &a, int q, int qq, int j0, const CdCol<T> &cdc,
                                          const PivLim<T> &plim, cx<T> *At,
                                          cx<T> *Gt, int BD, cx<T> (&y)[L], cx<T> &PA, cx<T> &PB) {
    // NTC: Nt as a compile-time constant (row strides become immediates), 0: a.nt
    const int nt = NTC ? NTC : a.nt, nr = a.nr, nq = a.tp;
    const cx<T> *fx = a.field + q;
    const cx<T> *fi = a.invden + qq;
    auto X = [&](int j) -> cx<T> {
        if (EDGE && (j < 0 || j >= nr)) return czero<T>();
        return ldg_cx(fx + FCN_IDX((size_t)j * nt, (size_t)nr * nt, 51));
    };
    cx<T> xm = X(j0 - 1), x0 = X(j0);
#pragma unroll
    for (int k = 0; k < L; ++k) {
        const int j = j0 + k;
        const cx<T> xp = X(j + 1);
        cx<T> inv = czero<T>();
        if (!EDGE || j < nr) inv = ldg_cx(fi + FCN_IDX((size_t)j * nq, (size_t)nr * nq, 52));
        CnCoef<T> cf;
        if (!EDGE || j < nr - 1) {
            cf = a.coef[FCN_IDX(j, nr, 53)];
        } else {
            cf = CnCoef<T>{};
        }
        const cx<T> rhs = ex_rhs(ex_row(cf, j == 0, cdc), xm, x0, xp);
        const cx<T> beta = piv_apply(rhs, inv, plim);
        const cx<T> ivf = piv_full(inv, plim);
        const cx<T> al = cmul_i(ivf, cf.sl);
        At[k * BD] = al;
        Gt[k * BD] = cmul_i(ivf, cf.sh);
        PB = cmul(al, PB) + beta;
        PA = cmul(al, PA);
        y[k] = beta;
        xm = x0;
        x0 = xp;
    }
}

template <typename T, int L, bool REG, int NTC = 0>
__device__ __forceinline__ void cn_staged_body(const ColArgs<T> &a, int C, int g, unsigned char *smem_raw) {
    const int BD = blockDim.x;
    const int tid = threadIdx.x;
    const int nwarp = BD >> 5;
    cx<T> *smA = reinterpret_cast<cx<T> *>(smem_raw);
    cx<T> *smB = smA + nwarp * C;
    cx<T> *smC = smB + nwarp * C;
    cx<T> *Xt = smC + nwarp * C + tid;          // slot k: Xt[k * BD]
    // staged: L+2 x slots then L pivot slots; register-fed: L alpha slots
    // then L gamma slots
    cx<T> *Gt = Xt + (REG ? L : L + 2) * BD;    // slot k: Gt[k * BD], k = 0 .. L-1

    const int col = tid % C;
    const int chunk = tid / C;
    const int q = g * C + col;
    const int nt = NTC ? NTC : a.nt, nr = a.nr;
    const int nq = a.tp;
    const int qq = (q <= nt / 2) ? q : nt - q;
    CdCol<T> cdc;
    PivLim<T> plim;
    col_consts<T>(a.cc, a.pivlim, a.s64, a.dk64, qq, &cdc, &plim);
    const int j0 = chunk * L;

    cx<T> y[L];
    cx<T> PA = mk(T(1), T(0)), PB = czero<T>();
    // slot of alpha_j: Xt[(k+1) BD] (staged: where x_j was), At[k BD] below
    cx<T> *At = REG ? Xt : Xt + BD;
    if constexpr (REG) {
        if (j0 >= 1 && j0 + L < nr)
            cn_f1_reg<T, L, false, NTC>(a, q, qq, j0, cdc, plim, At, Gt, BD, y, PA, PB);
        else
            cn_f1_reg<T, L, true, NTC>(a, q, qq, j0, cdc, plim, At, Gt, BD, y, PA, PB);
    } else {
    if (j0 >= 1 && j0 + L < nr) {
        // interior chunk: every row j0-1 .. j0+L exists
        const cx<T> *src = a.field + (size_t)(j0 - 1) * nt + q;
#pragma unroll
        for (int k = 0; k < L + 2; ++k) cp_async_cx_full(Xt + k * BD, src + (size_t)k * nt);
        const cx<T> *pv = a.invden + (size_t)j0 * nq + qq;
#pragma unroll
        for (int k = 0; k < L; ++k) cp_async_cx_full(Gt + k * BD, pv + (size_t)k * nq);
    } else {
        // rows outside 0..nr-1 are zero-filled (the source is then not read;
        // the base address stands in for it)
        const cx<T> *src = a.field + (ptrdiff_t)(j0 - 1) * nt + q;
#pragma unroll
        for (int k = 0; k < L + 2; ++k, src += nt) {
            const int j = j0 - 1 + k;
            const bool ok = j >= 0 && j < nr;
            cp_async_cx(Xt + k * BD, ok ? src : a.field, ok);
        }
        const cx<T> *pv = a.invden + (size_t)j0 * nq + qq;
#pragma unroll
        for (int k = 0; k < L; ++k, pv += nq) {
            const bool ok = j0 + k < nr;
            cp_async_cx(Gt + k * BD, ok ? pv : a.invden, ok);
        }
    }
    cp_async_wait_all();

    // forward sweep, pass 1: beta_j, alpha_j, gamma_j and the chunk map
    cx<T> xm = Xt[0], x0 = Xt[BD];
#pragma unroll
    for (int k = 0; k < L; ++k) {
        const int j = j0 + k;
        const cx<T> xp = Xt[(k + 2) * BD];
        const cx<T> inv = Gt[k * BD];
        CnCoef<T> cf;
        if (j < nr - 1) {
            cf = a.coef[FCN_IDX(j, nr, 46)];
        } else {
            cf = CnCoef<T>{};
        }
        const cx<T> rhs = ex_rhs(ex_row(cf, j == 0, cdc), xm, x0, xp);
        const cx<T> beta = piv_apply(rhs, inv, plim);
        const cx<T> ivf = piv_full(inv, plim);
        const cx<T> al = cmul_i(ivf, cf.sl);
        Xt[(k + 1) * BD] = al;                  // x_j (slot k+1) is no longer read
        Gt[k * BD] = cmul_i(ivf, cf.sh);
        PB = cmul(al, PB) + beta;
        PA = cmul(al, PA);
        y[k] = beta;
        xm = x0;
        x0 = xp;
        asm volatile("" ::: "memory");          // keep the slot loads in row order
    }
    }
    // forward sweep, pass 2: exact y from the carry entering the chunk
    {
        cx<T> yp = chunk_scan<T, false>(PA, PB, C, col, smA, smB, smC);
#pragma unroll
        for (int k = 0; k < L; ++k) {
            y[k] = cmul(At[k * BD], yp) + y[k];
            yp = y[k];
            asm volatile("" ::: "memory");
        }
    }
    // backward sweep, pass 1: chunk map x_first = QA x_next + QB
    cx<T> QA = mk(T(1), T(0)), QB = czero<T>();
#pragma unroll
    for (int k = L - 1; k >= 0; --k) {
        const cx<T> ga = Gt[k * BD];
        QB = cmul(ga, QB) + y[k];
        QA = cmul(ga, QA);
        asm volatile("" ::: "memory");
    }
    // backward sweep, pass 2 and store
    cx<T> xn = chunk_scan<T, true>(QA, QB, C, col, smA, smB, smC);
    const DispPhase<T> ph = disp_phase<T>(a.disp, qq);
    cx<T> *fo = a.field + (size_t)j0 * nt + q;
#pragma unroll
    for (int k = L - 1; k >= 0; --k) {
        const int j = j0 + k;
        xn = cmul(Gt[k * BD], xn) + y[k];
        if (j < nr) fo[FCN_IDX((size_t)k * nt, (size_t)(nr - j0) * nt, 47)] = disp_apply(xn, ph);
        asm volatile("" ::: "memory");
    }
}

// Register budget: 3 CTAs of 256 threads per SM for 16-row chunks, 2 CTAs of
// 512 threads for 8-row chunks (the launcher keeps the CTA within this size).
template <typename T, int L>
constexpr int staged_threads() { return L >= 16 ? 256 : 512; }

template <typename T, int L, bool REG, int NTC>
__global__ void __launch_bounds__(staged_threads<T, L>(), L >= 16 ? 3 : 2)
cn_staged_kernel(ColArgs<T> a, int C) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    pdl_enter();
    const int ngroups = a.nt / C;
    const int b = blockIdx.x;
    const int g = (b & 1) ? (ngroups - 1 - (b >> 1)) : (b >> 1);
    cn_staged_body<T, L, REG, NTC>(a, C, g, smem_raw);
}

template <typename T>
__global__ void cn_coef_kernel(TableArgs a, CnCoef<T> *coef) {
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= a.nr) return;
    CnCoef<T> c = CnCoef<T>{};
    if (j < a.nr - 1) {
        // sl, sh from their FP64 values, rounded once; the lo parts hold the
        // rounding errors (zero in FP64)
        const double vl = j == 0 ? 0.0 : a.s * a.lo[j];
        const double vh = j == 0 ? 4.0 * a.s : a.s * a.hi[j];
        c.sl = T(vl);
        c.sh = T(vh);
        c.sll = T(vl - double(c.sl));
        c.shl = T(vh - double(c.sh));
        c.c0 = T((j == 0 ? 4.0 : 2.0) * a.s);
        c.d = T(1);
    }
    coef[j] = c;
}

// Chunk length L; C columns per CTA (one 32-byte sector when the column fits
// the CTA size, fewer for tall grids, more for short ones).  Returns
// cudaErrorInvalidConfiguration when the grid does not fit (the caller then
// falls back to the register variant).
template <typename T, int L, bool REG, int NTC>
cudaError_t launch_cn_staged_l(const ColArgs<T> &a, cudaStream_t st) {
    if (!a.coef) return cudaErrorInvalidConfiguration;
    constexpr int CMIN = 32 / int(sizeof(cx<T>));
    constexpr int TMAX = staged_threads<T, L>();
    const int P = (a.nr + L - 1) / L;
    int C = CMIN;
    while (C > 1 && C * P > TMAX) C /= 2;                 // tall grids: fewer columns
    while (C * 2 * P <= TMAX / 2 && C * 2 <= 32) C *= 2;  // short grids: more columns
    if (C > a.nt) C = a.nt;
    const int threads = ((C * P + 31) / 32) * 32;
    if (threads > TMAX) return cudaErrorInvalidConfiguration;
    const size_t slots = REG ? 2 * L : 2 * L + 2;
    const size_t smem = sizeof(cx<T>) * (3 * (size_t)(threads / 32) * C + slots * threads);
    if (smem > kCnStagedSmemMax) return cudaErrorInvalidConfiguration;
    return launch_k(cn_staged_kernel<T, L, REG, NTC>, dim3(a.nt / C), dim3(threads), smem, st, a, C);
}

template <typename T, int L>
cudaError_t launch_cn_l(const ColArgs<T> &a, int target, cudaStream_t st) {
    constexpr int CMIN = 32 / int(sizeof(cx<T>));   // one 32-byte sector of columns
    const int P = (a.nr + L - 1) / L;
    int C = CMIN;
    while (C * 2 * P <= target && C * 2 <= 32) C *= 2;
    if (C > a.nt) C = a.nt;
    // whole warps: chunks beyond P are empty (identity maps)
    const int threads = ((C * P + 31) / 32) * 32;
    if (threads > 512) return cudaErrorInvalidConfiguration;
    const size_t smem = sizeof(cx<T>) * 3 * (size_t)(threads / 32) * C;
    const int grid = a.nt / C;
    return launch_k(cn_kernel<T, L>, dim3(grid), dim3(threads), smem, st, a, C);
}

// ---------------------------------------------------------------------------
// Paired variant: one CTA solves the same column group of two pulses that
// share the grid and the pivot table (a batch of equal pulses).  The pivots,
// alpha_j, gamma_j, the row coefficients and the A part of every chunk map
// are the same for both; each thread runs the two pulses' recurrences side by
// side (two independent dependency chains).  Register-fed, chunks of L rows.
// ---------------------------------------------------------------------------


template <typename T, int L, bool EDGE, int NTC>
__device__ __forceinline__ void cn_f1_pair(const ColArgs<T> &a, const cx<T> *f2, int q, int qq, int j0,
                                           const CdCol<T> &cdc, const PivLim<T> &plim, cx<T> *At, cx<T> *Gt,
                                           int BD, cx<T> (&y1)[L],
                                           cx<T> (&y2)[L], cx<T> &PA, cx<T> &PB1, cx<T> &PB2) {
    const int nt = NTC ? NTC : a.nt, nr = a.nr, nq = a.tp;
    const cx<T> *fx = a.field + q;
    const cx<T> *fy = f2 + q;
    const cx<T> *fi = a.invden + qq;
    auto X = [&](const cx<T> *f, int j) -> cx<T> {
        if (EDGE && (j < 0 || j >= nr)) return czero<T>();
        return ldg_cx(f + FCN_IDX((size_t)j * nt, (size_t)nr * nt, 60));
    };
    cx<T> xm1 = X(fx, j0 - 1), x01 = X(fx, j0);
    cx<T> xm2 = X(fy, j0 - 1), x02 = X(fy, j0);
#pragma unroll
    for (int k = 0; k < L; ++k) {
        const int j = j0 + k;
        const cx<T> xp1 = X(fx, j + 1), xp2 = X(fy, j + 1);
        cx<T> inv = czero<T>();
        if (!EDGE || j < nr) inv = ldg_cx(fi + FCN_IDX((size_t)j * nq, (size_t)nr * nq, 61));
        CnCoef<T> cf;
        if (!EDGE || j < nr - 1) {
            cf = a.coef[FCN_IDX(j, nr, 62)];
        } else {
            cf = CnCoef<T>{};
        }
        const ExRow<T> e = ex_row(cf, j == 0, cdc);
        const cx<T> ivf = piv_full(inv, plim);
        const cx<T> al = cmul_i(ivf, cf.sl);
        At[k * BD] = al;
        Gt[k * BD] = cmul_i(ivf, cf.sh);
        {
            const cx<T> beta = piv_apply(ex_rhs(e, xm1, x01, xp1), inv, plim);
            PB1 = cmul(al, PB1) + beta;
            y1[k] = beta;
        }
        {
            const cx<T> beta = piv_apply(ex_rhs(e, xm2, x02, xp2), inv, plim);
            PB2 = cmul(al, PB2) + beta;
            y2[k] = beta;
        }
        PA = cmul(al, PA);
        xm1 = x01; x01 = xp1;
        xm2 = x02; x02 = xp2;
    }
}

template <typename T, int L, int NTC>
__device__ __forceinline__ void cn_pair_body(const ColArgs<T> &a, cx<T> *field2, int C, int g,
                                             unsigned char *smem_raw) {
    const int BD = blockDim.x;
    const int tid = threadIdx.x;
    const int nwarp = BD >> 5;
    cx<T> *smA = reinterpret_cast<cx<T> *>(smem_raw);
    cx<T> *smB = smA + nwarp * C;
    cx<T> *smC = smB + 2 * nwarp * C;
    cx<T> *At = smC + 2 * nwarp * C + tid;     // alpha slot k: At[k * BD]
    cx<T> *Gt = At + L * BD;                   // gamma slot k: Gt[k * BD]

    const int col = tid % C;
    const int chunk = tid / C;
    const int q = g * C + col;
    const int nt = NTC ? NTC : a.nt, nr = a.nr;
    const int qq = (q <= nt / 2) ? q : nt - q;
    CdCol<T> cdc;
    PivLim<T> plim;
    col_consts<T>(a.cc, a.pivlim, a.s64, a.dk64, qq, &cdc, &plim);
    const int j0 = chunk * L;

    cx<T> y1[L], y2[L];
    cx<T> PA = mk(T(1), T(0)), PB[2] = {czero<T>(), czero<T>()};
    if (j0 >= 1 && j0 + L < nr)
        cn_f1_pair<T, L, false, NTC>(a, field2, q, qq, j0, cdc, plim, At, Gt, BD, y1, y2, PA, PB[0], PB[1]);
    else
        cn_f1_pair<T, L, true, NTC>(a, field2, q, qq, j0, cdc, plim, At, Gt, BD, y1, y2, PA, PB[0], PB[1]);
    {
        cx<T> yp[2];
        chunk_scan_n<T, false, 2>(PA, PB, C, col, smA, smB, smC, yp);
#pragma unroll
        for (int k = 0; k < L; ++k) {
            const cx<T> al = At[k * BD];
            y1[k] = cmul(al, yp[0]) + y1[k];
            y2[k] = cmul(al, yp[1]) + y2[k];
            yp[0] = y1[k];
            yp[1] = y2[k];
            asm volatile("" ::: "memory");
        }
    }
    cx<T> QA = mk(T(1), T(0)), QB[2] = {czero<T>(), czero<T>()};
#pragma unroll
    for (int k = L - 1; k >= 0; --k) {
        const cx<T> ga = Gt[k * BD];
        QB[0] = cmul(ga, QB[0]) + y1[k];
        QB[1] = cmul(ga, QB[1]) + y2[k];
        QA = cmul(ga, QA);
        asm volatile("" ::: "memory");
    }
    cx<T> xn[2];
    chunk_scan_n<T, true, 2>(QA, QB, C, col, smA, smB, smC, xn);
    const DispPhase<T> ph = disp_phase<T>(a.disp, qq);
    cx<T> *fo1 = a.field + (size_t)j0 * nt + q;
    cx<T> *fo2 = field2 + (size_t)j0 * nt + q;
#pragma unroll
    for (int k = L - 1; k >= 0; --k) {
        const int j = j0 + k;
        const cx<T> ga = Gt[k * BD];
        xn[0] = cmul(ga, xn[0]) + y1[k];
        xn[1] = cmul(ga, xn[1]) + y2[k];
        if (j < nr) {
            fo1[FCN_IDX((size_t)k * nt, (size_t)(nr - j0) * nt, 63)] = disp_apply(xn[0], ph);
            fo2[FCN_IDX((size_t)k * nt, (size_t)(nr - j0) * nt, 64)] = disp_apply(xn[1], ph);
        }
        asm volatile("" ::: "memory");
    }
}

// One 512-thread CTA per SM: the two pulses' registers (126 per thread) fit
// without spills, which measured faster than two CTAs at 64 registers.
template <typename T, int L, int NTC>
__global__ void __launch_bounds__(512, 1)
cn_pair_kernel(ColArgs<T> a, cx<T> *field2, int C) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    pdl_enter();
    const int ngroups = a.nt / C;
    const int b = blockIdx.x;
    const int g = (b & 1) ? (ngroups - 1 - (b >> 1)) : (b >> 1);
    cn_pair_body<T, L, NTC>(a, field2, C, g, smem_raw);
}

template <typename T, int L, int NTC>
cudaError_t launch_cn_pair_l(const ColArgs<T> &a, cx<T> *field2, cudaStream_t st) {
    if (!a.coef) return cudaErrorInvalidConfiguration;
    constexpr int CMIN = 32 / int(sizeof(cx<T>));
    constexpr int TMAX = 512;
    const int P = (a.nr + L - 1) / L;
    int C = CMIN;
    while (C > 1 && C * P > TMAX) C /= 2;
    while (C * 2 * P <= TMAX / 2 && C * 2 <= 32) C *= 2;
    if (C > a.nt) C = a.nt;
    const int threads = ((C * P + 31) / 32) * 32;
    if (threads > TMAX) return cudaErrorInvalidConfiguration;
    const size_t smem = sizeof(cx<T>) * (5 * (size_t)(threads / 32) * C + 2 * (size_t)L * threads);
    if (smem > kCnStagedSmemMax) return cudaErrorInvalidConfiguration;
    return launch_k(cn_pair_kernel<T, L, NTC>, dim3(a.nt / C), dim3(threads), smem, st, a, field2, C);
}

// The column kernels keep the driver's carveout choice: forcing the largest
// shared-memory carveout (the row kernels') measured slower, as the column
// stage's loads lean on L1.
template <typename Kern>
cudaError_t set_col_attrs(Kern k) {
    return cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kCnStagedSmemMax);
}

template <typename T, int L, int NTC>
cudaError_t set_pair_attr() {
    return set_col_attrs(cn_pair_kernel<T, L, NTC>);
}

// Register-fed variant with Nt as a compile-time constant for the grids of
// 512 .. 8192 points in FP32 (every row offset an immediate), generic otherwise.
template <typename T, int L>
cudaError_t launch_cn_reg_nt(const ColArgs<T> &a, cudaStream_t st) {
    if constexpr (sizeof(T) == 4) {
        switch (a.nt) {
            case 512: return launch_cn_staged_l<T, L, true, 512>(a, st);
            case 1024: return launch_cn_staged_l<T, L, true, 1024>(a, st);
            case 2048: return launch_cn_staged_l<T, L, true, 2048>(a, st);
            case 4096: return launch_cn_staged_l<T, L, true, 4096>(a, st);
            case 8192: return launch_cn_staged_l<T, L, true, 8192>(a, st);
            default: break;
        }
    }
    return launch_cn_staged_l<T, L, true, 0>(a, st);
}

template <typename T, int L, bool REG, int NTC>
cudaError_t set_staged_attr() {
    return set_col_attrs(cn_staged_kernel<T, L, REG, NTC>);
}

}  // namespace

// Variants: bit 0 selects the shorter chunk (more threads, fewer registers
// per thread), bit 1 a target CTA size of 512 instead of 256 threads.  A
// variant that does not fit (more than 512 threads) falls back to variant 0.
template <typename T>
cudaError_t launch_cn(const ColArgs<T> &a_in, cudaStream_t st) {
    constexpr int LL = sizeof(T) == 4 ? 16 : 8;     // long chunk
    constexpr int LS = LL / 2;                      // short chunk
    ColArgs<T> a = a_in;
    if (!a.tp) a.tp = a.nt / 2 + 1;
    const int target = (a.variant & 2) ? 512 : 256;
    cudaError_t e = cudaErrorInvalidConfiguration;
    if (a.variant == kColSeq) {
        cx<T> *f = a.field;
        e = launch_cn_seq<T>(a, &f, 1, st);
        if (e != cudaErrorInvalidConfiguration) return e;
        a.variant = kColStagedFirst + 3;            // not supported here: register-fed
    }
    if (a.variant >= kColStagedFirst) {
        switch (a.variant - kColStagedFirst) {
            case 0: e = launch_cn_staged_l<T, LL, false, 0>(a, st); break;
            case 1: e = launch_cn_staged_l<T, LS, false, 0>(a, st); break;
            case 2: e = launch_cn_reg_nt<T, LL>(a, st); break;
            default: e = launch_cn_reg_nt<T, LS>(a, st); break;
        }
        if (e != cudaErrorInvalidConfiguration) return e;
    }
    if (a.variant < kColStagedFirst && (a.variant & 1)) e = launch_cn_l<T, LS>(a, target, st);
    if (e == cudaErrorInvalidConfiguration) e = launch_cn_l<T, LL>(a, target, st);
    if (e == cudaErrorInvalidConfiguration) e = launch_cn_l<T, LL>(a, 256, st);
    return e;
}

template <typename T>
cudaError_t launch_cn_pair(const ColArgs<T> &a_in, cx<T> *field2, cudaStream_t st) {
    constexpr int L = 8;
    ColArgs<T> a = a_in;
    if (!a.tp) a.tp = a.nt / 2 + 1;
    if (a.variant == kColSeq) {
        cx<T> *f[2] = {a.field, field2};
        const cudaError_t e = launch_cn_seq<T>(a, f, 2, st);
        if (e != cudaErrorInvalidConfiguration) return e;
    }
    if constexpr (sizeof(T) == 4) {
        switch (a.nt) {
            case 512: return launch_cn_pair_l<T, L, 512>(a, field2, st);
            case 1024: return launch_cn_pair_l<T, L, 1024>(a, field2, st);
            case 2048: return launch_cn_pair_l<T, L, 2048>(a, field2, st);
            case 4096: return launch_cn_pair_l<T, L, 4096>(a, field2, st);
            case 8192: return launch_cn_pair_l<T, L, 8192>(a, field2, st);
            default: break;
        }
    }
    return launch_cn_pair_l<T, L, 0>(a, field2, st);
}

template <typename T>
cudaError_t launch_cn_coef(const TableArgs &a, CnCoef<T> *coef, cudaStream_t st) {
    cn_coef_kernel<T><<<(a.nr + 127) / 128, 128, 0, st>>>(a, coef);
    return cudaGetLastError();
}

template <typename T>
cudaError_t prepare_cn() {
    constexpr int LL = sizeof(T) == 4 ? 16 : 8, LS = LL / 2;
    cudaError_t e = set_staged_attr<T, LL, false, 0>();
    if (e == cudaSuccess) e = set_staged_attr<T, LS, false, 0>();
    if (e == cudaSuccess) e = set_staged_attr<T, LL, true, 0>();
    if (e == cudaSuccess) e = set_staged_attr<T, LS, true, 0>();
    if (e == cudaSuccess) e = set_pair_attr<T, 8, 0>();
    if constexpr (sizeof(T) == 4) {
        if (e == cudaSuccess) e = set_pair_attr<T, 8, 512>();
        if (e == cudaSuccess) e = set_pair_attr<T, 8, 1024>();
        if (e == cudaSuccess) e = set_pair_attr<T, 8, 2048>();
        if (e == cudaSuccess) e = set_pair_attr<T, 8, 4096>();
        if (e == cudaSuccess) e = set_pair_attr<T, 8, 8192>();
        if (e == cudaSuccess) e = set_staged_attr<T, LL, true, 512>();
        if (e == cudaSuccess) e = set_staged_attr<T, LS, true, 512>();
        if (e == cudaSuccess) e = set_staged_attr<T, LL, true, 1024>();
        if (e == cudaSuccess) e = set_staged_attr<T, LS, true, 1024>();
        if (e == cudaSuccess) e = set_staged_attr<T, LL, true, 2048>();
        if (e == cudaSuccess) e = set_staged_attr<T, LS, true, 2048>();
        if (e == cudaSuccess) e = set_staged_attr<T, LL, true, 4096>();
        if (e == cudaSuccess) e = set_staged_attr<T, LS, true, 4096>();
        if (e == cudaSuccess) e = set_staged_attr<T, LL, true, 8192>();
        if (e == cudaSuccess) e = set_staged_attr<T, LS, true, 8192>();
    }
    return e;
}

template <typename T>
cudaError_t launch_cn_table(const TableArgs &a, cx<T> *table, cudaStream_t st) {
    const int nq = a.nt / 2 + 1;
    const int threads = 32;   // spread the latency-bound recurrences over many SMs
    if constexpr (sizeof(T) == 4) {
        if (a.nr >= 128) {
            // rows in chunks (cn_table_kernel_f32_chunked): the serial
            // recurrence down a tall column is the cost of a table
            const size_t smem = sizeof(f2) * a.nr + sizeof(c2) * kTabChunks * 32 * 5;
            static std::once_flag once;
            static cudaError_t attr = cudaSuccess;
            std::call_once(once, [] {
                attr = cudaFuncSetAttribute(cn_table_kernel_f32_chunked, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                            (int)(sizeof(f2) * 4096 + sizeof(c2) * kTabChunks * 32 * 5));
            });
            if (attr != cudaSuccess) return attr;
            if (a.nr > 4096) return cudaErrorInvalidValue;
            cn_table_kernel_f32_chunked<<<(nq + 31) / 32, 32 * kTabChunks, smem, st>>>(a, table);
        } else {
            cn_table_kernel_f32<<<(nq + threads - 1) / threads, threads, sizeof(double) * a.nr, st>>>(a, table);
        }
    } else
        cn_table_kernel<T><<<(nq + threads - 1) / threads, threads, sizeof(double) * 2 * a.nr, st>>>(a, table);
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_cn_batch(const ColArgs<T> *pulses, const int4 *items, int nitems, unsigned *counter,
                            int grid, cudaStream_t st) {
    constexpr int L = sizeof(T) == 4 ? 16 : 8;
    const size_t smem = sizeof(cx<T>) * 3 * 16 * 32;     // 16 warps x C <= 32 x 3 maps
    cn_batch_kernel<T, L><<<grid, 512, smem, st>>>(pulses, items, nitems, counter);
    return cudaGetLastError();
}

template cudaError_t launch_cn<float>(const ColArgs<float> &, cudaStream_t);
template cudaError_t launch_cn_batch<float>(const ColArgs<float> *, const int4 *, int, unsigned *, int,
                                            cudaStream_t);
template cudaError_t launch_cn<double>(const ColArgs<double> &, cudaStream_t);
template cudaError_t launch_cn_table<float>(const TableArgs &, cx<float> *, cudaStream_t);
template cudaError_t launch_cn_coef<float>(const TableArgs &, CnCoef<float> *, cudaStream_t);
template cudaError_t launch_cn_coef<double>(const TableArgs &, CnCoef<double> *, cudaStream_t);
template cudaError_t prepare_cn<float>();
template cudaError_t launch_cn_pair<float>(const ColArgs<float> &, cx<float> *, cudaStream_t);
template cudaError_t launch_cn_pair<double>(const ColArgs<double> &, cx<double> *, cudaStream_t);
template cudaError_t prepare_cn<double>();
template cudaError_t launch_cn_table<double>(const TableArgs &, cx<double> *, cudaStream_t);

}  // namespace fcn
