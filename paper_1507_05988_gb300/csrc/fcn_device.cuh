// fcn_device.cuh -- device types and kernel launch interfaces of the GB300
// FCN z-step (Ma & Lin, arXiv:1507.05988, Sec. 3).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>
#include <cstdlib>

// Optional self-checking build (-DFCN_CHECKED, used to locate memory faults):
// every indexed access in the kernels goes through FCN_IDX, which prints the
// site and index of the first violations and redirects the access to index 0
// instead of leaving the buffer.  Off by default (FCN_IDX is the identity).
#ifdef FCN_CHECKED
#include <cstdio>
static __device__ int g_fcn_reports;
__device__ __forceinline__ long long fcn_chk(long long i, long long n, int site) {
    if (i < 0 || i >= n) {
        if (atomicAdd(&g_fcn_reports, 1) < 16)
            printf("FCN_CHECK site %d index %lld size %lld block %d thread %d\n", site, i, n,
                   (int)blockIdx.x, (int)threadIdx.x);
        return 0;
    }
    return i;
}
#define FCN_IDX(i, n, site) fcn_chk((long long)(i), (long long)(n), (site))
#else
#define FCN_IDX(i, n, site) (i)
#endif

namespace fcn {

// Interleaved complex value; 8-byte aligned for float, 16 for double so that
// one complex moves in one vector load/store.
template <typename T>
struct alignas(2 * sizeof(T)) cx {
    T x, y;
};

template <typename T>
__host__ __device__ __forceinline__ cx<T> mk(T x, T y) { cx<T> r; r.x = x; r.y = y; return r; }
template <typename T>
__device__ __forceinline__ cx<T> operator+(cx<T> a, cx<T> b) { return mk(a.x + b.x, a.y + b.y); }
template <typename T>
__device__ __forceinline__ cx<T> operator-(cx<T> a, cx<T> b) { return mk(a.x - b.x, a.y - b.y); }
template <typename T>
__device__ __forceinline__ cx<T> cmul(cx<T> a, cx<T> b) {
    return mk(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
template <typename T>
__device__ __forceinline__ cx<T> cscale(cx<T> a, T s) { return mk(a.x * s, a.y * s); }
// a * (i s) for real s
template <typename T>
__device__ __forceinline__ cx<T> cmul_i(cx<T> a, T s) { return mk(-a.y * s, a.x * s); }
template <typename T>
__device__ __forceinline__ T cnorm(cx<T> a) { return a.x * a.x + a.y * a.y; }

// Programmatic dependent launch of the z-step kernels (off unless the
// environment has FCN_PDL=1).  Each kernel first lets the next kernel of its
// stream be scheduled (which happens once every CTA of this kernel has
// started, so the next kernel's CTAs only take the slots this one frees in
// its last wave), then waits until its predecessor has completed and its
// memory is visible, before any access.  Launched without the attribute,
// both instructions return at once.  Measured on the 1024 x 4096 pulses it
// is slower (column CTAs placed early on SMs that still hold row CTAs run
// with the row kernel's small L1), hence off by default.
__device__ __forceinline__ void pdl_enter() {
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
    asm volatile("griddepcontrol.wait;" ::: "memory");
}

inline bool pdl_enabled() {
    static const bool on = [] {
        const char *e = std::getenv("FCN_PDL");
        return e && e[0] == '1';
    }();
    return on;
}

template <typename... KArgs, typename... Args>
cudaError_t launch_k(void (*kernel)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t st,
                     Args... args) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    at[0].val.programmaticStreamSerializationAllowed = pdl_enabled() ? 1 : 0;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, kernel, args...);
}

// Read-only cached load of one complex value.
__device__ __forceinline__ cx<float> ldg_cx(const cx<float> *p) {
    const float2 v = __ldg(reinterpret_cast<const float2 *>(p));
    return mk(v.x, v.y);
}
__device__ __forceinline__ cx<double> ldg_cx(const cx<double> *p) {
    const double2 v = __ldg(reinterpret_cast<const double2 *>(p));
    return mk(v.x, v.y);
}

// Physics switches (same bits as the C-ABI).
enum : unsigned {
    PH_DIFFRACTION = 1u, PH_DISPERSION = 2u, PH_KERR = 4u, PH_PLASMA = 8u,
    PH_MPI = 16u, PH_MPI_SAT = 32u
};

// Row-stage operations (same bits as the C-ABI FCN_OP_*), plus internal ones.
enum : int {
    OP_IFFT = 1, OP_NL = 2, OP_NL2 = 4, OP_FFT = 8, OP_RHO = 16,
    OP_STATS = 32,   // per-row FP64 statistics of the final time-domain row
    OP_SPEC = 64,    // spectral moments of the final time-domain row (no store)
    OP_NOSTORE = 128, // do not write the field back (diagnostics only)
    // with OP_FFT | OP_SPEC: store the time-domain row as without OP_FFT and
    // transform it only for the spectral moments (the spectrum is not stored)
    OP_SPEC_OF_TIME = 256,
    // with the time-domain store: the step-doubling norm's per-row sums
    // against RowArgs::cmp into RowArgs::diff (diff[2m] = sum |cmp - A|^2,
    // diff[2m+1] = sum |A|^2 over row m of the stored field A)
    OP_DIFF = 512
};

// Coefficients of one nonlinear half step in scaled intensity units
// Ihat = I / I_s (I_s a power of two, so the scaling is exact).
//   phase rate  = sum_j kerr[j] Ihat^(j+1) - plasma * u        [rad/m]
//   loss rate   = loss * Ihat^(K-1) [* (1 - u)]                [1/m]
//   RK4 step of u = rho/rho_nt along tau uses x = sdt * Ihat^K (= dtau w)
template <typename T>
struct NLCoef {
    T h;        // half-step length dz/2 [m]
    T kerr[4];  // (k0/n0) n_2j I_s^j
    T plasma;   // k0/(2 n0^2 rho_c) rho_nt
    T loss;     // (beta_K/2) I_s^(K-1)
    T sdt;      // sigma_K dtau I_s^K
    T inv_is;   // 1 / I_s
    T inv_nt;   // 1 / Nt (applied after the inverse FFT)
    T rho_nt;   // rho = u rho_nt for the rho output
    // The same terms as the row kernel uses them, with the half-step length
    // and the physics switches folded in (a switched-off term has a zero
    // coefficient, so the kernel needs no per-point flag tests):
    T hk[4];    // h kerr_j, or 0 without the Kerr term
    T hplasma;  // h plasma, or 0 without plasma defocusing
    T hloss;    // h loss, or 0 without MPI loss
    T sat;      // 1 with saturation of the MPI loss (factor 1 - u), else 0
    T is_root;  // sdt^(1/K) / I_s: with j = |A|^2 is_root, sdt (|A|^2/I_s)^K = j^K
    int K;
    int nkerr;  // number of leading Kerr orders in use (1..4; trailing zeros dropped)
    unsigned flags;
};

// Pass structure of the row stage's in-place FFT of Nt points and the layout
// of its twiddle table.  Two decompositions (plans), chosen per grid by the
// autotuner through the row variant; the last pass is radix 16 in both (a
// thread's 16 consecutive samples then sit at one position stride):
//   plan 0: one radix 2/4/8 pass first for the factor left over by radix 16,
//           then radix-16 passes (Nt = 4096: 16 16 16);
//   plan 1 (Nt >= 256): radix-8 passes, one radix 2/4 pass first for the
//           factor left over, then the radix-16 pass (Nt = 4096: 4 8 8 16).
// Nt < 16: one pass of radix Nt.  A kernel's Nt template argument carries
// the plan in its high bits (fft_tag); fft_nt / fft_plan decode it.
// Twiddle table: for every pass p >= 1 (radix R_p, Ns_p = product of the
// earlier radices) one block of (R_p - 1) Ns_p factors, entry (r - 1) Ns_p +
// k = W^(r k Nt / (Ns_p R_p)), W = exp(-2 pi i / Nt), r = 1..R_p-1,
// k = 0..Ns_p-1: the threads of a warp (consecutive k) read consecutive
// entries.  An FP32 entry is a two-float pair (hi, lo) of complex floats,
// 16 bytes; an FP64 entry one complex double.
constexpr int kFftPlanShift = 20;
__host__ __device__ constexpr int fft_tag(int nt, int plan) { return nt | (plan << kFftPlanShift); }
__host__ __device__ constexpr int fft_nt(int ntp) { return ntp & ((1 << kFftPlanShift) - 1); }
__host__ __device__ constexpr int fft_plan(int ntp) { return ntp >> kFftPlanShift; }
__host__ __device__ constexpr int fft_log2(int n) { return n <= 1 ? 0 : 1 + fft_log2(n / 2); }
__host__ __device__ constexpr int fft_n16(int nt) { return nt >= 16 ? fft_log2(nt) / 4 : 0; }
__host__ __device__ constexpr int fft_rem(int nt) { return nt >= 16 ? (1 << (fft_log2(nt) % 4)) : nt; }
// plan 1: m = log2(Nt/16) radix-2 factors before the radix-16 pass, as
// radix-8 passes and a radix 2^(m mod 3) pass first
__host__ __device__ constexpr int fft_m8(int nt) { return fft_log2(nt) - 4; }
__host__ __device__ constexpr bool fft_plan1(int ntp) { return fft_plan(ntp) == 1 && fft_nt(ntp) >= 256; }
__host__ __device__ constexpr int fft_npass(int ntp) {
    return fft_plan1(ntp) ? (fft_m8(fft_nt(ntp)) % 3 ? 1 : 0) + fft_m8(fft_nt(ntp)) / 3 + 1
                          : fft_n16(fft_nt(ntp)) + (fft_rem(fft_nt(ntp)) > 1 ? 1 : 0);
}
__host__ __device__ constexpr int fft_radix(int ntp, int p) {
    return fft_nt(ntp) < 16 ? fft_nt(ntp)
         : fft_plan1(ntp)
             ? (p == fft_npass(ntp) - 1 ? 16
                : ((fft_m8(fft_nt(ntp)) % 3 && p == 0) ? (1 << (fft_m8(fft_nt(ntp)) % 3)) : 8))
             : ((fft_rem(fft_nt(ntp)) > 1 && p == 0) ? fft_rem(fft_nt(ntp)) : 16);
}
__host__ __device__ constexpr int fft_ns(int ntp, int p) {
    int ns = 1;
    for (int q = 0; q < p; ++q) ns *= fft_radix(ntp, q);
    return ns;
}
__host__ __device__ constexpr int tw_offset(int nt, int p) {
    int o = 0;
    for (int q = 1; q < p; ++q) o += (fft_radix(nt, q) - 1) * fft_ns(nt, q);
    return o;
}
__host__ __device__ constexpr int tw_size(int nt) { return tw_offset(nt, fft_npass(nt)); }

// Statistics written per row by the row stage (FP64).
enum : int {
    ST_SUM_I = 0,   // sum_p |A|^2
    ST_MAX_I = 1,   // max_p |A|^2
    ST_MAX_U = 2,   // max_p rho/rho_nt of the last half step
    ST_NONFINITE = 3,
    ST_S0 = 4,      // sum_q |A~_q|^2
    ST_S1 = 5,      // sum_q omega_q |A~_q|^2 (omega in units of domega)
    ST_S2 = 6,      // sum_q omega_q^2 |A~_q|^2
    NSTAT = 8
};

// One row-stage work item list entry (batched launches): rows [row0, row0+nrows)
// of the pulse whose field starts at `field`.
template <typename T>
struct RowArgs {
    cx<T> *field;         // [nr][nt]
    const cx<T> *tw;      // twiddle table of FFT plan 0 (layout: tw_offset)
    T *rho;               // [nr][nt] or null
    double *stats;        // [nr][NSTAT] or null
    int nr;
    int nt;
    int ops;
    int variant;          // 0..2: occupancy variants; 3: persistent, next rows
                          // prefetched by bulk copies (FP32, K = 8, Nt >= 512);
                          // 4, 5: FFT plan 1 (radix-8 passes) with the
                          // occupancy of variants 1, 2 (FP32, K = 8, Nt >= 256);
                          // chosen by the autotuner
    NLCoef<T> nl;
    int *err = nullptr;   // set nonzero by a kernel whose bounded wait gave up
    const cx<T> *tw1 = nullptr;   // twiddle table of FFT plan 1 (variants 4, 5)
    const cx<T> *in = nullptr;    // rows read from here instead of field (output
                                  // still to field; may not alias it), or null
    const cx<T> *cmp = nullptr;   // OP_DIFF: the field compared against, [nr][nt]
    double *diff = nullptr;       // OP_DIFF: per-row sums, [nr][2]
};

// One launch of the row stage over up to kRowMulti pulses that share the
// grid, the coefficients and the kernel variant: a's own field, rho and
// stats are ignored; pulse y (blockIdx.y) uses field[y], rho[y], stats[y].
constexpr int kRowMulti = 8;
template <typename T>
struct RowMultiArgs {
    RowArgs<T> a;
    cx<T> *field[kRowMulti];
    T *rho[kRowMulti];
    double *stats[kRowMulti];
    const cx<T> *in[kRowMulti] = {};   // per pulse as RowArgs::in (null: field)
    const cx<T> *cmp[kRowMulti] = {};  // per pulse as RowArgs::cmp
    double *diff[kRowMulti] = {};      // per pulse as RowArgs::diff
};

// Per-row coefficients of the Crank-Nicolson system (Eqs. (Ma)-(Mb)) for one
// dz, in the form the column kernels use: with delta_q = dk q^2,
//   explicit side  w_j = sl x_{j-1} + sh x_{j+1} - d (c0 - delta_q) x_j,
//                  rhs_j = d x_j + i w_j,
//   sweep factors  alpha_j = i sl / piv_j,  gamma_j = i sh / piv_j.
// Row 0 (symmetry axis): sl = 0, sh = c0 = 4s, d = 1; rows 1..Nr-2:
// sl = s lo_j, sh = s hi_j, c0 = 2s, d = 1; the boundary row Nr-1 and the
// padding rows of a ragged last chunk are all zero (A = 0 there).
//
// In FP32 the explicit side takes every coefficient as a two-float pair
// (hi + lo, lo = the FP32 rounding error of the FP64 value): rounded once,
// sl, sh and c0 - delta_q would perturb the discrete operator itself by
// ~6e-8 the same way at every z-step, an error that adds up coherently
// over a run (it was the largest systematic FP32 error of a step).  sll and
// shl hold the lo parts of sl and sh; the pair of c0 - delta_q is formed per
// column from the FP64 s and dk (CdCol).  The sweep factors keep sl and sh.
template <typename T>
struct alignas(8 * sizeof(T)) CnCoef {
    T sl, sh, c0, d;
    T sll, shl, pad0, pad1;
};

// c0 - delta_q of one column as two-float pairs, for the axis row (c0 = 4s)
// and the interior rows (c0 = 2s); in FP64 the lo parts are zero.
template <typename T>
struct CdCol {
    T ah, al, ih, il;
};
template <typename T>
__device__ __forceinline__ CdCol<T> cd_col(double s, double dk, int qq) {
    const double dl = dk * double(qq) * double(qq);
    const double a = 4.0 * s - dl, i = 2.0 * s - dl;
    CdCol<T> c;
    c.ah = T(a);
    c.ih = T(i);
    c.al = T(a - double(c.ah));
    c.il = T(i - double(c.ih));
    return c;
}

// The explicit side of one row: sl, sh, cd = d (c0 - delta_q) and their lo
// parts (all zero in FP64 and for rows without a CnCoef row).
template <typename T>
struct ExRow {
    T sl, sh, cd, d, sll, shl, cdl;
};
template <typename T>
__device__ __forceinline__ ExRow<T> ex_row(const CnCoef<T> &cf, bool axis, const CdCol<T> &c) {
    ExRow<T> e;
    e.sl = cf.sl;
    e.sh = cf.sh;
    e.d = cf.d;
    e.cd = cf.d * (axis ? c.ah : c.ih);
    if constexpr (sizeof(T) == 4) {
        e.sll = cf.sll;
        e.shl = cf.shl;
        e.cdl = cf.d * (axis ? c.al : c.il);
    } else {
        e.sll = e.shl = e.cdl = T(0);
    }
    return e;
}
// w = sl xm + sh xp - cd x0 for one real component; in FP32 the lo-part
// products go first, then the hi parts accumulate onto them through FMAs.
template <typename T>
__device__ __forceinline__ T ex_w(const ExRow<T> &e, T xm, T xp, T x0) {
    if constexpr (sizeof(T) == 4) {
        float t = e.sll * xm;
        t = fmaf(e.shl, xp, t);
        t = fmaf(-e.cdl, x0, t);
        t = fmaf(e.sl, xm, t);
        t = fmaf(e.sh, xp, t);
        return fmaf(-e.cd, x0, t);
    } else {
        return e.sl * xm + e.sh * xp - e.cd * x0;
    }
}
// rhs_j = d x0 + i w for one pulse
template <typename T>
__device__ __forceinline__ cx<T> ex_rhs(const ExRow<T> &e, cx<T> xm, cx<T> x0, cx<T> xp) {
    const T wx = ex_w(e, xm.x, xp.x, x0.x);
    const T wy = ex_w(e, xm.y, xp.y, x0.y);
    return mk(e.d * x0.x - wy, e.d * x0.y + wx);
}

// Per-column constants of an FP32 context table, one per |q| (written by
// the table kernel, so that the column kernels' threads do no FP64 work of
// their own): lim = 1/p_inf(q) as a two-float pair (x, y hi; z, w lo), cd =
// c0 - delta_q as two-float pairs for the axis row (x hi, y lo) and the
// interior rows (z hi, w lo).
struct ColConst {
    float4 lim, cd;
};

template <typename T>
struct ColArgs {
    cx<T> *field;            // [nr][nt], frequency domain, in place
    const cx<T> *invden;     // [nr][tp]: 1/pivot_j per |q| = 0..nt/2
    const T *lo;             // [nr]: 1 - 1/(2j) (j >= 1), 0 at j = 0
    const T *hi;             // [nr]: 1 + 1/(2j) (j >= 1), 0 at j = 0
    const CnCoef<T> *coef = nullptr;   // [nr] row coefficients (staged variants)
    int nr, nt;
    T s;                     // dz / (4 k0 dr^2), 0 without diffraction
    T dk;                    // k'' dz/4 domega^2, 0 without dispersion: delta_q = dk q^2
    double s64 = 0.0, dk64 = 0.0;   // the same in FP64 (the coef variants' c0 - delta_q)
    double disp = 0.0;       // FCN_EXACT_DISPERSION: dk goes here instead, and the
                             // stage multiplies column q by exp(2 i disp q^2)
    int variant;             // 0..3: register chunks, long/short x CTA 256/512;
                             // 4, 5: cp.async-staged chunks of 16 / 8 rows (FP32);
                             // 6, 7: register-fed staged chunks of 16 / 8 rows;
                             // 8: one sequential sweep per column, TMA-fed
                             // (4..8 need coef)
    int tp = 0;              // row pitch of invden in complex values (>= nt/2 + 1)
    int *err = nullptr;      // set nonzero by a kernel whose bounded wait gave up
    int pivlim = 0;          // 1 (FP32 context tables): invden holds 1/pivot_j - 1/p_inf(q)
                             // (see piv_limit), applied with the limit as a two-float pair
    const ColConst *cc = nullptr;   // FP32 context tables: per-column constants (|q|)
};

struct TableArgs {
    int nr, nt;
    double s, dk;
    const double *lo, *hi;   // FP64 copies of the ratio tables
    int tp = 0;              // row pitch of the table in complex values (0: nt/2 + 1)
    int pivlim = 0;          // FP32: store 1/pivot_j - 1/p_inf(q) (ColArgs::pivlim)
    ColConst *cc = nullptr;  // FP32: per-column constants (tp entries), or none
};

// 1/p_inf(q), the limit of 1/pivot_j for large j in column q: with lo_j,
// hi_j -> 1 the pivot recurrence piv_j = b + s^2 lo_j hi_{j-1} / piv_{j-1}
// (b = 1 + i (2s - delta_q)) tends to the fixed point p of p = b + s^2 / p,
// p = (b + sqrt(b^2 + 4 s^2)) / 2 (the root of larger modulus; the
// principal square root, Re b = 1 > 0).  Where the coefficients hardly
// change with j (small s, large j) the pivots settle to this value within a
// few rows, and their FP32 roundings then repeat from row to row: rounded
// once, they made the discrete step non-unitary coherently (an FP32
// emulation on the 1350 x 1024 grid of the 1.1 km run: +2.9e-8 energy per
// step, -1.4e-10 with the pivots applied exactly).  FP32 context tables
// therefore hold 1/pivot_j - 1/p_inf, small wherever the pivots have
// settled, and the column kernels add the limit back as a two-float pair.
__host__ __device__ inline cx<double> piv_limit(double s, double dk, int qq) {
    const double g = 2.0 * s - dk * double(qq) * double(qq);
    // z = b^2 + 4 s^2 with b = 1 + i g
    const double zx = 1.0 - g * g + 4.0 * s * s, zy = 2.0 * g;
    const double r = hypot(zx, zy);
    const double u = sqrt(0.5 * (r + fabs(zx)));
    double sx, sy;
    if (zx >= 0.0) {
        sx = u;
        sy = u > 0.0 ? 0.5 * zy / u : 0.0;
    } else {
        sx = u > 0.0 ? 0.5 * fabs(zy) / u : 0.0;
        sy = copysign(u, zy);
    }
    const double px = 0.5 * (1.0 + sx), py = 0.5 * (g + sy);
    const double m = px * px + py * py;
    cx<double> inv;
    inv.x = px / m;
    inv.y = -py / m;
    return inv;
}

// The limit as the column kernels use it: 1/p_inf = h + l two-float, or
// h = l = 0 for plain 1/pivot tables (stateless FP32 launches; FP64 always),
// with which piv_full and piv_apply reduce to the plain forms exactly.
template <typename T>
struct PivLim {
    cx<T> h, l;
};
template <typename T>
__device__ __forceinline__ PivLim<T> piv_lim(int pivlim, double s, double dk, int qq) {
    PivLim<T> L;
    L.h = L.l = mk(T(0), T(0));
    if constexpr (sizeof(T) == 4) {
        if (pivlim) {
            const cx<double> v = piv_limit(s, dk, qq);
            L.h = mk(float(v.x), float(v.y));
            L.l = mk(float(v.x - double(L.h.x)), float(v.y - double(L.h.y)));
        }
    }
    return L;
}
// 1/pivot_j from a table entry (rounded to T; for the sweep factors).  In
// FP32 branch-free: without the limit h = l = 0 and the sums are exact, so
// the straight-line sweeps keep no data-dependent branch.
template <typename T>
__device__ __forceinline__ cx<T> piv_full(cx<T> v, const PivLim<T> &L) {
    if constexpr (sizeof(T) == 4) return mk(L.h.x + (v.x + L.l.x), L.h.y + (v.y + L.l.y));
    else return v;
}
// The explicit side's c0 - delta_q pairs and the pivot limit of column |q|:
// from the table's per-column constants when there are (FP32 contexts),
// else formed here (FP64; stateless FP32 launches, which have no limit).
template <typename T>
__device__ __forceinline__ void col_consts(const ColConst *cc, int pivlim, double s, double dk, int qq,
                                           CdCol<T> *cd, PivLim<T> *L) {
    if constexpr (sizeof(T) == 4) {
        if (cc) {
            const float4 lim = __ldg(&cc[qq].lim), c = __ldg(&cc[qq].cd);
            cd->ah = c.x;
            cd->al = c.y;
            cd->ih = c.z;
            cd->il = c.w;
            L->h = pivlim ? mk(lim.x, lim.y) : mk(0.f, 0.f);
            L->l = pivlim ? mk(lim.z, lim.w) : mk(0.f, 0.f);
            return;
        }
    }
    *cd = cd_col<T>(s, dk, qq);
    *L = piv_lim<T>(pivlim, s, dk, qq);
}

// rhs / pivot_j: with the limit on, rhs (h + (v + l)), the small part first
// (FP32: branch-free as piv_full; without the limit the result is rhs v
// exactly as the plain product computes it)
template <typename T>
__device__ __forceinline__ cx<T> piv_apply(cx<T> rhs, cx<T> v, const PivLim<T> &L) {
    if constexpr (sizeof(T) == 4) {
        const cx<T> lo = mk(v.x + L.l.x, v.y + L.l.y);
        const cx<T> t = cmul(rhs, lo);
        return mk(fmaf(rhs.x, L.h.x, fmaf(-rhs.y, L.h.y, t.x)), fmaf(rhs.x, L.h.y, fmaf(rhs.y, L.h.x, t.y)));
    } else {
        return cmul(rhs, v);
    }
}

// Row pitch (complex values) of the pivot tables a context builds: nt/2 + 1
// rounded up to even, so that every row starts on 16 bytes (a TMA row stride).
inline int table_pitch(int nt) { return (nt / 2 + 1 + 1) & ~1; }

// ---- launchers (defined in the .cu files) ----
template <typename T>
cudaError_t launch_rows(const RowArgs<T> &a, int nt, cudaStream_t st);
template <typename T>
cudaError_t launch_rows_multi(const RowMultiArgs<T> &m, int npulse, int nt, cudaStream_t st);
// Sets the kernel's shared-memory attribute for this Nt (call before the
// first launch, outside stream capture).
template <typename T>
cudaError_t prepare_rows(int nt);
template <typename T>
cudaError_t launch_cn(const ColArgs<T> &a, cudaStream_t st);
constexpr int kRowVariants = 6;
constexpr int kColVariants = 9;
constexpr int kColStagedFirst = 4;      // variants >= this need ColArgs::coef
constexpr int kColSeq = 8;              // the sequential TMA-fed column kernel (col_seq.cu)
// Sequential column stage of npulse (1..8) pulses sharing the grid, the
// coefficients and the pivot table (fields[k], blockIdx.y = k);
// cudaErrorInvalidConfiguration when cn_seq_supported(a) is false.
template <typename T>
cudaError_t launch_cn_seq(const ColArgs<T> &a, cx<T> *const *fields, int npulse, cudaStream_t st, int shape = 0);
constexpr int kSeqShapes = 3;   // ring shapes of the all-pulse sequential launch (launch_cn_seq)
template <typename T>
bool cn_seq_supported(const ColArgs<T> &a);
template <typename T>
cudaError_t launch_cn_table(const TableArgs &a, cx<T> *table, cudaStream_t st);
// Row coefficients for the staged column variants (nr rows).
template <typename T>
cudaError_t launch_cn_coef(const TableArgs &a, CnCoef<T> *coef, cudaStream_t st);
// Column stage of two pulses with the same grid and pivot table in one launch
// (a.field and field2; a's other arguments serve both).
template <typename T>
cudaError_t launch_cn_pair(const ColArgs<T> &a, cx<T> *field2, cudaStream_t st);
// Sets the staged column kernels' shared-memory attribute (outside capture).
template <typename T>
cudaError_t prepare_cn();

// Batched work lists (pulses of uneven grids in one launch per stage).
// Row items: (pulse, first row), 512/(Nt/16) rows each, Nt in 512..8192.
// Column items: (pulse, column group); every pulse uses 512-thread CTAs.
// counter: 2 unsigned, zero before the first launch (kernels reset them).
template <typename T>
cudaError_t launch_rows_batch(const RowArgs<T> *pulses, const int2 *items, int nitems, int ops,
                              unsigned *counter, size_t smem, int grid, cudaStream_t st);
template <typename T>
cudaError_t prepare_rows_batch(size_t smem);
template <typename T>
cudaError_t launch_cn_batch(const ColArgs<T> *pulses, const int4 *items, int nitems,
                            unsigned *counter, int grid, cudaStream_t st);
// shared-memory bytes of the batched row kernel for rows of nt points
size_t row_batch_smem(int nt, int bytes_per_complex);

// Cartesian transverse grid (xy_kernel.cu).  One launch solves the
// Crank-Nicolson system of every transverse line of one axis for every
// frequency bin: line (b, c) holds the n values
//   field[b * bstride + j * pitch + c],  j = 0..n-1 (j = 0, n-1 the walls),
// for b = 0..batch-1 and columns c = 0..width-1; the column's frequency bin
// is q = c mod nt.  The y lines of an [nx][ny][nt] field are (b = x, c = q):
// batch nx, width nt, pitch nt, bstride ny nt; the x lines are (b = y, c = q):
// batch ny, width nt, pitch ny nt, bstride nt.
template <typename T>
struct XYLine {
    cx<T> *field;
    const cx<T> *invden;     // [n][nt/2+1]: 1/pivot_j per |q|
    int n, nt, width, batch;
    long long pitch, bstride;
    long long total;         // elements of the field buffer
    T s;                     // dz / (4 k0 h^2), 0 without diffraction
    T dk;                    // delta_q = dk q^2 (0 in a line without dispersion)
    double s64, dk64;        // s and dk in FP64 (two-float explicit side in FP32)
    double disp;             // exact dispersion factor exp(2 i disp q^2), 0: none
    // chunk length L (long: 16 nodes in FP32, 8 in FP64; short: half),
    // lines per thread NP and CTA size: 0 long/1/512, 1 short/1/512,
    // 2 short/2/512, 3 short/2/256, 4 long/1/256, 5 short/1/256,
    // 6 short/2/256 compiled for three CTAs per SM, 7 short/1/256 for four
    int variant;
};
template <typename T>
cudaError_t launch_xy_table(int n, int nt, double s, double dk, cx<T> *table, cudaStream_t st);
template <typename T>
cudaError_t launch_xy_line(const XYLine<T> &a, cudaStream_t st);
constexpr int kXYVariants = 8;

// Learned dz controller (mlp.cu).
struct MlpScalars {
    double i_ref, e_prev, peak_prev, dz_prev, err_prev, rtol, l_ref, domega, dz_lo, dz_hi;
};
int mlp_nparam();
cudaError_t launch_mlp_grad(const float *W, const float *X, const float *Y, const int *idx, int n,
                            float *partial, int max_cta, float *grad, float *loss, cudaStream_t st);
cudaError_t launch_mlp_adam(float *W, float *m, float *v, const float *g, float lr, int t, cudaStream_t st);
// One attempt's controller outputs in one launch of 256 threads: the
// step-doubling norm from the per-row sums diff_rows that a row launch with
// OP_DIFF leaves (summed as launch_diff_final does; null: no norm), the
// reduction of the per-row
// statistics (nr rows of NSTAT), the features and, with W, the proposal;
// out (8 doubles): [norm0, norm1, 8 feature floats in 4 doubles (f0..f5,
// fE, peak), dz, energy sum]
cudaError_t launch_mlp_step_control(const double *stats, int nr, const double *diff_rows, const MlpScalars &sc,
                                    const float *W, double *out, cudaStream_t st);
// The same for up to kCtlMulti pulses on one grid in one launch (a CTA per
// pulse): pulse b reads stats[b], rows[b] (null: no norm), sc[b] and writes
// out + 8 b.
constexpr int kCtlMulti = 8;
struct CtlMulti {
    const double *stats[kCtlMulti];
    const double *rows[kCtlMulti];
    MlpScalars sc[kCtlMulti];
    double *out;
    int nr, n;
};
cudaError_t launch_mlp_step_control_multi(const CtlMulti &p, const float *W, cudaStream_t st);

// reductions and conversions
template <typename T>
cudaError_t launch_widen(const cx<T> *src, double *dst, int64_t n, cudaStream_t st);
template <typename T>
cudaError_t launch_narrow(const double *src, cx<T> *dst, int64_t n, cudaStream_t st);
template <typename T>
cudaError_t launch_widen_real(const T *src, double *dst, int64_t n, cudaStream_t st);
// Final FP64 reduction of per-row statistics into out[0..7]:
// [energy_sum (sum_m W_m S_m), max I, max u, onaxis max I, S0, S1, S2, nonfinite]
cudaError_t launch_reduce_stats(const double *stats, int nr, double *out, cudaStream_t st);
// The same with weight 1 for every row (Cartesian grid) and out[3] the
// maximum of row axis_row.
cudaError_t launch_reduce_stats_flat(const double *stats, int nrows, int axis_row, double *out,
                                     cudaStream_t st);
// Per-row sums of |a-b|^2 and |b|^2 (FP64) then the final reduction into out[0..1].
// Radial weight of row m in the energy sums (1/8 at the axis, m beyond).
__device__ __forceinline__ double radial_weight(int m) { return m == 0 ? 0.125 : double(m); }

// Block-wide FP64 sum / maximum with a fixed shuffle and shared-memory tree
// (bit-identical from run to run); result in thread 0; every thread of the
// block calls it; sh holds 32 doubles.
__device__ __forceinline__ double block_sum(double x, double *sh) {
    for (int d = 16; d >= 1; d >>= 1) x += __shfl_down_sync(0xffffffffu, x, d);
    const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
    __syncthreads();
    if (l == 0) sh[w] = x;
    __syncthreads();
    if (w == 0) {
        x = (l < (int)(blockDim.x >> 5)) ? sh[l] : 0.0;
        for (int d = 16; d >= 1; d >>= 1) x += __shfl_down_sync(0xffffffffu, x, d);
    }
    return x;
}
__device__ __forceinline__ double block_max(double x, double *sh) {
    for (int d = 16; d >= 1; d >>= 1) x = fmax(x, __shfl_down_sync(0xffffffffu, x, d));
    const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
    __syncthreads();
    if (l == 0) sh[w] = x;
    __syncthreads();
    if (w == 0) {
        x = (l < (int)(blockDim.x >> 5)) ? sh[l] : 0.0;
        for (int d = 16; d >= 1; d >>= 1) x = fmax(x, __shfl_down_sync(0xffffffffu, x, d));
    }
    return x;
}

// The step-doubling norm from the per-row sums a row launch with OP_DIFF
// leaves (rows[2m] = sum_p |cmp - A|^2, rows[2m+1] = sum_p |A|^2):
// out[0] = sum_m rows[2m], out[1] = sum_m rows[2m+1], FP64, one fixed tree.
cudaError_t launch_diff_final(const double *rows, int nr, double *out, cudaStream_t st);
// Power P(tau_p) (unscaled: sum_m W_m |A|^2) and fluence rows (sum_p |A|^2), FP64.
template <typename T>
cudaError_t launch_profiles(const cx<T> *f, int nr, int nt, double *power, double *rowsum,
                            cudaStream_t st);

}  // namespace fcn
