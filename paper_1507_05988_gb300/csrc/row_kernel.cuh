// row_kernel.cuh -- the row stage of the FCN z-step: FFTs along tau fused with
// the nonlinear half steps (Ma & Lin, arXiv:1507.05988, Sec. 3.1 first/third
// loops, Sec. 3.2, Eqs. (Anhalf)/(Anhalf1), and the re-organised step of
// Sec. 4 where the nonlinear part and the transforms share the radial
// decomposition).
//
// One row (fixed radial index m) is one independent unit of work.  Rows of
// Nt <= 4096 points run on 256 threads (several rows per CTA for Nt < 4096);
// Nt = 8192 runs on 512 threads.  Each thread owns E = 16 complex values
// (E = Nt when Nt < 16).
//
// Transform: in-place decimation-in-time FFT (one radix 2/4/8 pass for the
// factor left by radix 16, then radix-16 passes) in one padded shared-memory
// buffer with the butterfly operands in registers; every pass reads and
// writes the same positions in the same thread, so one barrier per pass
// suffices.  The forward transform takes the time samples in mixed-radix
// digit-reversed order (tpos) and leaves natural frequency order; the
// inverse transform is its exact adjoint (the forward passes in reverse
// order, transposed, with conjugate constants).  The first inverse pass
// reads HBM directly and the last forward pass writes HBM directly, in
// natural frequency order; both are coalesced (consecutive threads touch
// consecutive complex values).  Shared-memory rows are padded by one value
// per 16 so that the passes and the nonlinear stage's per-thread samples are
// free of bank conflicts.
//
// Nonlinear half step (Eq. (nonlinearpart)):  A <- A exp(h N(I, rho)).
// rho(tau) follows Eq. (ionization) integrated by RK4 along tau from
// rho(tau_min) = 0, with the RK4 midpoint intensity the mean of the two
// neighbours.  Because the ODE is linear in u = rho/rho_nt, one RK4 step is
// u_{p+1} = u_p + c_p (1 - u_p) with c_p a function of I_p and I_{p+1} only, so
// u_p = c_0 (+) c_1 (+) ... (+) c_{p-1} for the associative, commutative
// operation a (+) b = a + b - a b = 1 - (1-a)(1-b).  That makes the
// integration an exclusive parallel scan: sequential over each thread's 16
// points, warp shuffles across threads, and (rows wider than a warp) an FP64
// scan of the warp totals.  (+) never cancels (all terms are in [0, 1]), so
// the scan keeps the relative precision of the working type.
#pragma once
#include "fcn_device.cuh"

namespace fcn {
namespace {

constexpr int ilog2(int n) { return n <= 1 ? 0 : 1 + ilog2(n / 2); }

// FP64 scratch per CTA for the cross-warp parts of the row scans and
// reductions (rows per CTA x warps per row x values <= 64)
constexpr int kRowScratch = 64;

// NT is the row length with the FFT plan in its high bits (fft_tag); N is
// the length itself.
template <int NT>
struct RowCfg {
    static constexpr int N = fft_nt(NT);                    // points per row
    static constexpr int PLAN = fft_plan(NT);               // FFT decomposition
    static constexpr int E = N < 16 ? N : 16;               // values per thread
    static constexpr int TPR = N / E;                       // threads per row
    static constexpr int THREADS = TPR >= 256 ? TPR : 256;  // CTA size
    static constexpr int RPC = THREADS / TPR;               // rows per CTA
    static constexpr int PADN = N >= 16 ? N + N / 16 : N;
    static constexpr int NPASS = fft_npass(NT);
    static constexpr int WARPS_PER_ROW = TPR > 32 ? TPR / 32 : 1;
    static_assert(fft_radix(NT, NPASS - 1) == E, "the last pass has the radix of a thread's samples");
};

// Pass P of the transform: radix R (fft_radix: the plan's sequence, its last
// pass radix 16) and Ns, the product of the radices of the earlier passes.
template <int NT, int P>
struct PassCfg {
    static constexpr int R = fft_radix(NT, P);
    static constexpr int NS = fft_ns(NT, P);
};

__host__ __device__ __forceinline__ int pidx(int i, int nt) { return nt >= 16 ? i + (i >> 4) : i; }

// cos(2 pi m / 16)
__host__ __device__ constexpr double cos16(int m) {
    m &= 15;
    return m == 0 ? 1.0
         : m == 1 ? 0.92387953251128675613
         : m == 2 ? 0.70710678118654752440
         : m == 3 ? 0.38268343236508977173
         : m == 4 ? 0.0
         : m == 5 ? -0.38268343236508977173
         : m == 6 ? -0.70710678118654752440
         : m == 7 ? -0.92387953251128675613
         : m == 8 ? -1.0
         : m == 9 ? -0.92387953251128675613
         : m == 10 ? -0.70710678118654752440
         : m == 11 ? -0.38268343236508977173
         : m == 12 ? 0.0
         : m == 13 ? 0.38268343236508977173
         : m == 14 ? 0.70710678118654752440
         : 0.92387953251128675613;
}

// o * exp(DIR 2 pi i m / 16); exact shortcuts for the quarter turns.
//
// FP32 constants: a float (cos, sin) pair of a codelet or twiddle angle
// carries a phase and a modulus error of up to ~6e-8.  The same constants act
// on every row at every z-step, so such errors do not average out: they add
// up coherently over the steps (field error ~5e-7 per step, energy drift
// ~1e-8 per step on a 1024 x 4096 pulse).  So every non-trivial FP32 constant
// is applied as a two-float (hi + lo) pair inside the FMAs that multiply by
// it: the pi/8 family here, 1/sqrt(2) for the pi/4 family, and the twiddles
// (tw_mul).  Together with the inverse transform being the exact adjoint of
// the forward one (InvDispatch), the constants then leave errors at the
// level of the random rounding of the arithmetic only.
__device__ __forceinline__ void c16f_pair2(int m, float *ch, float *cl, float *sh, float *sl) {
    // cos(pi/8), sin(pi/8) = hi + lo (hi the nearest float, lo the nearest
    // float to the rest; residual below 7e-16)
    constexpr float C8H = 0.9238795042037964f, C8L = 2.830748968563057e-08f;
    constexpr float S8H = 0.3826834261417389f, S8L = 6.2233507236442165e-09f;
    switch (m & 15) {
        case 1: *ch = C8H; *cl = C8L; *sh = S8H; *sl = S8L; break;
        case 3: *ch = S8H; *cl = S8L; *sh = C8H; *sl = C8L; break;
        case 5: *ch = -S8H; *cl = -S8L; *sh = C8H; *sl = C8L; break;
        case 7: *ch = -C8H; *cl = -C8L; *sh = S8H; *sl = S8L; break;
        case 9: *ch = -C8H; *cl = -C8L; *sh = -S8H; *sl = -S8L; break;
        case 11: *ch = -S8H; *cl = -S8L; *sh = -C8H; *sl = -C8L; break;
        case 13: *ch = S8H; *cl = S8L; *sh = -C8H; *sl = -C8L; break;
        default: *ch = C8H; *cl = C8L; *sh = -S8H; *sl = -S8L; break;        // 15
    }
}

template <typename T, int DIR>
__device__ __forceinline__ cx<T> rot16(cx<T> o, int m) {
    m &= 15;
    if (m == 0) return o;
    if (m == 8) return mk(-o.x, -o.y);
    if (m == 4) return DIR > 0 ? mk(-o.y, o.x) : mk(o.y, -o.x);
    if (m == 12) return DIR > 0 ? mk(o.y, -o.x) : mk(-o.y, o.x);
    if constexpr (sizeof(T) == 4) {
        if ((m & 1) == 0) {
            // odd multiples of pi/4: (c, s) = (+-1, +-1)/sqrt(2)
            constexpr float H_HI = 0.70710676908493042f;       // float(1/sqrt 2)
            constexpr float H_LO = 1.2101617485882343e-8f;     // 1/sqrt 2 - H_HI
            const float sc = (m == 2 || m == 14) ? 1.f : -1.f;             // sign of cos
            const float ss = float(DIR) * ((m == 2 || m == 6) ? 1.f : -1.f);  // sign of sin
            const float re = sc * o.x - ss * o.y;
            const float im = ss * o.x + sc * o.y;
            return mk(T(fmaf(re, H_HI, re * H_LO)), T(fmaf(im, H_HI, im * H_LO)));
        }
        float ch, cl, sh, sl;
        c16f_pair2(m, &ch, &cl, &sh, &sl);
        if (DIR < 0) { sh = -sh; sl = -sl; }
        // (o.x + i o.y)(c + i s), the lo parts first
        const float lre = fmaf(o.x, cl, -o.y * sl);
        const float lim = fmaf(o.x, sl, o.y * cl);
        return mk(T(fmaf(o.x, ch, fmaf(-o.y, sh, lre))), T(fmaf(o.x, sh, fmaf(o.y, ch, lim))));
    } else {
        const T c = T(cos16(m));
        const T s = T(DIR) * T(cos16(m - 4));
        return mk(o.x * c - o.y * s, o.x * s + o.y * c);
    }
}

// Complex add / subtract; FP32 as one packed f32x2 instruction (each lane an
// IEEE single add, the same result as two scalar adds).
__device__ __forceinline__ cx<float> cadd2(cx<float> a, cx<float> b) {
    unsigned long long ra, rb, rc;
    asm("mov.b64 %0, {%1, %2};" : "=l"(ra) : "f"(a.x), "f"(a.y));
    asm("mov.b64 %0, {%1, %2};" : "=l"(rb) : "f"(b.x), "f"(b.y));
    asm("add.rn.f32x2 %0, %1, %2;" : "=l"(rc) : "l"(ra), "l"(rb));
    cx<float> r;
    asm("mov.b64 {%0, %1}, %2;" : "=f"(r.x), "=f"(r.y) : "l"(rc));
    return r;
}
__device__ __forceinline__ cx<float> csub2(cx<float> a, cx<float> b) {
    unsigned long long ra, rb, rc;
    asm("mov.b64 %0, {%1, %2};" : "=l"(ra) : "f"(a.x), "f"(a.y));
    asm("mov.b64 %0, {%1, %2};" : "=l"(rb) : "f"(b.x), "f"(b.y));
    asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(rc) : "l"(ra), "l"(rb));
    cx<float> r;
    asm("mov.b64 {%0, %1}, %2;" : "=f"(r.x), "=f"(r.y) : "l"(rc));
    return r;
}
__device__ __forceinline__ cx<double> cadd2(cx<double> a, cx<double> b) { return a + b; }
__device__ __forceinline__ cx<double> csub2(cx<double> a, cx<double> b) { return a - b; }

// In-register DFT of size R (power of two <= 16), natural order in and out,
// X_k = sum_n x_n exp(DIR 2 pi i n k / R), by radix-2 decimation in time.
template <typename T, int R, int DIR>
struct Dft {
    __device__ __forceinline__ static void run(cx<T> *v) {
        cx<T> e[R / 2], o[R / 2];
#pragma unroll
        for (int k = 0; k < R / 2; ++k) { e[k] = v[2 * k]; o[k] = v[2 * k + 1]; }
        Dft<T, R / 2, DIR>::run(e);
        Dft<T, R / 2, DIR>::run(o);
#pragma unroll
        for (int k = 0; k < R / 2; ++k) {
            const int m = k * (16 / R);
            cx<T> t = rot16<T, DIR>(o[k], m);
            if ((m & 7) == 4) {
                // quarter turn: t is o with its parts swapped, which the
                // scalar adds take as operands at no cost
                v[k] = e[k] + t;
                v[k + R / 2] = e[k] - t;
            } else {
                v[k] = cadd2(e[k], t);
                v[k + R / 2] = csub2(e[k], t);
            }
        }
    }
};
template <typename T, int DIR>
struct Dft<T, 1, DIR> {
    __device__ __forceinline__ static void run(cx<T> *) {}
};

// v * W_e (DIR < 0) or v * conj(W_e) (DIR > 0) for twiddle entry e.  FP32
// tables hold each twiddle as a two-float pair, 16 bytes per entry
// (hi.x, hi.y, lo.x, lo.y); FP64 tables one complex double.
template <typename T, int DIR>
__device__ __forceinline__ cx<T> tw_mul(cx<T> v, const cx<T> *__restrict__ tw, int e, int entries) {
    if constexpr (sizeof(T) == 4) {
        const float4 w = __ldg(reinterpret_cast<const float4 *>(tw) + FCN_IDX(e, entries, 3));
        const float hy = DIR > 0 ? -w.y : w.y;
        const float ly = DIR > 0 ? -w.w : w.w;
        const float lre = fmaf(v.x, w.z, -v.y * ly);
        const float lim = fmaf(v.x, ly, v.y * w.z);
        return mk(T(fmaf(v.x, w.x, fmaf(-v.y, hy, lre))), T(fmaf(v.x, hy, fmaf(v.y, w.x, lim))));
    } else {
        cx<T> w = ldg_cx(&tw[FCN_IDX(e, entries, 3)]);
        if (DIR > 0) w.y = -w.y;
        return cmul(v, w);
    }
}

// Adjoint of Dft<T, R, -1>: the same butterflies transposed, with the
// conjugate constants (decimation in frequency).  Exact transpose in exact
// arithmetic, so that Inverse(Forward(x)) = x to first order in the errors of
// the rounded constants.
template <typename T, int R>
struct DftAdj {
    __device__ __forceinline__ static void run(cx<T> *v) {
        cx<T> e[R / 2], o[R / 2];
#pragma unroll
        for (int k = 0; k < R / 2; ++k) {
            const int m = k * (16 / R);
            const cx<T> a = v[k], b = v[k + R / 2];
            e[k] = cadd2(a, b);
            if (m == 4) {
                o[k] = mk(b.y - a.y, a.x - b.x);          // i (a - b)
            } else if (m == 12) {
                o[k] = mk(a.y - b.y, b.x - a.x);          // -i (a - b)
            } else {
                o[k] = rot16<T, +1>(csub2(a, b), m);
            }
        }
        DftAdj<T, R / 2>::run(e);
        DftAdj<T, R / 2>::run(o);
#pragma unroll
        for (int k = 0; k < R / 2; ++k) { v[2 * k] = e[k]; v[2 * k + 1] = o[k]; }
    }
};
template <typename T>
struct DftAdj<T, 1> {
    __device__ __forceinline__ static void run(cx<T> *) {}
};

// Twiddle and butterfly of forward pass P for this thread's butterflies
// (operands already in v[i*R + r]).
template <typename T, int NT, int P>
__device__ __forceinline__ void pass_compute(cx<T> (&v)[RowCfg<NT>::E], int t,
                                             const cx<T> *__restrict__ tw) {
    using C = RowCfg<NT>;
    constexpr int R = PassCfg<NT, P>::R;
    constexpr int NS = PassCfg<NT, P>::NS;
    constexpr int NB = C::E / R;
    constexpr int OFF = tw_offset(NT, P);
    static_assert(R == fft_radix(NT, P) && NS == fft_ns(NT, P), "pass structure");
#pragma unroll
    for (int i = 0; i < NB; ++i) {
        const int j = t + C::TPR * i;
        if (NS > 1) {
            const int k = j & (NS - 1);
#pragma unroll
            for (int r = 1; r < R; ++r)
                v[i * R + r] = tw_mul<T, -1>(v[i * R + r], tw, OFF + (r - 1) * NS + k, tw_size(NT));
        }
        Dft<T, R, -1>::run(&v[i * R]);
    }
}

// Adjoint of forward pass P: the transposed butterfly, then the conjugate
// twiddles.
template <typename T, int NT, int P>
__device__ __forceinline__ void pass_compute_adj(cx<T> (&v)[RowCfg<NT>::E], int t,
                                                 const cx<T> *__restrict__ tw) {
    using C = RowCfg<NT>;
    constexpr int R = PassCfg<NT, P>::R;
    constexpr int NS = PassCfg<NT, P>::NS;
    constexpr int NB = C::E / R;
    constexpr int OFF = tw_offset(NT, P);
#pragma unroll
    for (int i = 0; i < NB; ++i) {
        DftAdj<T, R>::run(&v[i * R]);
        if (NS > 1) {
            const int k = (t + C::TPR * i) & (NS - 1);
#pragma unroll
            for (int r = 1; r < R; ++r)
                v[i * R + r] = tw_mul<T, +1>(v[i * R + r], tw, OFF + (r - 1) * NS + k, tw_size(NT));
        }
    }
}

// Operands of forward pass P (in-place decimation in time): butterfly
// j = t + TPR i combines the positions base + r NS (r < R), base =
// (j / NS) NS R + j mod NS, and writes its outputs back to them.
template <typename T, int NT, int P>
__device__ __forceinline__ void pass_load(cx<T> (&v)[RowCfg<NT>::E], const cx<T> *S, int t) {
    using C = RowCfg<NT>;
    constexpr int R = PassCfg<NT, P>::R;
    constexpr int NS = PassCfg<NT, P>::NS;
    constexpr int NB = C::E / R;
#pragma unroll
    for (int i = 0; i < NB; ++i) {
        const int j = t + C::TPR * i;
        const int base = (j / NS) * NS * R + (j & (NS - 1));
#pragma unroll
        for (int r = 0; r < R; ++r) v[i * R + r] = S[FCN_IDX(pidx(base + r * NS, fft_nt(NT)), C::PADN, 1)];
    }
}

template <typename T, int NT, int P>
__device__ __forceinline__ void pass_store(const cx<T> (&v)[RowCfg<NT>::E], cx<T> *S, int t) {
    using C = RowCfg<NT>;
    constexpr int R = PassCfg<NT, P>::R;
    constexpr int NS = PassCfg<NT, P>::NS;
    constexpr int NB = C::E / R;
#pragma unroll
    for (int i = 0; i < NB; ++i) {
        const int j = t + C::TPR * i;
        const int base = (j / NS) * NS * R + (j & (NS - 1));
#pragma unroll
        for (int r = 0; r < R; ++r) S[FCN_IDX(pidx(base + r * NS, fft_nt(NT)), C::PADN, 2)] = v[i * R + r];
    }
}

// Inverse transform: the exact adjoint of the forward transform, i.e. the
// forward passes in reverse order, each applying the transposed butterfly
// and the conjugate twiddles in place (input already in registers in the
// last forward pass's order, i.e. natural frequency order; result in S in
// the forward transform's input order, scaled by sc in its last pass).
// Every pass reads and writes the same positions in the same thread, so one
// barrier per pass (before other threads read them) suffices.
template <typename T, int NT, int P, bool DONE>
struct InvDispatch;
template <typename T, int NT, int P>
struct InvDispatch<T, NT, P, false> {
    // sc (the 1/Nt of the inverse transform) scales the last pass's outputs
    __device__ __forceinline__ static void run(cx<T> (&v)[RowCfg<NT>::E], cx<T> *S, int t,
                                               const cx<T> *tw, T sc) {
        using C = RowCfg<NT>;
        if (P + 1 < C::NPASS) pass_load<T, NT, P>(v, S, t);
        asm volatile("" ::: "memory");
        pass_compute_adj<T, NT, P>(v, t, tw);
        if (P == 0) {
#pragma unroll
            for (int e = 0; e < C::E; ++e) v[e] = mk(v[e].x * sc, v[e].y * sc);
        }
        pass_store<T, NT, P>(v, S, t);
        __syncthreads();
        InvDispatch<T, NT, P - 1, (P < 1)>::run(v, S, t, tw, sc);
    }
};
template <typename T, int NT, int P>
struct InvDispatch<T, NT, P, true> {
    __device__ __forceinline__ static void run(cx<T> (&)[RowCfg<NT>::E], cx<T> *, int,
                                               const cx<T> *, T) {}
};

// Forward transform in place: input in S in the digit-reversed order of
// tpos, output of the last pass (natural frequency order, positions
// j + r NS) left in registers for the caller.  The caller's barrier before
// the first pass makes S complete.
template <typename T, int NT, int P, bool LAST>
struct FwdDispatch;
template <typename T, int NT, int P>
struct FwdDispatch<T, NT, P, false> {
    __device__ __forceinline__ static void run(cx<T> (&v)[RowCfg<NT>::E], cx<T> *S, int t,
                                               const cx<T> *tw) {
        pass_load<T, NT, P>(v, S, t);
        // compiler-only fence: the twiddle loads stay behind the operand
        // loads (issuing them together costs registers the 4-CTA variant lacks)
        asm volatile("" ::: "memory");
        pass_compute<T, NT, P>(v, t, tw);
        if (P + 1 < RowCfg<NT>::NPASS) {
            pass_store<T, NT, P>(v, S, t);
            __syncthreads();
        }
        FwdDispatch<T, NT, P + 1, (P + 1 >= RowCfg<NT>::NPASS)>::run(v, S, t, tw);
    }
};
template <typename T, int NT, int P>
struct FwdDispatch<T, NT, P, true> {
    __device__ __forceinline__ static void run(cx<T> (&)[RowCfg<NT>::E], cx<T> *, int,
                                               const cx<T> *) {}
};

// Padded shared-memory index of the e-th of the E samples a thread owns,
// whose first sits at unpadded position p0 (tpos): when the sample stride
// NSL is a multiple of 16 the padding is linear in e, so that the indices
// are one base plus compile-time offsets.
template <int NT, int NSL>
__host__ __device__ __forceinline__ int own_idx(int q0, int p0, int e) {
    if constexpr (fft_nt(NT) >= 16 && NSL % 16 == 0) return q0 + e * (NSL + NSL / 16);
    else return pidx(p0 + e * NSL, fft_nt(NT));
}

// Position in S of time sample tau.  The forward transform takes its input
// in mixed-radix digit-reversed order: the least significant digit of tau
// (radix R of the last pass) is the most significant digit of the position
// (place value NS of the last pass), and so on.  With the last pass of
// radix E, a thread's E consecutive samples tau = E t + e sit at
// tpos(E t) + e NS_last.
template <int NT>
__host__ __device__ __forceinline__ int tpos(int tau) {
    int p = 0;
#pragma unroll
    for (int s = RowCfg<NT>::NPASS - 1; s >= 0; --s) {
        p += (tau % fft_radix(NT, s)) * fft_ns(NT, s);
        tau /= fft_radix(NT, s);
    }
    return p;
}

// Time-domain rows between HBM (natural order) and S (digit-reversed
// positions, tpos).  Consecutive tau sit NS_last apart in S, which for the
// usual sizes is one bank (4096 points: 272 values apart): lanes moving
// consecutive tau would meet a 32-way bank conflict on every access of S.
// Instead, per instruction, lanes 2b and 2b+1 move the two 16-byte halves of
// one 32-byte sector of line b of a group of 16 consecutive 128-byte lines:
// whole sectors to and from HBM, and the 16 lines' values sit in different
// banks of S (their positions differ in the higher digits).  A thread moves
// its E values as E / CPC 16-byte chunks.  Needs whole warps per row and
// whole groups of 16 lines; otherwise the per-value coalesced loop is used.
template <typename T, int NT>
struct RowIo {
    static constexpr int N = fft_nt(NT);
    static constexpr int CPC = 16 / (int)sizeof(cx<T>);   // values per 16-byte chunk
    static constexpr int LW = 128 / (int)sizeof(cx<T>);   // values per 128-byte line
    static constexpr int UNITS = RowCfg<NT>::E / CPC;      // chunks per thread
    static constexpr int NSL = PassCfg<NT, RowCfg<NT>::NPASS - 1>::NS;
    static constexpr bool OK = RowCfg<NT>::E == 16 && RowCfg<NT>::TPR % 32 == 0 &&
                               (N * (int)sizeof(cx<T>)) % 2048 == 0 && UNITS % 4 == 0;
};

// The row at p can move in 16-byte chunks (complex<double> is 16-byte aligned
// by its type; a float row needs a 16-byte aligned start).
template <typename T, int NT>
__device__ __forceinline__ bool row_io_chunks(const cx<T> *p) {
    if constexpr (!RowIo<T, NT>::OK) return false;
    else return sizeof(T) == 8 || (reinterpret_cast<uintptr_t>(p) & 15) == 0;
}

template <typename T>
__device__ __forceinline__ void ld_chunk(const cx<T> *p, cx<T> *v) {
    if constexpr (sizeof(T) == 4) {
        const float4 q = *reinterpret_cast<const float4 *>(p);
        v[0] = mk(q.x, q.y);
        v[1] = mk(q.z, q.w);
    } else {
        v[0] = *p;
    }
}

template <typename T>
__device__ __forceinline__ void st_chunk(cx<T> *p, const cx<T> *v) {
    if constexpr (sizeof(T) == 4) *reinterpret_cast<float4 *>(p) = make_float4(v[0].x, v[0].y, v[1].x, v[1].y);
    else *p = v[0];
}

// Visits the thread's chunks: f(tau, q0, p0) with tau the chunk's first time
// sample and (q0, p0) the padded and unpadded S positions of tau rounded down
// to a multiple of 16 (own_idx then places tau & 15 and the next values).
template <typename T, int NT, typename F>
__host__ __device__ __forceinline__ void row_chunks(int t, F f) {
    using IO = RowIo<T, NT>;
    const int lane = t & 31, w = t >> 5;
#pragma unroll
    for (int gi = 0; gi < IO::UNITS / 4; ++gi) {
        const int line = 16 * (w * (IO::UNITS / 4) + gi) + (lane >> 1);
        const int tl = line * IO::LW;
        const int p0 = tpos<NT>(tl & ~15);
        const int q0 = pidx(p0, IO::N);
#pragma unroll
        for (int j = 0; j < 4; ++j) f(tl + (2 * j + (lane & 1)) * IO::CPC, q0, p0);
    }
}

// The same sector-wise order for a row of reals (the rho output from the u
// rows): 16-byte chunks of RC reals, 128-byte lines of 8 RC reals.  Used with
// FFT plan 0, where it cuts the wavefronts at every Nt (4096 float points:
// 2 instead of 8); with plan 1 it would not at every Nt, and the per-value
// loop stays.
template <typename T, int NT>
struct RowIoReal {
    static constexpr int N = fft_nt(NT);
    static constexpr int RC = 16 / (int)sizeof(T);        // reals per 16-byte chunk
    static constexpr int LW = 128 / (int)sizeof(T);       // reals per 128-byte line
    static constexpr int UNITS = RowCfg<NT>::E / RC;       // chunks per thread
    static constexpr bool OK = fft_plan(NT) == 0 && RowCfg<NT>::E == 16 && RowCfg<NT>::TPR % 32 == 0 &&
                               (N * (int)sizeof(T)) % 2048 == 0 && UNITS % 4 == 0;
};

template <typename T, int NT>
__device__ __forceinline__ bool row_io_real_chunks(const T *p) {
    if constexpr (!RowIoReal<T, NT>::OK) return false;
    else return (reinterpret_cast<uintptr_t>(p) & 15) == 0;
}

// Visits the thread's chunks of a real row: f(tau), tau the chunk's first
// time sample (a chunk never crosses a multiple of 16).
template <typename T, int NT, typename F>
__host__ __device__ __forceinline__ void row_real_chunks(int t, F f) {
    using IO = RowIoReal<T, NT>;
    const int lane = t & 31, w = t >> 5;
#pragma unroll
    for (int gi = 0; gi < IO::UNITS / 4; ++gi) {
        const int line = 16 * (w * (IO::UNITS / 4) + gi) + (lane >> 1);
#pragma unroll
        for (int j = 0; j < 4; ++j) f(line * IO::LW + (2 * j + (lane & 1)) * IO::RC);
    }
}

// ---------------------------------------------------------------------------
// Nonlinear half step
// ---------------------------------------------------------------------------

template <typename T>
__device__ __forceinline__ T ipow(T x, int k) {
    T r = T(1);
    while (k) {
        if (k & 1) r *= x;
        x *= x;
        k >>= 1;
    }
    return r;
}

// x^K with K a compile-time constant when KT > 0 (squarings unrolled), the
// runtime exponent k otherwise.
template <int KT, typename T>
__device__ __forceinline__ T powk(T x, int k) {
    if constexpr (KT == 8) {
        const T x2 = x * x, x4 = x2 * x2;
        return x4 * x4;
    } else if constexpr (KT == 7) {
        const T x2 = x * x, x4 = x2 * x2;
        return x4 * x2 * x;
    } else {
        return ipow(x, k);
    }
}

template <typename T>
__device__ __forceinline__ T uplus(T a, T b) { return a + b - a * b; }

// RK4 increment of u over one dtau cell (du/dtau = w (1 - u), w = sigma_K
// I^K): with xa, xb, xm = dtau w at the cell's ends and midpoint,
// u_next = u + c (1 - u),
//   6 c = xa + 2 xm t1 + 2 xm t2 + xb t3,
//   t1 = 1 - xa/2,  t2 = 1 - (xm/2) t1,  t3 = 1 - xm t2.
// Returns 6 c (the caller folds the 1/6 into the (+) update).
template <typename T>
__device__ __forceinline__ T rk4_coef6(T xa, T xb, T xm) {
    const T t1 = fma(T(-0.5), xa, T(1));
    const T t2 = fma(T(-0.5) * xm, t1, T(1));
    const T t3 = fma(-xm, t2, T(1));
    const T acc = fma(xm + xm, t1 + t2, xa);
    return fma(xb, t3, acc);
}

// run (+) c for c = c6 / 6: run + c (1 - run)
template <typename T>
__device__ __forceinline__ T uplus6(T run, T c6) {
    return fma(c6, fma(-run, T(1.0 / 6.0), T(1.0 / 6.0)), run);
}

template <typename T>
__device__ __forceinline__ void sincos_t(T x, T *s, T *c);
// FP32 sine and cosine minus one of a nonlinear phase.  The factor
// exp(i x) is applied in delta form (A + A (exp(i x) - 1)), because a float
// cosine that rounds to 1 for small x gives |(cos, sin)|^2 = 1 + x^2 > 1 --
// a systematic energy gain in the weak tails of the pulse.  Evaluation:
// |x| < 1e-3: series (next terms below 5e-14);  otherwise Cody & Waite's
// reduction x = n pi/2 + r with pi/2 split into two floats (n*PIO2_HI exact
// inside the FMA) and Taylor polynomials of degree 9 (sin) and 10 (cos) on
// |r| <= pi/4, truncation below 2e-9 and 1.2e-10, with cos r - 1 kept
// without adding 1 (no cancellation); arguments beyond 1e4 rad, where the
// two-float reduction loses digits, go to the library.
__device__ __forceinline__ void sincos_m1_f32(float x, float *s, float *cm1) {
    if (fabsf(x) < 1.0e-3f) {
        const float x2 = x * x;
        *cm1 = -0.5f * x2;
        *s = fmaf(x * x2, -1.66666666666666666667e-1f, x);
        return;
    }
    if (fabsf(x) > 1.0e4f) {
        float c;
        sincosf(x, s, &c);
        *cm1 = c - 1.0f;
        return;
    }
    constexpr float TWO_OVER_PI = 0.636619772367581343076f;
    constexpr float PIO2_HI = 1.57079637050628662109f;       // float nearest pi/2
    constexpr float PIO2_LO = -4.37113900018624283e-8f;       // pi/2 - PIO2_HI
    const float n = rintf(x * TWO_OVER_PI);
    float r = fmaf(-n, PIO2_HI, x);
    r = fmaf(-n, PIO2_LO, r);
    const float r2 = r * r;
    // sin r = r - r^3/3! + r^5/5! - r^7/7! + r^9/9!
    float ps = fmaf(r2, 2.75573192239858906526e-6f, -1.98412698412698412698e-4f);
    ps = fmaf(r2, ps, 8.33333333333333333333e-3f);
    ps = fmaf(r2, ps, -1.66666666666666666667e-1f);
    const float sr = fmaf(r * r2, ps, r);
    // cos r - 1 = -r^2/2! + r^4/4! - r^6/6! + r^8/8! - r^10/10!
    float pc = fmaf(r2, -2.75573192239858906526e-7f, 2.48015873015873015873e-5f);
    pc = fmaf(r2, pc, -1.38888888888888888889e-3f);
    pc = fmaf(r2, pc, 4.16666666666666666667e-2f);
    pc = fmaf(r2, pc, -0.5f);
    const float crm1 = r2 * pc;
    const float cr = crm1 + 1.0f;
    switch (int(n) & 3) {
        case 0: *s = sr; *cm1 = crm1; break;
        case 1: *s = cr; *cm1 = -sr - 1.0f; break;
        case 2: *s = -sr; *cm1 = -cr - 1.0f; break;
        default: *s = -cr; *cm1 = sr - 1.0f; break;
    }
}

// exp(x) - 1 in FP32: the loss exponent is tiny except near the peak; the
// series x + x^2/2 is exact to float rounding there (x^3/6 < 2e-13).
__device__ __forceinline__ float expm1_f32(float x) {
    if (fabsf(x) < 1.0e-4f) return fmaf(0.5f * x, x, x);
    return expm1f(x);
}

template <typename T>
__device__ __forceinline__ void sincos_t(T x, T *s, T *c);
template <>
__device__ __forceinline__ void sincos_t<double>(double x, double *s, double *c) { sincos(x, s, c); }
template <typename T>
__device__ __forceinline__ T exp_t(T x);
template <>
__device__ __forceinline__ float exp_t<float>(float x) { return expf(x); }
template <>
__device__ __forceinline__ double exp_t<double>(double x) { return exp(x); }

// A <- A exp(h N(Ihat, u)) with h folded into the coefficients:
//   phi = Ihat (hk0 + Ihat (hk1 + Ihat (hk2 + Ihat hk3))) - hplasma u,
//   lnamp = -hloss Ihat^(K-1) (1 - sat u),  A <- A exp(lnamp + i phi).
// nl_terms gives (phi, lnamp); ihKm1 = Ihat^(K-1).
template <typename T>
__device__ __forceinline__ void nl_terms(T ih, T ihKm1, T u, const NLCoef<T> &c, T *phi, T *lnamp) {
    T p = fma(ih, c.hk[3], c.hk[2]);
    p = fma(ih, p, c.hk[1]);
    p = fma(ih, p, c.hk[0]);
    *phi = fma(-c.hplasma, u, ih * p);
    *lnamp = -(c.hloss * fma(-c.sat, u, T(1))) * ihKm1;
}

// FP32 delta form: A + A D with D = amp exp(i phi) - 1
//   = (em1 + cm1 + em1 cm1) + i s (1 + em1),  em1 = amp - 1.
// A D is formed first and added to A with one rounding per component.
// Folding the terms into A one FMA at a time (A + first-order part, then +
// second-order part) rounds A plus the first-order part before the
// second-order part (dre ~ -phi^2/2, a few ulps of A or less) is added, and
// that rounding is not unbiased: it dropped part of the modulus-reducing
// term and raised |A| by ~1e-8 of the energy per step on a Kerr-phase pulse
// (an FP32 emulation of both orders: +9.7e-9 against -2.5e-11 per
// application at phi up to 2e-3).
__device__ __forceinline__ cx<float> nl_delta(cx<float> a, float sn, float cm1, float em1) {
    const float dre = fmaf(em1, cm1, em1 + cm1);
    const float dim = fmaf(sn, em1, sn);
    const float dx = fmaf(a.x, dre, -(a.y * dim));
    const float dy = fmaf(a.y, dre, a.x * dim);
    return mk(a.x + dx, a.y + dy);
}

// Small arguments (|phi| < 1e-3, |lnamp| < 1e-4): the series of sin, cos - 1
// and exp - 1 are exact to float rounding there (see sincos_m1_f32 and
// expm1_f32 for the bounds).
__device__ __forceinline__ bool nl_small(float phi, float lnamp) {
    return fabsf(phi) < 1.0e-3f && fabsf(lnamp) < 1.0e-4f;
}
__device__ __forceinline__ cx<float> nl_apply_small(cx<float> a, float phi, float lnamp) {
    const float p2 = phi * phi;
    const float cm1 = -0.5f * p2;
    const float sn = fmaf(phi * p2, -1.66666666666666666667e-1f, phi);
    const float em1 = fmaf(0.5f * lnamp, lnamp, lnamp);
    return nl_delta(a, sn, cm1, em1);
}

template <typename T>
__device__ __forceinline__ cx<T> nl_apply_terms(cx<T> a, T phi, T lnamp);

// The update of a group of points that is not all small-argument, kept out
// of line: the unrolled nonlinear loop inlines only the common FP32
// small-argument path (the general one is rare: the pulse's core).
template <typename T>
__device__ __noinline__ cx<T> nl_apply_general(cx<T> a, T phi, T lnamp) {
    return nl_apply_terms<T>(a, phi, lnamp);
}

template <typename T>
__device__ __forceinline__ cx<T> nl_apply_terms(cx<T> a, T phi, T lnamp) {
    if constexpr (sizeof(T) == 4) {
        if (nl_small(phi, lnamp)) return nl_apply_small(a, phi, lnamp);
        float sn, cm1;
        sincos_m1_f32(phi, &sn, &cm1);
        return nl_delta(a, sn, cm1, expm1_f32(lnamp));
    } else {
        T s, co;
        sincos_t<T>(phi, &s, &co);
        const T amp = exp_t<T>(lnamp);
        return cmul(a, mk(amp * co, amp * s));
    }
}

// Exclusive (+)-scan of one value per thread across the TPR threads of a row.
// Returns the carry entering this thread.  FP64 carries between warps.
template <typename T, int NT>
__device__ __forceinline__ T row_scan_exclusive(T tot, int t, double *scr, int rloc) {
    using C = RowCfg<NT>;
    if (C::TPR == 1) return T(0);
    constexpr int W = C::TPR < 32 ? C::TPR : 32;
    const int lane = t & (W - 1);
    T incl = tot;
#pragma unroll
    for (int d = 1; d < W; d <<= 1) {
        T y = __shfl_up_sync(0xffffffffu, incl, d, W);
        if (lane >= d) incl = uplus(incl, y);
    }
    T excl = __shfl_up_sync(0xffffffffu, incl, 1, W);
    if (lane == 0) excl = T(0);
    if (C::WARPS_PER_ROW > 1) {
        const int w = t >> 5;
        double *ws = scr + rloc * C::WARPS_PER_ROW;
        if (lane == 31) scr[FCN_IDX(rloc * C::WARPS_PER_ROW + w, 32, 14)] = double(incl);
        __syncthreads();
        if (t < 32) {
            // FP64 exclusive scan of the warp totals of this row (<= 16)
            double x = (lane < C::WARPS_PER_ROW) ? scr[FCN_IDX(rloc * C::WARPS_PER_ROW + lane, 32, 15)] : 0.0;
            double in = x;
            // log2(warps per row) levels: the FP64 latency of this serial
            // part is paid while the row's other warps wait at the barrier
#pragma unroll
            for (int d = 1; d < C::WARPS_PER_ROW; d <<= 1) {
                double y = __shfl_up_sync(0xffffffffu, in, d, 32);
                if (lane >= d) in = in + y - in * y;
            }
            double ex = __shfl_up_sync(0xffffffffu, in, 1, 32);
            if (lane == 0) ex = 0.0;
            __syncwarp();
            if (lane < C::WARPS_PER_ROW) scr[FCN_IDX(rloc * C::WARPS_PER_ROW + lane, 32, 16)] = ex;
        }
        __syncthreads();
        // the carries are not rewritten before the caller's next barrier
        const T wc = T(scr[FCN_IDX(rloc * C::WARPS_PER_ROW + w, 32, 17)]);
        excl = uplus(wc, excl);
    }
    return excl;
}

// One nonlinear half step of this thread's E contiguous points p = E t + e
// of the row in S (natural order, padded, already scaled), in place.  Two
// phases: (A) the RK4 coefficients of the cells (p, p+1) -- the last one
// needs the next thread's first point -- and the thread-local exclusive
// (+)-scan into U, then the row scan for the carry; (B) the update
// A <- A exp(h N), four points per iteration of a rolled loop (one copy of
// the rare general-argument code keeps the kernel small).  STORE_U writes the
// final u_p back to U (statistics, rho output).  Callers put a barrier
// between two half steps (phase A reads the neighbour's point).
template <typename T, int NT, int KT, bool STORE_U>
__device__ __forceinline__ void nl_half_smem(cx<T> *S, T *U, int t, const NLCoef<T> &c, bool need_u,
                                             double *scr, int rloc) {
    using C = RowCfg<NT>;
    constexpr int E = C::E;
    constexpr int NSL = PassCfg<NT, C::NPASS - 1>::NS;
    static_assert(PassCfg<NT, C::NPASS - 1>::R == E, "a thread's samples differ in the last digit only");
    // the thread's samples tau = E t + e sit at p0 + e NSL (tpos)
    const int p0 = tpos<NT>(E * t);
    const int q0 = pidx(p0, fft_nt(NT));
    const bool last_thread = (t == C::TPR - 1);
    // |A|^2 of the thread's points and of the next thread's first point
    T cn[E + 1];
#pragma unroll
    for (int e = 0; e < E; ++e) cn[e] = cnorm(S[FCN_IDX((own_idx<NT, NSL>(q0, p0, e)), C::PADN, 8)]);
    cn[E] = last_thread ? T(0) : cnorm(S[FCN_IDX(pidx(tpos<NT>(E * (t + 1)), fft_nt(NT)), C::PADN, 8)]);
    T cmax = T(0);
#pragma unroll
    for (int e = 0; e < E; ++e) cmax = fmax(cmax, cn[e]);
    T carry = T(0), umax = T(0);
    // the thread's exclusive local prefixes of the (+)-scan; u at point e is
    // carry (+) lp[e] once the carry is known (registers: U exists only when
    // the caller keeps u for rho or statistics)
    T lp[E];
#pragma unroll
    for (int e = 0; e < E; ++e) lp[e] = T(0);
    if (need_u) {
        T run = T(0);
        // j = |A|^2 is_root: x = dtau sigma_K Ihat^K = j^K
        T jv[E + 1];
#pragma unroll
        for (int e = 0; e <= E; ++e) jv[e] = cn[e] * c.is_root;
        T jmax = T(0);
#pragma unroll
        for (int e = 0; e <= E; ++e) jmax = fmax(jmax, jv[e]);
        // Where every j^K of the thread's cells underflows to zero (the pulse's
        // wings: j^8 rounds to 0 for j below 2.4e-6 in FP32, 4e-41 in FP64),
        // every RK4 increment is exactly zero and u keeps its entering value:
        // the arithmetic below would give the same bits.
        const bool idle = (KT == 8) && jmax < (sizeof(T) == 4 ? T(2e-6) : T(1e-41));
        if (!idle) {
            T ja = jv[0];
            T xa = powk<KT>(ja, c.K);
#pragma unroll
            for (int e = 0; e < E; ++e) {
                lp[e] = run;
                if ((e + 1 < E) || !last_thread) {
                    const T jb = jv[e + 1];
                    const T xb = powk<KT>(jb, c.K);
                    const T xm = powk<KT>(T(0.5) * (ja + jb), c.K);
                    run = uplus6(run, rk4_coef6(xa, xb, xm));
                    ja = jb;
                    xa = xb;
                }
            }
        }
        carry = row_scan_exclusive<T, NT>(run, t, scr, rloc);
        umax = uplus(carry, run);      // u only grows along tau
    }
    const T omc = T(1) - carry;
    if constexpr (sizeof(T) == 4) {
        // FP32: where |phi| and |lnamp| stay below 2^-27 at every point of the
        // thread (the pulse's wings), exp(lnamp + i phi) - 1 is below 1/8 ulp
        // of 1 and the update leaves A as it is to float rounding; bounds
        // from the largest |A|^2 and the largest u (the scan's right end).
        const T ihm = cmax * c.inv_is;
        const T pk = fabsf(c.hk[0]) + ihm * (fabsf(c.hk[1]) + ihm * (fabsf(c.hk[2]) + ihm * fabsf(c.hk[3])));
        const T phib = ihm * pk + fabsf(c.hplasma) * umax;
        const T lnab = fabsf(c.hloss) * powk<(KT > 0 ? KT - 1 : 0)>(ihm, c.K - 1);
        if (phib < T(7.450580596923828e-9) && lnab < T(7.450580596923828e-9)) {
            if (STORE_U && need_u) {
#pragma unroll
                for (int e = 0; e < E; ++e)
                    U[FCN_IDX((own_idx<NT, NSL>(q0, p0, e)), C::PADN, 28)] = fma(lp[e], omc, carry);
            }
            return;
        }
    }
    constexpr int UN = E >= 4 ? 4 : E;
#pragma unroll
    for (int e0 = 0; e0 < E; e0 += UN) {
        cx<T> x[UN];
        T u[UN];
#pragma unroll
        for (int k = 0; k < UN; ++k) {
            const int ip = own_idx<NT, NSL>(q0, p0, e0 + k);
            x[k] = S[FCN_IDX(ip, C::PADN, 27)];
            u[k] = need_u ? fma(lp[e0 + k], omc, carry) : T(0);
        }
        T phi[UN], lna[UN];
#pragma unroll
        for (int k = 0; k < UN; ++k) {
            const T ih = cnorm(x[k]) * c.inv_is;
            nl_terms(ih, powk<(KT > 0 ? KT - 1 : 0)>(ih, c.K - 1), u[k], c, &phi[k], &lna[k]);
        }
        bool small = false;
        if constexpr (sizeof(T) == 4) {
            small = true;
#pragma unroll
            for (int k = 0; k < UN; ++k) small = small && nl_small(phi[k], lna[k]);
        }
        if (small) {
            // the common case, decided once for the group of points
#pragma unroll
            for (int k = 0; k < UN; ++k) {
                if constexpr (sizeof(T) == 4)
                    S[own_idx<NT, NSL>(q0, p0, e0 + k)] = nl_apply_small(x[k], phi[k], lna[k]);
            }
        } else {
#pragma unroll
            for (int k = 0; k < UN; ++k) S[own_idx<NT, NSL>(q0, p0, e0 + k)] = nl_apply_general(x[k], phi[k], lna[k]);
        }
        if (STORE_U) {
#pragma unroll
            for (int k = 0; k < UN; ++k) U[FCN_IDX((own_idx<NT, NSL>(q0, p0, e0 + k)), C::PADN, 31)] = u[k];
        }
    }
}

// Reduction of NV FP64 values across the TPR threads of a row in one pass
// (warp shuffles, then one exchange of the warp partials); mx[k] selects max
// instead of sum for value k.  Results valid in thread t = 0.
template <int NT, int NV>
__device__ __forceinline__ void row_reduce(double (&x)[NV], const bool (&mx)[NV], int t, double *scr,
                                           int rloc) {
    using C = RowCfg<NT>;
    constexpr int W = C::TPR < 32 ? C::TPR : 32;
#pragma unroll
    for (int d = W / 2; d >= 1; d >>= 1) {
#pragma unroll
        for (int k = 0; k < NV; ++k) {
            const double o = __shfl_down_sync(0xffffffffu, x[k], d, W);
            x[k] = mx[k] ? fmax(x[k], o) : x[k] + o;
        }
    }
    if (C::WARPS_PER_ROW > 1) {
        static_assert(C::WARPS_PER_ROW * NV <= kRowScratch, "row scratch");
        __syncthreads();
        if ((t & 31) == 0) {
#pragma unroll
            for (int k = 0; k < NV; ++k)
                scr[FCN_IDX((rloc * C::WARPS_PER_ROW + (t >> 5)) * NV + k, kRowScratch, 18)] = x[k];
        }
        __syncthreads();
        if (t == 0) {
#pragma unroll
            for (int k = 0; k < NV; ++k) {
                double acc = scr[FCN_IDX(rloc * C::WARPS_PER_ROW * NV + k, kRowScratch, 20)];
                for (int w = 1; w < C::WARPS_PER_ROW; ++w) {
                    const double o = scr[FCN_IDX((rloc * C::WARPS_PER_ROW + w) * NV + k, kRowScratch, 21)];
                    acc = mx[k] ? fmax(acc, o) : acc + o;
                }
                x[k] = acc;
            }
        }
        __syncthreads();
    }
}

// Compensated (Kahan) FP32 running sum: the per-thread partials of the FP32
// path keep float relative accuracy whatever the count; rows and the final
// reductions are FP64.
struct KahanF {
    float s = 0.f, c = 0.f;
    __device__ __forceinline__ void add(float v) {
        const float y = v - c;
        const float t2 = s + y;
        c = (t2 - s) - y;
        s = t2;
    }
};

// MB: minimum resident CTAs per SM requested from the compiler (register cap
// 64K / (MB * THREADS)); the autotuner picks it per (precision, Nt).
// One CTA of TH threads processes rows [row_base, row_base + TH/TPR) of one
// pulse: TH = RowCfg<NT>::THREADS in the per-Nt kernels, 512 in the batched
// work-list kernel.  Every thread of the CTA must call it (barriers inside).
struct NoHook {
    __device__ __forceinline__ void operator()() const {}
};

// The time-domain store of a row (when `store`) and the step-doubling norm's
// sums of the stored row A against cmp (diff[2 row] = sum |cmp - A|^2,
// diff[2 row + 1] = sum |A|^2; per-thread sums in the working precision over
// the thread's few points, FP64 from the row sum on).  Called by every
// thread of the CTA (row_reduce has block barriers).
template <typename T, int NT>
__device__ __forceinline__ void row_store_diff(cx<T> *g, const cx<T> *S, const cx<T> *cmp, double *diff, int nr,
                                               int row, int t, bool valid, bool store, double *scr, int rloc) {
    using C = RowCfg<NT>;
    constexpr int E = C::E;
    T d2 = T(0), b2 = T(0);
    const cx<T> *gc = cmp ? cmp + (size_t)(valid ? row : 0) * C::N : nullptr;
    auto acc = [&](cx<T> x, cx<T> y) {             // x: stored value, y: compared value
        const T dx = y.x - x.x, dy = y.y - x.y;
        d2 = fma(dx, dx, fma(dy, dy, d2));
        b2 = fma(x.x, x.x, fma(x.y, x.y, b2));
    };
    if (store && valid) {
        if (row_io_chunks<T, NT>(g) && (!gc || row_io_chunks<T, NT>(gc))) {
            using IO = RowIo<T, NT>;
            row_chunks<T, NT>(t, [&](int tau, int cq0, int cp0) {
                cx<T> cv[IO::CPC];
#pragma unroll
                for (int m = 0; m < IO::CPC; ++m)
                    cv[m] = S[FCN_IDX((own_idx<NT, IO::NSL>(cq0, cp0, (tau & 15) + m)), C::PADN, 11)];
                st_chunk<T>(g + FCN_IDX(tau, IO::N - IO::CPC + 1, 10), cv);
                if (gc) {
                    cx<T> yv[IO::CPC];
                    ld_chunk<T>(gc + FCN_IDX(tau, IO::N - IO::CPC + 1, 32), yv);
#pragma unroll
                    for (int m = 0; m < IO::CPC; ++m) acc(cv[m], yv[m]);
                }
            });
        } else {
#pragma unroll
            for (int i = 0; i < E; ++i) {
                const int idx = t + C::TPR * i;
                const cx<T> x = S[FCN_IDX(pidx(tpos<NT>(idx), fft_nt(NT)), C::PADN, 11)];
                g[FCN_IDX(idx, fft_nt(NT), 10)] = x;
                if (gc) acc(x, gc[FCN_IDX(idx, fft_nt(NT), 32)]);
            }
        }
    }
    double v2[2] = {double(d2), double(b2)};
    const bool sk[2] = {false, false};
    row_reduce<NT, 2>(v2, sk, t, scr, rloc);
    if (t == 0 && valid && diff) {
        diff[FCN_IDX((size_t)2 * row, (size_t)2 * nr, 33)] = v2[0];
        diff[FCN_IDX((size_t)2 * row + 1, (size_t)2 * nr, 34)] = v2[1];
    }
    __syncthreads();                               // the scratch is reused
}

// One row stage of RPC rows.  PF: the input rows were staged in shared memory
// (xs: RPC rows of Nt values in natural order, row_base's first) and are read
// from there; hook() runs once every thread has finished reading them (the
// prefetch of the next rows may then overwrite xs).
template <typename T, int NT, int KT, int TH, bool PF = false, typename Hook = NoHook, bool DIFFK = false>
__device__ __forceinline__ void row_body(const RowArgs<T> &a, int row_base, int ops,
                                         unsigned char *smem_raw, const cx<T> *xs = nullptr,
                                         Hook hook = Hook(), const RowMultiArgs<T> *mp = nullptr) {
    using C = RowCfg<NT>;
    constexpr int E = C::E;
    constexpr int RPC = TH / C::TPR;
    static_assert(RPC * C::TPR == TH, "CTA size must hold whole rows");
    // shared memory: the rows S, the FP64 scratch, then the u rows U, which
    // only launches with rho or statistics output allocate
    cx<T> *S_all = reinterpret_cast<cx<T> *>(smem_raw);
    double *scr = reinterpret_cast<double *>(S_all + RPC * C::PADN);
    T *U_all = reinterpret_cast<T *>(scr + kRowScratch);

#ifdef FCN_CHECKED
    {
        unsigned dsm;
        asm volatile("mov.u32 %0, %%dynamic_smem_size;" : "=r"(dsm));
        const bool with_u = (ops & (OP_RHO | OP_STATS)) != 0;
        if (threadIdx.x == 0)
            FCN_IDX((sizeof(cx<T>) + (with_u ? sizeof(T) : 0)) * RPC * C::PADN + sizeof(double) * kRowScratch - 1,
                    dsm, 25);
    }
#endif
    const int tid = threadIdx.x;
    const int rloc = tid / C::TPR;
    const int t = tid - rloc * C::TPR;
    const int row = row_base + rloc;
    const bool valid = row < a.nr;
    cx<T> *S = S_all + rloc * C::PADN;
    T *U = U_all + rloc * C::PADN;
    cx<T> *g = a.field + (size_t)(valid ? row : 0) * C::N;
    // the row's input: the field itself, or a separate source (out of place)
    const cx<T> *gin = a.in ? a.in + (size_t)(valid ? row : 0) * C::N : g;

    cx<T> v[E];
    if (ops & OP_IFFT) {
        // the inverse's first pass (the adjoint of the last forward pass) takes
        // its operands straight from HBM: X[j + r*NS], j = t + TPR*i, coalesced
        constexpr int PL = C::NPASS - 1;
        constexpr int RL = PassCfg<NT, PL>::R;
        constexpr int NSL = PassCfg<NT, PL>::NS;
        const cx<T> *src = PF ? xs + rloc * C::N : gin;
#pragma unroll
        for (int i = 0; i < E / RL; ++i) {
            const int j = t + C::TPR * i;
#pragma unroll
            for (int r = 0; r < RL; ++r)
                v[i * RL + r] = valid ? src[FCN_IDX(j + r * NSL, fft_nt(NT), 4)] : mk(T(0), T(0));
        }
        InvDispatch<T, NT, PL, (PL < 0)>::run(v, S, t, C::PLAN ? a.tw1 : a.tw, a.nl.inv_nt);
        hook();
    } else {
        const cx<T> *src = PF ? xs + rloc * C::N : gin;
        if (!PF && row_io_chunks<T, NT>(src)) {
            using IO = RowIo<T, NT>;
            row_chunks<T, NT>(t, [&](int tau, int cq0, int cp0) {
                cx<T> cv[IO::CPC];
                if (valid) {
                    ld_chunk<T>(src + FCN_IDX(tau, IO::N - IO::CPC + 1, 6), cv);
                } else {
#pragma unroll
                    for (int m = 0; m < IO::CPC; ++m) cv[m] = mk(T(0), T(0));
                }
#pragma unroll
                for (int m = 0; m < IO::CPC; ++m)
                    S[FCN_IDX((own_idx<NT, IO::NSL>(cq0, cp0, (tau & 15) + m)), C::PADN, 5)] = cv[m];
            });
        } else {
#pragma unroll
            for (int i = 0; i < E; ++i) {
                const int idx = t + C::TPR * i;
                S[FCN_IDX(pidx(tpos<NT>(idx), fft_nt(NT)), C::PADN, 5)] = valid ? src[FCN_IDX(idx, fft_nt(NT), 6)] : mk(T(0), T(0));
            }
        }
        __syncthreads();
        hook();
    }

    // the time-domain stage runs whenever the row passes through tau space
    // (nonlinear step, statistics, rho output) or the 1/Nt of an inverse
    // transform has to be applied; it works in place on S
    const bool time_work = (ops & (OP_NL | OP_STATS | OP_RHO | OP_IFFT)) != 0;
    if (time_work) {
        const bool need_u = (a.nl.flags & (PH_PLASMA | PH_MPI_SAT)) || (ops & (OP_RHO | OP_STATS));
        const bool keep_u = (ops & (OP_RHO | OP_STATS)) != 0;
        bool have_u = false;
        const int nhalf = ((ops & OP_NL) ? 1 : 0) + ((ops & OP_NL2) ? 1 : 0);
        for (int hs = 0; hs < nhalf; ++hs) {
            if (keep_u && hs + 1 == nhalf)
                nl_half_smem<T, NT, KT, true>(S, U, t, a.nl, need_u, scr, rloc);
            else
                nl_half_smem<T, NT, KT, false>(S, U, t, a.nl, need_u, scr, rloc);
            have_u = need_u;
            __syncthreads();
        }
        // statistics of the final row; rho is written below, coalesced
        if (ops & (OP_STATS | OP_RHO)) {
            // v = {sum |A|^2, max |A|^2, max u, count of non-finite |A|^2}
            double v4[4] = {0.0, 0.0, 0.0, 0.0};
            if (ops & OP_STATS) {
                if constexpr (sizeof(T) == 4) {
                    KahanF ks;
                    float mxf = 0.f, muf = 0.f, badf = 0.f;
#pragma unroll 4
                    for (int e = 0; e < E; ++e) {
                        const int ip = own_idx<NT, PassCfg<NT, C::NPASS - 1>::NS>(pidx(tpos<NT>(E * t), fft_nt(NT)),
                                                                                  tpos<NT>(E * t), e);
                        const cx<T> x = S[FCN_IDX(ip, C::PADN, 29)];
                        const float i2 = fmaf(x.x, x.x, x.y * x.y);
                        if (!isfinite(i2)) badf += 1.f;
                        ks.add(i2);
                        mxf = fmaxf(mxf, i2);
                        if (have_u) muf = fmaxf(muf, U[ip]);
                    }
                    v4[0] = double(ks.s) - double(ks.c);
                    v4[1] = mxf;
                    v4[2] = muf;
                    v4[3] = badf;
                } else {
#pragma unroll 4
                    for (int e = 0; e < E; ++e) {
                        const int ip = own_idx<NT, PassCfg<NT, C::NPASS - 1>::NS>(pidx(tpos<NT>(E * t), fft_nt(NT)),
                                                                                  tpos<NT>(E * t), e);
                        const cx<T> x = S[FCN_IDX(ip, C::PADN, 29)];
                        const double i2 = double(x.x) * double(x.x) + double(x.y) * double(x.y);
                        if (!isfinite(i2)) v4[3] += 1.0;
                        v4[0] += i2;
                        v4[1] = fmax(v4[1], i2);
                        if (have_u) v4[2] = fmax(v4[2], double(U[ip]));
                    }
                }
            }
            if ((ops & OP_STATS) && a.stats) {
                const bool mxk[4] = {false, true, true, false};
                row_reduce<NT, 4>(v4, mxk, t, scr, rloc);
                if (t == 0 && valid) {
                    double *st = a.stats + FCN_IDX((size_t)row * NSTAT, (size_t)a.nr * NSTAT, 23);
                    st[ST_SUM_I] = v4[0];
                    st[ST_MAX_I] = v4[1];
                    if (ops & (OP_NL | OP_NL2)) st[ST_MAX_U] = v4[2];
                    st[ST_NONFINITE] = v4[3];
                }
            }
            __syncthreads();
            if ((ops & OP_RHO) && valid && a.rho) {
                T *rr = a.rho + (size_t)row * C::N;
                if (row_io_real_chunks<T, NT>(rr)) {
                    // 16-byte chunks in the sector-wise order of the field rows
                    using IO = RowIoReal<T, NT>;
                    constexpr int NSL = PassCfg<NT, C::NPASS - 1>::NS;
                    row_real_chunks<T, NT>(t, [&](int tau) {
                        const int cp0 = tpos<NT>(tau & ~15);
                        const int cq0 = pidx(cp0, fft_nt(NT));
                        T w[IO::RC];
#pragma unroll
                        for (int m = 0; m < IO::RC; ++m)
                            w[m] = have_u ? U[FCN_IDX((own_idx<NT, NSL>(cq0, cp0, (tau & 15) + m)), C::PADN, 30)] *
                                                a.nl.rho_nt
                                          : T(0);
                        T *dst = rr + FCN_IDX(tau, IO::N - IO::RC + 1, 12);
                        if constexpr (sizeof(T) == 4) *reinterpret_cast<float4 *>(dst) = make_float4(w[0], w[1], w[2], w[3]);
                        else *reinterpret_cast<double2 *>(dst) = make_double2(w[0], w[1]);
                    });
                } else {
                    // consecutive threads write consecutive tau points
#pragma unroll
                    for (int i = 0; i < E; ++i) {
                        const int idx = t + C::TPR * i;
                        rr[FCN_IDX(idx, fft_nt(NT), 12)] =
                            have_u ? U[FCN_IDX(pidx(tpos<NT>(idx), fft_nt(NT)), C::PADN, 30)] * a.nl.rho_nt : T(0);
                    }
                }
            }
        }
        if constexpr (DIFFK) {
            // the kernels of launches with OP_DIFF: the store and the norm sums
            // (a multi-pulse launch's per-pulse pointers from its parameters)
            const bool store = (!(ops & OP_FFT) || (ops & OP_SPEC_OF_TIME)) && !(ops & OP_NOSTORE);
            const cx<T> *cmp = mp ? mp->cmp[blockIdx.y] : a.cmp;
            double *diff = mp ? mp->diff[blockIdx.y] : a.diff;
            row_store_diff<T, NT>(g, S, cmp, diff, a.nr, row, t, valid, store, scr, rloc);
        } else if ((!(ops & OP_FFT) || (ops & OP_SPEC_OF_TIME)) && !(ops & OP_NOSTORE) && valid) {
            if (row_io_chunks<T, NT>(g)) {
                using IO = RowIo<T, NT>;
                row_chunks<T, NT>(t, [&](int tau, int cq0, int cp0) {
                    cx<T> cv[IO::CPC];
#pragma unroll
                    for (int m = 0; m < IO::CPC; ++m)
                        cv[m] = S[FCN_IDX((own_idx<NT, IO::NSL>(cq0, cp0, (tau & 15) + m)), C::PADN, 11)];
                    st_chunk<T>(g + FCN_IDX(tau, IO::N - IO::CPC + 1, 10), cv);
                });
            } else {
#pragma unroll
                for (int i = 0; i < E; ++i) {
                    const int idx = t + C::TPR * i;
                    g[FCN_IDX(idx, fft_nt(NT), 10)] = S[FCN_IDX(pidx(tpos<NT>(idx), fft_nt(NT)), C::PADN, 11)];
                }
            }
        }
        // the in-place transform below overwrites S: every thread's store first
        if (ops & OP_SPEC_OF_TIME) __syncthreads();
    }

    if (ops & OP_FFT) {
        FwdDispatch<T, NT, 0, (C::NPASS <= 0)>::run(v, S, t, C::PLAN ? a.tw1 : a.tw);
        // last-pass outputs: index j + r*NS, j = t + TPR*i
        constexpr int PL = C::NPASS - 1;
        constexpr int R = PassCfg<NT, PL>::R;
        constexpr int NS = PassCfg<NT, PL>::NS;
        constexpr int NB = E / R;
        if (!(ops & (OP_NOSTORE | OP_SPEC_OF_TIME)) && valid) {
#pragma unroll
            for (int i = 0; i < NB; ++i) {
                const int j = t + C::TPR * i;
#pragma unroll
                for (int r = 0; r < R; ++r) g[FCN_IDX(j + r * NS, fft_nt(NT), 13)] = v[i * R + r];
            }
        }
        if ((ops & OP_SPEC) && a.stats) {
            // spectral moments sum_q w^k |A_q|^2, w = signed bin, k = 0, 1, 2
            double m3[3] = {0.0, 0.0, 0.0};
            if constexpr (sizeof(T) == 4) {
                KahanF k0, k1, k2;
#pragma unroll
                for (int i = 0; i < NB; ++i) {
                    const int j = t + C::TPR * i;
#pragma unroll
                    for (int r = 0; r < R; ++r) {
                        const int q = j + r * NS;
                        const float w = float(q < C::N / 2 ? q : q - C::N);
                        const cx<T> x = v[i * R + r];
                        const float p2 = fmaf(x.x, x.x, x.y * x.y);
                        k0.add(p2);
                        k1.add(w * p2);
                        k2.add(w * w * p2);
                    }
                }
                m3[0] = double(k0.s) - double(k0.c);
                m3[1] = double(k1.s) - double(k1.c);
                m3[2] = double(k2.s) - double(k2.c);
            } else {
#pragma unroll
                for (int i = 0; i < NB; ++i) {
                    const int j = t + C::TPR * i;
#pragma unroll
                    for (int r = 0; r < R; ++r) {
                        const int q = j + r * NS;
                        const double w = double(q < C::N / 2 ? q : q - C::N);
                        const cx<T> x = v[i * R + r];
                        const double p2 = double(x.x) * double(x.x) + double(x.y) * double(x.y);
                        m3[0] += p2;
                        m3[1] += w * p2;
                        m3[2] += w * w * p2;
                    }
                }
            }
            const bool mxk[3] = {false, false, false};
            row_reduce<NT, 3>(m3, mxk, t, scr, rloc);
            if (t == 0 && valid) {
                double *st = a.stats + FCN_IDX((size_t)row * NSTAT, (size_t)a.nr * NSTAT, 24);
                st[ST_S0] = m3[0];
                st[ST_S1] = m3[1];
                st[ST_S2] = m3[2];
            }
        }
    }
}

// DIFFK: the kernels for launches with OP_DIFF (the closing launch of a
// step-doubling attempt); the others are compiled without that code, so
// that it does not weigh on the register allocation of the launch that runs
// at almost every z-step.
template <typename T, int NT, int KT, int MB, bool DIFFK = false>
__global__ void __launch_bounds__(RowCfg<NT>::THREADS, MB)
row_kernel(RowArgs<T> a) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    pdl_enter();
    if constexpr (DIFFK)
        row_body<T, NT, KT, RowCfg<NT>::THREADS, false, NoHook, true>(a, blockIdx.x * RowCfg<NT>::RPC, a.ops,
                                                                       smem_raw);
    else
        row_body<T, NT, KT, RowCfg<NT>::THREADS>(a, blockIdx.x * RowCfg<NT>::RPC, a.ops, smem_raw);
}

// Several pulses of one grid and one set of coefficients in one launch:
// blockIdx.y selects the pulse (its field, rho and statistics pointers; all
// else is shared).  One launch over all pulses fills the waves that a launch
// per pulse leaves part-empty.
template <typename T, int NT, int KT, int MB, bool DIFFK = false>
__global__ void __launch_bounds__(RowCfg<NT>::THREADS, MB)
row_kernel_multi(const __grid_constant__ RowMultiArgs<T> m) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    pdl_enter();
    RowArgs<T> a = m.a;
    a.field = m.field[blockIdx.y];
    a.rho = m.rho[blockIdx.y];
    a.stats = m.stats[blockIdx.y];
    a.in = m.in[blockIdx.y];
    if constexpr (DIFFK)
        row_body<T, NT, KT, RowCfg<NT>::THREADS, false, NoHook, true>(a, blockIdx.x * RowCfg<NT>::RPC, a.ops,
                                                                       smem_raw, nullptr, NoHook(), &m);
    else
        row_body<T, NT, KT, RowCfg<NT>::THREADS>(a, blockIdx.x * RowCfg<NT>::RPC, a.ops, smem_raw);
}

// Persistent row stage with the next rows prefetched: each CTA walks the
// units (RPC consecutive rows of one pulse) u = blockIdx.x, + gridDim.x, ...
// of the launch's pulses; while it transforms and steps one unit, one bulk
// copy (cp.async.bulk, completion on an mbarrier) brings the next unit's
// rows from HBM into a staging buffer, so no thread waits on a global load
// when a unit starts.  The wait on the mbarrier is bounded (~1 s): after it
// the CTA records an error code, waits (bounded) for its copy in flight and
// returns.
constexpr long long kRowWaitCycles = 1ll << 31;

__device__ __forceinline__ bool row_mbar_wait(uint32_t bar, uint32_t parity) {
    uint32_t ok = 0;
    const long long t0 = clock64();
    for (;;) {
        asm volatile(
            "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
            " selp.u32 %0, 1, 0, p;\n}\n"
            : "=r"(ok)
            : "r"(bar), "r"(parity)
            : "memory");
        if (ok) return true;
        if (clock64() - t0 > kRowWaitCycles) return false;
    }
}

// Byte offset of the staging buffer: after the rows, the FP64 scratch and
// (launches with rho or statistics) the u rows, 128-byte aligned.
template <typename T, int NT>
__host__ __device__ constexpr size_t pf_stage_offset(bool with_u) {
    using C = RowCfg<NT>;
    return ((sizeof(cx<T>) + (with_u ? sizeof(T) : 0)) * C::RPC * C::PADN + sizeof(double) * kRowScratch +
            127) / 128 * 128;
}

template <typename T, int NT, int KT, int MB>
__global__ void __launch_bounds__(RowCfg<NT>::THREADS, MB)
row_kernel_pf(const __grid_constant__ RowMultiArgs<T> m, int npulse, int *err) {
    using C = RowCfg<NT>;
    extern __shared__ __align__(128) unsigned char smem_raw[];
    pdl_enter();
    const RowArgs<T> &a0 = m.a;
    const int upp = (a0.nr + C::RPC - 1) / C::RPC;      // units per pulse
    const int units = upp * npulse;
    if ((int)blockIdx.x >= units) return;
    const bool with_u = (a0.ops & (OP_RHO | OP_STATS)) != 0;
    cx<T> *xs = reinterpret_cast<cx<T> *>(smem_raw + pf_stage_offset<T, NT>(with_u));
    const uint32_t bar = (uint32_t)__cvta_generic_to_shared(xs + C::RPC * C::N);
    auto issue = [&](int u) {                           // thread 0 only
        const int pulse = u / upp, row0 = (u - pulse * upp) * C::RPC;
        const int rows = min(C::RPC, a0.nr - row0);
        const uint32_t bytes = (uint32_t)(rows * C::N * sizeof(cx<T>));
        const cx<T> *src = (m.in[pulse] ? m.in[pulse] : m.field[pulse]) + (size_t)row0 * C::N;
        asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
        asm volatile(
            "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];"
            ::"r"((uint32_t)__cvta_generic_to_shared(xs)), "l"(src), "r"(bytes), "r"(bar)
            : "memory");
    };
    if (threadIdx.x == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(bar) : "memory");
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        issue(blockIdx.x);
    }
    __syncthreads();
    uint32_t parity = 0;
    for (int u = blockIdx.x; u < units; u += gridDim.x, parity ^= 1u) {
        if (!row_mbar_wait(bar, parity)) {
            if (threadIdx.x == 0 && err) atomicExch(err, 2);
            row_mbar_wait(bar, parity);                 // the copy in flight, bounded
            return;
        }
        const int pulse = u / upp, row0 = (u - pulse * upp) * C::RPC;
        RowArgs<T> a = a0;
        a.field = m.field[pulse];
        a.rho = m.rho[pulse];
        a.stats = m.stats[pulse];
        const int next = u + gridDim.x;
        row_body<T, NT, KT, C::THREADS, true>(a, row0, a.ops, smem_raw, xs, [&] {
            if (threadIdx.x == 0 && next < units) issue(next);
        });
        __syncthreads();                                // S and the scratch are reused
    }
}

// Batched work list: each item (pulse, first row) covers 512 / (Nt/16) rows of
// one pulse; pulses may have different Nr and Nt (Nt = 512 ... 8192).  A
// persistent grid pulls items from a global counter, largest rows first.
template <typename T, int KT>
__global__ void __launch_bounds__(512, 1)
row_batch_kernel(const RowArgs<T> *__restrict__ pulses, const int2 *__restrict__ items, int nitems,
                 int ops, unsigned *counter) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ int next;
    for (;;) {
        if (threadIdx.x == 0) next = (int)atomicAdd(counter, 1u);
        __syncthreads();
        const int it = next;
        __syncthreads();
        if (it >= nitems) break;
        const int2 w = items[it];
        const RowArgs<T> a = pulses[w.x];
        switch (a.nt) {
            case 512: row_body<T, 512, KT, 512>(a, w.y, ops, smem_raw); break;
            case 1024: row_body<T, 1024, KT, 512>(a, w.y, ops, smem_raw); break;
            case 2048: row_body<T, 2048, KT, 512>(a, w.y, ops, smem_raw); break;
            case 4096: row_body<T, 4096, KT, 512>(a, w.y, ops, smem_raw); break;
            default: row_body<T, 8192, KT, 512>(a, w.y, ops, smem_raw); break;
        }
        __syncthreads();
    }
    // the last CTA out resets the counter for the next launch
    if (threadIdx.x == 0) {
        const unsigned done = atomicAdd(counter + 1, 1u) + 1;
        if (done == gridDim.x) {
            counter[0] = 0;
            counter[1] = 0;
        }
    }
}
}  // namespace

namespace rowimpl {

// Rows S and the FP64 scratch, plus the u rows when the launch outputs rho
// or statistics.
template <typename T, int NT>
size_t smem_bytes(bool with_u = true) {
    using C = RowCfg<NT>;
    return (sizeof(cx<T>) + (with_u ? sizeof(T) : 0)) * C::RPC * C::PADN + sizeof(double) * kRowScratch;
}

// Sets the dynamic shared-memory limit of the kernel; must run before any
// launch of it (and outside stream capture).
// Occupancy variants: v = 0 is the compiler's natural allocation; v = 1, 2
// ask for 3 and 4 CTAs of 256 threads per SM (80 and 64 registers), or 2 CTAs
// of 512 threads for Nt = 8192.  Only FP32 with K = 8 and Nt >= 256 has
// variants (smaller rows are cheap; their variants map to v = 0).
template <int NT>
constexpr int mb_of(int v) {
    return RowCfg<NT>::THREADS >= 512 ? (v == 0 ? 1 : 2) : (v == 0 ? 1 : (v == 1 ? 3 : 4));
}

template <typename T, int NT, int KT, int MB>
cudaError_t set_smem_attr() {
    cudaError_t e = cudaSuccess;
    for (int d = 0; d < 2 && e == cudaSuccess; ++d) {
        e = cudaFuncSetAttribute(d ? row_kernel<T, NT, KT, MB, true> : row_kernel<T, NT, KT, MB, false>,
                                 cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_bytes<T, NT>());
        if (e == cudaSuccess)
            e = cudaFuncSetAttribute(d ? row_kernel_multi<T, NT, KT, MB, true> : row_kernel_multi<T, NT, KT, MB, false>,
                                     cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_bytes<T, NT>());
    }
    return e;
}

// The prefetching persistent variant (3): FP32, K = 8, Nt >= 512; 3 CTAs of
// 256 threads per SM (the staging buffer leaves no room for a fourth), or
// 1 CTA of 512 threads for Nt = 8192.
template <int NT>
constexpr int mb_pf() { return RowCfg<NT>::THREADS >= 512 ? 1 : 3; }
template <typename T, int NT>
constexpr bool has_pf() { return sizeof(T) == 4 && fft_nt(NT) >= 512 && fft_plan(NT) == 0; }
template <typename T, int NT>
size_t pf_smem_bytes(bool with_u) {
    return pf_stage_offset<T, NT>(with_u) + sizeof(cx<T>) * RowCfg<NT>::RPC * RowCfg<NT>::N + 16;
}

template <typename T, int NT>
cudaError_t prepare_nt() {
    cudaError_t e = set_smem_attr<T, NT, 0, 1>();
    if (e == cudaSuccess) e = set_smem_attr<T, NT, 8, 1>();
    if constexpr (sizeof(T) == 4 && fft_nt(NT) >= 256) {
        constexpr int NT1 = fft_tag(NT, 1);
        if (e == cudaSuccess) e = set_smem_attr<T, NT, 8, mb_of<NT>(1)>();
        if (e == cudaSuccess) e = set_smem_attr<T, NT, 8, mb_of<NT>(2)>();
        if (e == cudaSuccess) e = set_smem_attr<T, NT1, 8, mb_of<NT1>(1)>();
        if (e == cudaSuccess) e = set_smem_attr<T, NT1, 8, mb_of<NT1>(2)>();
    }
    if constexpr (has_pf<T, NT>()) {
        if (e == cudaSuccess)
            e = cudaFuncSetAttribute(row_kernel_pf<T, NT, 8, mb_pf<NT>()>,
                                     cudaFuncAttributeMaxDynamicSharedMemorySize, (int)pf_smem_bytes<T, NT>(true));
    }
    return e;
}

// Launch of the prefetching variant over npulse pulses: one CTA per SM slot
// (occupancy queried once), each walking units of RPC rows.
template <typename T, int NT>
cudaError_t launch_nt_pf(const RowMultiArgs<T> &m, int npulse, cudaStream_t st) {
    using C = RowCfg<NT>;
    if constexpr (!has_pf<T, NT>()) {
        return cudaErrorInvalidConfiguration;
    } else {
        const RowArgs<T> &a = m.a;
        const bool with_u = (a.ops & (OP_RHO | OP_STATS)) != 0;
        const size_t smem = pf_smem_bytes<T, NT>(with_u);
        const int units = (a.nr + C::RPC - 1) / C::RPC * npulse;
        if (units <= 0) return cudaSuccess;
        auto k = row_kernel_pf<T, NT, 8, mb_pf<NT>()>;
        static int slots[2] = {0, 0};
        int &sl = slots[with_u ? 1 : 0];
        if (!sl) {
            int dev = 0, sms = 0, occ = 0;
            cudaError_t e = cudaGetDevice(&dev);
            if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
            if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k, C::THREADS, smem);
            if (e != cudaSuccess) return e;
            sl = sms * (occ > 0 ? occ : 1);
        }
        const int grid = units < sl ? units : sl;
        return launch_k(k, dim3(grid), dim3(C::THREADS), smem, st, m, npulse, a.err);
    }
}

// The kernel of the launch's variant (K = 8: unrolled powers; other K: the
// generic kernel), compiled with the norm sums (DIFFK) or without.
template <typename T, int NT, bool DIFFK>
auto multi_kernel_for(const RowArgs<T> &a) -> void (*)(const RowMultiArgs<T>) {
    if (a.nl.K != 8) return row_kernel_multi<T, NT, 0, 1, DIFFK>;
    void (*k)(const RowMultiArgs<T>) = row_kernel_multi<T, NT, 8, 1, DIFFK>;
    if constexpr (sizeof(T) == 4 && fft_nt(NT) >= 256) {
        constexpr int NT1 = fft_tag(NT, 1);
        if (a.variant == 1) k = row_kernel_multi<T, NT, 8, mb_of<NT>(1), DIFFK>;
        else if (a.variant == 2) k = row_kernel_multi<T, NT, 8, mb_of<NT>(2), DIFFK>;
        else if (a.variant == 4 && a.tw1) k = row_kernel_multi<T, NT1, 8, mb_of<NT1>(1), DIFFK>;
        else if (a.variant == 5 && a.tw1) k = row_kernel_multi<T, NT1, 8, mb_of<NT1>(2), DIFFK>;
    }
    return k;
}

template <typename T, int NT, bool DIFFK>
auto kernel_for(const RowArgs<T> &a) -> void (*)(RowArgs<T>) {
    if (a.nl.K != 8) return row_kernel<T, NT, 0, 1, DIFFK>;
    void (*k)(RowArgs<T>) = row_kernel<T, NT, 8, 1, DIFFK>;
    if constexpr (sizeof(T) == 4 && fft_nt(NT) >= 256) {
        constexpr int NT1 = fft_tag(NT, 1);
        if (a.variant == 1) k = row_kernel<T, NT, 8, mb_of<NT>(1), DIFFK>;
        else if (a.variant == 2) k = row_kernel<T, NT, 8, mb_of<NT>(2), DIFFK>;
        else if (a.variant == 4 && a.tw1) k = row_kernel<T, NT1, 8, mb_of<NT1>(1), DIFFK>;
        else if (a.variant == 5 && a.tw1) k = row_kernel<T, NT1, 8, mb_of<NT1>(2), DIFFK>;
    }
    return k;
}

template <typename T, int NT>
cudaError_t launch_nt_multi(const RowMultiArgs<T> &m, int npulse, cudaStream_t st) {
    using C = RowCfg<NT>;
    const RowArgs<T> &a = m.a;
    const size_t smem = smem_bytes<T, NT>((a.ops & (OP_RHO | OP_STATS)) != 0);
    const dim3 grid((a.nr + C::RPC - 1) / C::RPC, npulse);
    if (grid.x == 0 || npulse <= 0) return cudaSuccess;
    if (npulse > kRowMulti) return cudaErrorInvalidValue;
    const bool dk = (a.ops & OP_DIFF) != 0;
    if constexpr (has_pf<T, NT>())
        if (a.variant == 3 && a.nl.K == 8 && !dk) return launch_nt_pf<T, NT>(m, npulse, st);
    void (*k)(const RowMultiArgs<T>) = dk ? multi_kernel_for<T, NT, true>(a) : multi_kernel_for<T, NT, false>(a);
    return launch_k(k, grid, dim3(C::THREADS), smem, st, m);
}

template <typename T, int NT>
cudaError_t launch_nt(const RowArgs<T> &a, cudaStream_t st) {
    using C = RowCfg<NT>;
    const size_t smem = smem_bytes<T, NT>((a.ops & (OP_RHO | OP_STATS)) != 0);
    const int grid = (a.nr + C::RPC - 1) / C::RPC;
    if (grid == 0) return cudaSuccess;
    const bool dk = (a.ops & OP_DIFF) != 0;
    if constexpr (has_pf<T, NT>()) {
        if (a.variant == 3 && a.nl.K == 8 && !dk) {
            RowMultiArgs<T> m;
            m.a = a;
            for (int c = 0; c < kRowMulti; ++c) {
                m.field[c] = a.field;
                m.rho[c] = a.rho;
                m.stats[c] = a.stats;
                m.in[c] = a.in;
            }
            return launch_nt_pf<T, NT>(m, 1, st);
        }
    }
    // K = 8 (the photon number of 800 nm in air) gets unrolled powers
    void (*k)(RowArgs<T>) = dk ? kernel_for<T, NT, true>(a) : kernel_for<T, NT, false>(a);
    return launch_k(k, dim3(grid), dim3(C::THREADS), smem, st, a);
}

}  // namespace rowimpl

}  // namespace fcn
