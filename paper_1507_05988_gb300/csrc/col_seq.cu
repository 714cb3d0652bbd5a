// col_seq.cu -- the column stage of the FCN z-step (Ma & Lin,
// arXiv:1507.05988, Sec. 3.1, Eqs. (matrix), (matrix1)) as one sequential
// Thomas sweep per frequency column, fed by TMA.
//
// For every frequency bin q the system M_abc^q A~^{n+1} = M_def^q A~^n has
// its pivots cached per dz (the table kernel in col_kernel.cu), so the solve
// is two first-order recurrences down and up the radial index:
//   forward   y_j = alpha_j y_{j-1} + beta_j,   beta_j = rhs_j / piv_j,
//   backward  x_j = gamma_j x_{j+1} + y_j,
// with rhs_j = d_j x_j + i (sl_j x_{j-1} + sh_j x_{j+1} - d_j (c0_j - delta_q) x_j),
// alpha_j = i sl_j / piv_j, gamma_j = i sh_j / piv_j (the CnCoef rows).
//
// One thread owns one column and runs both recurrences in order, as the
// Thomas ("chasing") method states them: no scan, no block barrier, about
// 33 instructions per point.  A warp owns 32 adjacent columns, so each row
// it touches is one 256-byte (FP32) or 512-byte (FP64) segment.  The forward
// sweep writes y_j over x_j in place (x_j is dead once row j+1 is formed) and
// the backward sweep reads y back and writes x; between the two sweeps the
// column group's y stays in L2 when the launch covers one or two pulses.
//
// Latency: a warp holds only its own columns, so it must keep many rows in
// flight.  Each warp streams its rows through a ring of S stages in shared
// memory: lane 0 issues, per stage, a 2-D TMA box of R rows x 32 columns of
// the field, a box of R rows x 34 columns of the pivot table (bins q0..q0+33,
// or the mirrored range for bins above Nt/2, which share the pivots of
// |q|), and a bulk copy of the R CnCoef rows, all signalling one mbarrier.
// Every wait on an mbarrier is bounded: after ~1 s the warp records an error
// code, waits (bounded again) for its own copies still in flight, and
// returns.  The field tensor map covers only this pulse's buffer on this GPU;
// nothing is multicast.
#include <cuda.h>
#include <cudaTypedefs.h>

#include <cstring>
#include <mutex>

#include "col_scan.cuh"

namespace fcn {
namespace {

using namespace colscan;

constexpr int kSeqMaxPulses = 8;
constexpr long long kSeqWaitCycles = 1ll << 31;     // ~1 s at 2 GHz

template <typename T>
struct SeqParams {
    CUtensorMap fmap[kSeqMaxPulses];   // field of pulse y: {E nt, nr} of 8-byte elements
    CUtensorMap tmap;                  // pivot table: {E nq, nr}, row pitch E tp
    cx<T> *field[kSeqMaxPulses];
    const CnCoef<T> *coef;             // [nr]
    int nr, nt, ngroups;
    double s64, dk64;                  // s and dk: c0 - delta_q = {4, 2} s - dk q^2
    int pivlim;                        // table entries relative to 1/p_inf (ColArgs::pivlim)
    const ColConst *cc;                // per-column constants (FP32 contexts) or null
    double disp;                       // exact dispersion factor coefficient, 0: none
    int *err;                          // set to 1 when a wait gives up (may be null)
};

__device__ __forceinline__ uint32_t smem_u32(const void *p) {
    return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ void mbar_init(uint32_t bar) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(bar) : "memory");
}

__device__ __forceinline__ void mbar_expect(uint32_t bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes)
                 : "memory");
}

__device__ __forceinline__ bool mbar_try(uint32_t bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
        " selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok)
        : "r"(bar), "r"(parity)
        : "memory");
    return ok != 0;
}

// Bounded wait for phase `parity` of the barrier; false after ~1 s.
__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity) {
    if (mbar_try(bar, parity)) return true;
    const long long t0 = clock64();
    while (!mbar_try(bar, parity))
        if (clock64() - t0 > kSeqWaitCycles) return false;
    return true;
}

__device__ __forceinline__ void tma_2d(uint32_t dst, const CUtensorMap *map, int c0, int c1, uint32_t bar) {
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];"
        ::"r"(dst), "l"(reinterpret_cast<uint64_t>(map)), "r"(c0), "r"(c1), "r"(bar)
        : "memory");
}

__device__ __forceinline__ void bulk_1d(uint32_t dst, const void *src, uint32_t bytes, uint32_t bar) {
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];"
        ::"r"(dst), "l"(src), "r"(bytes), "r"(bar)
        : "memory");
}

// Shared-memory layout of one warp's ring: per stage NP field boxes, one
// pivot box and the coefficient rows, then the S mbarriers.
template <typename T, int R, int S, int NP>
struct SeqRing {
    static constexpr int kX = ((R * 32 * (int)sizeof(cx<T>)) + 127) / 128 * 128;   // field rows
    static constexpr int kI = ((R * 34 * (int)sizeof(cx<T>)) + 127) / 128 * 128;   // pivot rows
    static constexpr int kC = ((R * (int)sizeof(CnCoef<T>)) + 127) / 128 * 128;    // coefficient rows
    static constexpr int kStage = NP * kX + kI + kC;
    static constexpr int kBytes = S * kStage + 128;
};

// One warp: 32 adjacent columns of NP pulses (launch slot blockIdx.y holds
// pulses NP y .. NP y + NP - 1).  Each thread runs the NP pulses' sweeps of
// its column side by side: the pivots, coefficients and sweep factors are
// read and formed once for all of them, and the NP recurrences are
// independent dependency chains.
template <typename T, int R, int S, int W, int NP>
__global__ void __launch_bounds__(32 * W)
cn_seq_kernel(const __grid_constant__ SeqParams<T> p) {
    using Ring = SeqRing<T, R, S, NP>;
    constexpr int E = int(sizeof(cx<T>)) / 8;          // 8-byte tensor elements per complex
    extern __shared__ __align__(128) unsigned char smem[];
    pdl_enter();
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    // groups g and ngroups-1-g use the same pivot columns: with W even they
    // share a CTA, otherwise they are adjacent CTAs
    const int ng = p.ngroups;
    int g;
    if (W % 2 == 0) {
        const int k = blockIdx.x * (W / 2) + (warp >> 1);
        g = (warp & 1) ? ng - 1 - k : k;
        if (k >= ng / 2) return;
    } else {
        const int b = blockIdx.x * W + warp;
        g = (b & 1) ? ng - 1 - (b >> 1) : (b >> 1);
        if (b >= ng) return;
    }
    const int pulse0 = NP * blockIdx.y;
    const int nr = p.nr, nt = p.nt;
    const int q0 = 32 * g;
    const int q = q0 + lane;
    const bool mirror = q0 >= nt / 2;                   // Nt/2 is a multiple of 32
    const int qq = mirror ? nt - q : q;
    const int tx = mirror ? nt - q0 - 32 : q0;          // first pivot column of the box
    const int il = mirror ? 32 - lane : lane;           // this lane's pivot column in the box
    CdCol<T> cdc;
    PivLim<T> plim;
    col_consts<T>(p.cc, p.pivlim, p.s64, p.dk64, qq, &cdc, &plim);
    const CUtensorMap *tmap = &p.tmap;
    cx<T> *col[NP];
#pragma unroll
    for (int k = 0; k < NP; ++k) col[k] = p.field[pulse0 + k] + q;

    unsigned char *ring = smem + (size_t)warp * Ring::kBytes;
    const uint32_t ring_s = smem_u32(ring);
    const uint32_t bar0 = ring_s + S * Ring::kStage;
    if (lane == 0) {
        for (int s = 0; s < S; ++s) mbar_init(bar0 + 8 * s);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncwarp();

    const int nb = (nr + R - 1) / R;
    const int ntask = 2 * nb;            // tasks 0..nb-1: forward blocks; nb..2nb-1: backward
    // block of task t and its stage; the u-th use of a stage waits for parity u & 1
    auto block_of = [&](int t) { return t < nb ? t : 2 * nb - 1 - t; };
    auto issue = [&](int t) {            // lane 0 only
        const int s = t % S;
        const int jb = R * block_of(t);
        const int rows = min(R, nr - jb);
        const uint32_t st = ring_s + s * Ring::kStage;
        const uint32_t bar = bar0 + 8 * s;
        const uint32_t cbytes = (uint32_t)(rows * (int)sizeof(CnCoef<T>));
        mbar_expect(bar, (uint32_t)(NP * R * 32 * sizeof(cx<T>) + R * 34 * sizeof(cx<T>)) + cbytes);
#pragma unroll
        for (int k = 0; k < NP; ++k) tma_2d(st + k * Ring::kX, &p.fmap[pulse0 + k], E * q0, jb, bar);
        tma_2d(st + NP * Ring::kX, tmap, E * tx, jb, bar);
        bulk_1d(st + NP * Ring::kX + Ring::kI, p.coef + jb, cbytes, bar);
    };
    int issued = 0;                      // tasks issued so far (lane 0)
    // on a wait that gives up: record it, wait (bounded) for the copies
    // still in flight so none lands after the CTA ends, and leave
    auto give_up = [&](int t) {
        if (lane == 0 && p.err) atomicExch(p.err, 1);
        for (int u = t; u < issued; ++u) mbar_wait(bar0 + 8 * (u % S), (u / S) & 1);
    };
    auto stage_x = [&](int s, int k) { return reinterpret_cast<const cx<T> *>(ring + s * Ring::kStage + k * Ring::kX); };
    auto stage_i = [&](int s) { return reinterpret_cast<const cx<T> *>(ring + s * Ring::kStage + NP * Ring::kX); };
    auto stage_c = [&](int s) {
        return reinterpret_cast<const CnCoef<T> *>(ring + s * Ring::kStage + NP * Ring::kX + Ring::kI);
    };

    if (lane == 0)
        for (; issued < min(S, nb); ++issued) issue(issued);
    __syncwarp();

    // ---------------- forward sweep ----------------
    // Each block of R rows runs as straight-line code: first every beta_j
    // and alpha_j of the block (independent across rows), then the y
    // recurrences (two dependent FMAs per row and pulse).  Rows past nr in
    // the last block compute on zero-filled data and store nothing.
    cx<T> xm[NP], x0[NP], y[NP];
#pragma unroll
    for (int k = 0; k < NP; ++k) xm[k] = x0[k] = y[k] = czero<T>();
    for (int t = 0; t < nb; ++t) {
        const int s = t % S;
        if (!mbar_wait(bar0 + 8 * s, (t / S) & 1)) { give_up(t); return; }
        cx<T> xnext[NP];                               // x of the next block's first row
#pragma unroll
        for (int k = 0; k < NP; ++k) xnext[k] = czero<T>();
        if (t + 1 < nb) {
            const int s1 = (t + 1) % S;
            if (!mbar_wait(bar0 + 8 * s1, ((t + 1) / S) & 1)) { give_up(t); return; }
#pragma unroll
            for (int k = 0; k < NP; ++k) xnext[k] = stage_x(s1, k)[lane];
        }
        const cx<T> *I = stage_i(s);
        const CnCoef<T> *Cf = stage_c(s);
        const int jb = R * t;
        const int rows = min(R, nr - jb);
        if (t == 0) {
#pragma unroll
            for (int k = 0; k < NP; ++k) x0[k] = stage_x(s, k)[lane];
        }
        cx<T> al[R], be[NP][R];
#pragma unroll
        for (int r = 0; r < R; ++r) {
            const cx<T> inv = I[r * 34 + il];
            const CnCoef<T> cf = Cf[r];
            const ExRow<T> e = ex_row(cf, jb + r == 0, cdc);
            al[r] = cmul_i(piv_full(inv, plim), cf.sl);
#pragma unroll
            for (int k = 0; k < NP; ++k) {
                const cx<T> xp = (r + 1 < R) ? stage_x(s, k)[(r + 1) * 32 + lane] : xnext[k];
                be[k][r] = piv_apply(ex_rhs(e, xm[k], x0[k], xp), inv, plim);
                xm[k] = x0[k];
                x0[k] = xp;
            }
        }
        // stage s is consumed: refill it now, so that issuing the copies
        // overlaps the recurrences below
        __syncwarp();
        if (lane == 0 && issued < nb && issued == t + S) issue(issued++);
#pragma unroll
        for (int r = 0; r < R; ++r) {
#pragma unroll
            for (int k = 0; k < NP; ++k) {
                y[k] = cmul(al[r], y[k]) + be[k][r];
                if (r < rows) col[k][(size_t)(jb + r) * nt] = y[k];
            }
        }
    }
    // y must reach the async proxy before the backward boxes read it back
    asm volatile("fence.proxy.async.global;" ::: "memory");
    __syncwarp();
    if (lane == 0)
        for (; issued < min(nb + S, ntask); ++issued) issue(issued);
    __syncwarp();

    // ---------------- backward sweep ----------------
    const DispPhase<T> ph = disp_phase<T>(p.disp, qq);
    cx<T> xn[NP];
#pragma unroll
    for (int k = 0; k < NP; ++k) xn[k] = czero<T>();
    for (int t = nb; t < ntask; ++t) {
        const int s = t % S;
        if (!mbar_wait(bar0 + 8 * s, (t / S) & 1)) { give_up(t); return; }
        const cx<T> *I = stage_i(s);
        const CnCoef<T> *Cf = stage_c(s);
        const int jb = R * block_of(t);
        const int rows = min(R, nr - jb);
        cx<T> ga[R], yv[NP][R];
#pragma unroll
        for (int r = 0; r < R; ++r) {
            ga[r] = cmul_i(piv_full(I[r * 34 + il], plim), Cf[r].sh);
#pragma unroll
            for (int k = 0; k < NP; ++k) yv[k][r] = stage_x(s, k)[r * 32 + lane];
        }
        __syncwarp();
        if (lane == 0 && issued < ntask && issued == t + S) issue(issued++);
#pragma unroll
        for (int r = R - 1; r >= 0; --r) {
#pragma unroll
            for (int k = 0; k < NP; ++k) {
                const cx<T> xv = cmul(ga[r], xn[k]) + yv[k][r];
                if (r < rows) {                        // rows past nr keep x = 0
                    xn[k] = xv;
                    col[k][(size_t)(jb + r) * nt] = disp_apply(xv, ph);
                }
            }
        }
    }
}

PFN_cuTensorMapEncodeTiled_v12000 encode_fn() {
    static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
    static std::once_flag once;
    std::call_once(once, [] {
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
    });
    return fn;
}

// 2-D map of 8-byte elements: `cols` per row (pitch `pitch` elements), `rows`
// rows, boxes of box_cols x box_rows.  Out-of-range elements read as zero.
bool make_map(CUtensorMap *m, const void *base, uint64_t cols, uint64_t pitch, uint64_t rows,
              uint32_t box_cols, uint32_t box_rows) {
    auto fn = encode_fn();
    if (!fn) return false;
    const cuuint64_t dims[2] = {cols, rows};
    const cuuint64_t strides[1] = {pitch * 8};
    const cuuint32_t box[2] = {box_cols, box_rows};
    const cuuint32_t estr[2] = {1, 1};
    return fn(m, CU_TENSOR_MAP_DATA_TYPE_UINT64, 2, const_cast<void *>(base), dims, strides, box, estr,
              CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
              CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

}  // namespace

// Whether the sequential kernel can run this column stage: Nt a multiple of
// 64 (32-column groups never straddle Nt/2), the row coefficients present,
// rows of the pivot table 16-byte aligned, every buffer 16-byte aligned.
template <typename T>
bool cn_seq_supported(const ColArgs<T> &a) {
    const uint64_t tpb = (uint64_t)a.tp * sizeof(cx<T>);
    return a.nt >= 64 && a.nt % 64 == 0 && a.coef && tpb % 16 == 0 &&
           ((uintptr_t)a.invden % 16) == 0 && ((uintptr_t)a.coef % 16) == 0 && a.nr >= 2;
}

template <typename T, int R, int S, int W, int NP>
cudaError_t launch_seq_shape(const ColArgs<T> &a, cx<T> *const *fields, int npulse, cudaStream_t st) {
    constexpr int E = int(sizeof(cx<T>)) / 8;
    using Ring = SeqRing<T, R, S, NP>;
    if (npulse % NP) return cudaErrorInvalidConfiguration;
    SeqParams<T> p;
    memset(&p, 0, sizeof(p));
    const int nq = a.nt / 2 + 1;
    if (!make_map(&p.tmap, a.invden, (uint64_t)E * nq, (uint64_t)E * a.tp, a.nr, 34 * E, R))
        return cudaErrorInvalidConfiguration;
    for (int k = 0; k < npulse; ++k) {
        if (((uintptr_t)fields[k] % 16) != 0) return cudaErrorInvalidConfiguration;
        if (!make_map(&p.fmap[k], fields[k], (uint64_t)E * a.nt, (uint64_t)E * a.nt, a.nr, 32 * E, R))
            return cudaErrorInvalidConfiguration;
        p.field[k] = fields[k];
    }
    p.coef = a.coef;
    p.nr = a.nr;
    p.nt = a.nt;
    p.ngroups = a.nt / 32;
    p.s64 = a.s64;
    p.dk64 = a.dk64;
    p.pivlim = a.pivlim;
    p.cc = a.cc;
    p.disp = a.disp;
    p.err = a.err;
    const size_t smem = (size_t)W * Ring::kBytes;
    static std::once_flag once;
    static cudaError_t attr = cudaSuccess;
    std::call_once(once, [&] {
        attr = cudaFuncSetAttribute(cn_seq_kernel<T, R, S, W, NP>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                    (int)smem);
    });
    if (attr != cudaSuccess) return attr;
    const int ctas = (p.ngroups + W - 1) / W;
    return launch_k(cn_seq_kernel<T, R, S, W, NP>, dim3(ctas, npulse / NP), dim3(32 * W), smem, st, p);
}

template <typename T>
cudaError_t launch_cn_seq(const ColArgs<T> &a, cx<T> *const *fields, int npulse, cudaStream_t st, int shape) {
    if (npulse < 1 || npulse > kSeqMaxPulses || !cn_seq_supported(a)) return cudaErrorInvalidConfiguration;
    // Two pulses per thread when their count is even (measured on 8 pulses
    // of 1024 x 4096: 172 us per launch against 230 us with one pulse per
    // thread and 190 us with four).  Each warp runs its columns' sweeps
    // with few other warps beside it (the rings take the shared memory), so
    // the ring shape trades rows in flight per warp against warps per SM;
    // the autotuner times the shapes (kSeqShapes):
    //   FP32: 0: 4 stages x 16 rows, 2 warps per CTA (4 warps per SM),
    //         1: 4 x 8 rows, 4 warps (8 per SM), 2: 4 x 4 rows, 4 warps (16 per SM);
    //   FP64: 0: 4 x 8 rows, 2 warps, 1: 4 x 4 rows, 4 warps, 2: 4 x 2 rows, 4 warps.
    // Odd pulse counts: one pulse per thread, 4 x 16 rows and 4 warps (FP32),
    // 4 x 8 rows and 2 warps (FP64).
    if (npulse % 2 == 0) {
        if constexpr (sizeof(T) == 4) {
            if (shape == 1) return launch_seq_shape<T, 8, 4, 4, 2>(a, fields, npulse, st);
            if (shape == 2) return launch_seq_shape<T, 4, 4, 4, 2>(a, fields, npulse, st);
            return launch_seq_shape<T, 16, 4, 2, 2>(a, fields, npulse, st);
        } else {
            if (shape == 1) return launch_seq_shape<T, 4, 4, 4, 2>(a, fields, npulse, st);
            if (shape == 2) return launch_seq_shape<T, 2, 4, 4, 2>(a, fields, npulse, st);
            return launch_seq_shape<T, 8, 4, 2, 2>(a, fields, npulse, st);
        }
    }
    if constexpr (sizeof(T) == 4) return launch_seq_shape<T, 16, 4, 4, 1>(a, fields, npulse, st);
    else return launch_seq_shape<T, 8, 4, 2, 1>(a, fields, npulse, st);
}

template bool cn_seq_supported<float>(const ColArgs<float> &);
template bool cn_seq_supported<double>(const ColArgs<double> &);
template cudaError_t launch_cn_seq<float>(const ColArgs<float> &, cx<float> *const *, int, cudaStream_t, int);
template cudaError_t launch_cn_seq<double>(const ColArgs<double> &, cx<double> *const *, int, cudaStream_t, int);

}  // namespace fcn
