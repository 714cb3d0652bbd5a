// mlp.cu -- the learned dz controller: a 6 -> 64 -> 64 -> 1 MLP (tanh hidden
// layers, linear output) whose output y corrects the step-doubling law: the
// proposal is log(dz / L_ref) = g + y with g = f4 - f5/3, the step that
// would have brought the last accepted attempt's error to rtol (Strang:
// local error O(dz^3)), so an untrained (zero) network reproduces the law
// without its safety factor and training learns how the safe step moves
// from one state to the next.  The network sees inputs that do not depend
// on the step sizes the controller happened to take (so data gathered under
// plain step doubling describes the learned controller's states too):
//   n = (f0, f1, f2, f3 s, g, fE s),   s = exp(-f5/3),
// f3 s and fE s being the changes of the peak intensity and of the energy
// over the last step scaled to a step of size exp(g) L_ref (both changes are
// proportional to the step).  Weights are used in BF16 (rounded from FP32
// master weights) with FP32 accumulation; training runs on the GPU with
// these kernels (the gradient's matrix products on the tensor cores, per-CTA
// partials reduced in a fixed order, then Adam).  Not in the paper, which
// uses a fixed dz; step doubling still judges every step.
//
// Parameter layout (floats): W1[64][6], b1[64], W2[64][64], b2[64], W3[64], b3.
//
// Features, all from the FP64 per-row statistics that the closing row
// launch of an attempt computes anyway (reduced by the controller kernel
// itself), so they cost no pass over the field of their own:
//   f0 = log(peak I / I_ref)          f1 = log10(peak rho / rho_nt + 1e-30) / 10
//   f2 = log(on-axis peak I / peak I) f3 = relative change of peak I over the last step
//   f4 = log(dz_prev / L_ref)         f5 = log(err_prev / rtol)
//   fE = relative change of the energy over the last step
// with I_ref taken from the field at the start of the run and
// L_ref = k0 (r_max/5)^2 / 2 (the Rayleigh length of a beam of waist r_max/5).
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <cstdint>
#include <mutex>

#include "fcn_device.cuh"

namespace fcn {
namespace {

constexpr int NIN = 6, NH = 64;
constexpr int O_W1 = 0, O_B1 = O_W1 + NH * NIN, O_W2 = O_B1 + NH, O_B2 = O_W2 + NH * NH,
              O_W3 = O_B2 + NH, O_B3 = O_W3 + NH, NP = O_B3 + 1;

__device__ __forceinline__ float bf16r(float x) { return __bfloat162float(__float2bfloat16_rn(x)); }

// Forward pass of one sample held in sx (6 floats); h1, h2 (64 each) in
// shared memory; returns y in thread 0 (all threads must call it).
__device__ __forceinline__ float forward_one(const float *sw, const float *sx, float *h1, float *h2,
                                             float *red) {
    const int u = threadIdx.x;
    if (u < NH) {
        float a = sw[O_B1 + u];
#pragma unroll
        for (int k = 0; k < NIN; ++k) a = fmaf(sw[O_W1 + u * NIN + k], sx[k], a);
        h1[u] = tanhf(a);
    }
    __syncthreads();
    if (u < NH) {
        float a = sw[O_B2 + u];
#pragma unroll 8
        for (int k = 0; k < NH; ++k) a = fmaf(sw[O_W2 + u * NH + k], h1[k], a);
        h2[u] = tanhf(a);
    }
    __syncthreads();
    if (u < 32) {
        float a = sw[O_W3 + u] * h2[u] + sw[O_W3 + u + 32] * h2[u + 32];
        for (int d = 16; d >= 1; d >>= 1) a += __shfl_down_sync(0xffffffffu, a, d);
        if (u == 0) red[0] = a + sw[O_B3];
    }
    __syncthreads();
    return red[0];
}

// ---- Gradient on the tensor cores ------------------------------------------
// The same MSE gradient with every matrix product of the forward and the
// backward pass on mma.sync m16n8k16 (BF16 operands, FP32 accumulation): one
// warp takes 16 samples at a time,
//   Z1 = Xa W1a^T  (Xa = [x, 1, 0...]: 16 inputs, b1 folded in as a column)
//   Z2 = H1 W2^T + b2,   G1 = (G2 W2) (1 - H1^2),
//   dW2 += G2^T H1,      dW1a += G1^T Xa,
// and the output layer, G2 = dy w3 (1 - H2^2), dw3, db2, db3 in FP32.  The
// weights are BF16 already (the network's definition), so they enter the
// products exactly; an FP32 activation a enters as three BF16 parts hi + mid
// + lo (each the BF16 rounding of what the earlier parts leave, a - hi and
// then a - hi - mid being exact in FP32), which carry its 24 bits: a product
// weight x activation is three MMAs, activation x activation six (the part
// products above 2^-24 relative).  So the result equals the scalar FP32
// evaluation up to FP32 rounding.  Fragment layouts are those of the PTX ISA
// for m16n8k16: g = lane / 4, t2 = 2 (lane % 4); A rows g, g + 8, columns
// t2, t2 + 1 (+ 8); B rows (k) t2, t2 + 1 (+ 8), column g; C rows g, g + 8,
// columns t2, t2 + 1.
constexpr int TW = 4;              // warps per CTA
constexpr int TS = 68;             // row stride (floats) of the per-warp activation tiles
constexpr int TX = 20;             // row stride of the per-warp input tile
constexpr int KA = 16;             // layer-1 inputs: f (NIN), 1, zero padding
constexpr int TC_WARP_FLOATS = 16 * TX + 3 * 16 * TS + 64 * 64 + 64 * KA;
// b2, w3 (+ pad), the warps' column sums [TW][2][64] and scalars [TW][2] (+ pad)
constexpr int TC_SHARED_FLOATS = 64 + 68 + TW * 2 * 64 + 16;
constexpr size_t TC_SMEM = sizeof(__nv_bfloat16) * (64 * KA + 2 * 64 * 64) +
                           sizeof(float) * (TC_SHARED_FLOATS + (size_t)TW * TC_WARP_FLOATS);

struct Split3 {
    uint32_t h, m, l;
};
__device__ __forceinline__ uint32_t pack_bf(__nv_bfloat16 lo, __nv_bfloat16 hi) {
    return (uint32_t)__bfloat16_as_ushort(lo) | ((uint32_t)__bfloat16_as_ushort(hi) << 16);
}
// Two FP32 values (lower index first) as three packed BF16 pairs.
__device__ __forceinline__ Split3 split_pair(float a, float b) {
    const __nv_bfloat16 ah = __float2bfloat16_rn(a), bh = __float2bfloat16_rn(b);
    const float ar = a - __bfloat162float(ah), br = b - __bfloat162float(bh);
    const __nv_bfloat16 am = __float2bfloat16_rn(ar), bm = __float2bfloat16_rn(br);
    const float ar2 = ar - __bfloat162float(am), br2 = br - __bfloat162float(bm);
    return {pack_bf(ah, bh), pack_bf(am, bm), pack_bf(__float2bfloat16_rn(ar2), __float2bfloat16_rn(br2))};
}
__device__ __forceinline__ void mma_bf16(float (&d)[4], const uint32_t (&a)[4], uint32_t b0, uint32_t b1) {
    asm volatile(
        "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
        "{%0,%1,%2,%3};"
        : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
        : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}
// A operand (16 x 16) of an FP32 matrix read as at(row, col), in three parts.
template <class F>
__device__ __forceinline__ void load_a3(F at, uint32_t (&ah)[4], uint32_t (&am)[4], uint32_t (&al)[4]) {
    const int lane = threadIdx.x & 31, g = lane >> 2, t2 = (lane & 3) * 2;
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        const int r = g + 8 * (q & 1), c = t2 + 8 * (q >> 1);
        const Split3 v = split_pair(at(r, c), at(r, c + 1));
        ah[q] = v.h;
        am[q] = v.m;
        al[q] = v.l;
    }
}
// B operand (16 x 8) of an FP32 matrix read as at(k, n), in three parts.
template <class F>
__device__ __forceinline__ void load_b3(F at, uint32_t (&bh)[2], uint32_t (&bm)[2], uint32_t (&bl)[2]) {
    const int lane = threadIdx.x & 31, g = lane >> 2, t2 = (lane & 3) * 2;
#pragma unroll
    for (int q = 0; q < 2; ++q) {
        const Split3 v = split_pair(at(t2 + 8 * q, g), at(t2 + 8 * q + 1, g));
        bh[q] = v.h;
        bm[q] = v.m;
        bl[q] = v.l;
    }
}
// B operand (16 x 8) with B[k][n] = M[n0 + n][k0 + k] of a row-major BF16
// matrix M (row stride ld): two consecutive k of one row per register.
__device__ __forceinline__ void load_bw(const __nv_bfloat16 *M, int ld, int n0, int k0, uint32_t &b0,
                                        uint32_t &b1) {
    const int lane = threadIdx.x & 31, g = lane >> 2, t2 = (lane & 3) * 2;
    const __nv_bfloat16 *p = M + (size_t)(n0 + g) * ld + k0 + t2;
    b0 = *reinterpret_cast<const uint32_t *>(p);
    b1 = *reinterpret_cast<const uint32_t *>(p + 8);
}
// D += A x B for an FP32 activation A (three parts) and a BF16 weight B.
__device__ __forceinline__ void mma3(float (&d)[4], const uint32_t (&ah)[4], const uint32_t (&am)[4],
                                     const uint32_t (&al)[4], uint32_t b0, uint32_t b1) {
    mma_bf16(d, al, b0, b1);
    mma_bf16(d, am, b0, b1);
    mma_bf16(d, ah, b0, b1);
}
// D += A x B for two FP32 activations (the six part products above 2^-24).
__device__ __forceinline__ void mma6(float (&d)[4], const uint32_t (&ah)[4], const uint32_t (&am)[4],
                                     const uint32_t (&al)[4], const uint32_t (&bh)[2], const uint32_t (&bm)[2],
                                     const uint32_t (&bl)[2]) {
    mma_bf16(d, al, bh[0], bh[1]);
    mma_bf16(d, ah, bl[0], bl[1]);
    mma_bf16(d, am, bm[0], bm[1]);
    mma_bf16(d, am, bh[0], bh[1]);
    mma_bf16(d, ah, bm[0], bm[1]);
    mma_bf16(d, ah, bh[0], bh[1]);
}

// Partial gradient of CTA c over samples [c per, min(n, (c + 1) per)) of the
// permutation idx, written to partial[c][0..NP) in the parameter layout and
// the sum of squared residuals to partial[c][NP].  Tiles of 16 samples go to
// the warps round robin; each warp sums its tiles in order, then the warps
// are summed in order (deterministic).
__global__ void __launch_bounds__(32 * TW)
mlp_grad_tc(const float *__restrict__ W, const float *__restrict__ X, const float *__restrict__ Y,
            const int *__restrict__ idx, int n, int per, float inv_batch, float *partial) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __nv_bfloat16 *w1a = reinterpret_cast<__nv_bfloat16 *>(smem_raw);   // [64][KA]
    __nv_bfloat16 *w2 = w1a + 64 * KA;                                   // [64][64]: W2[u][k]
    __nv_bfloat16 *w2t = w2 + 64 * 64;                                   // [64][64]: W2[u][k] at [k][u]
    float *b2 = reinterpret_cast<float *>(w2t + 64 * 64);
    float *w3 = b2 + 64;
    float *vec = w3 + 64 + 4;          // [TW][2][64] column sums of the warps (dw3, db2)
    float *wbase = b2 + TC_SHARED_FLOATS;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int g = lane >> 2, t2 = (lane & 3) * 2;
    float *xa = wbase + (size_t)warp * TC_WARP_FLOATS;   // [16][TX]
    float *h1 = xa + 16 * TX;                            // [16][TS]
    float *g2 = h1 + 16 * TS;                            // [16][TS]
    float *g1 = g2 + 16 * TS;                            // [16][TS]
    float *aw2 = g1 + 16 * TS;                           // dW2, fragment order [4][8][32][4]
    float *aw1 = aw2 + 64 * 64;                          // dW1a, fragment order [4][2][32][4]

    for (int p = threadIdx.x; p < 64 * KA; p += blockDim.x) {
        const int u = p / KA, i = p % KA;
        const float v = i < NIN ? W[O_W1 + u * NIN + i] : (i == NIN ? W[O_B1 + u] : 0.f);
        w1a[p] = __float2bfloat16_rn(v);
    }
    for (int p = threadIdx.x; p < 64 * 64; p += blockDim.x) {
        const __nv_bfloat16 v = __float2bfloat16_rn(W[O_W2 + p]);
        w2[p] = v;
        w2t[(p % 64) * 64 + p / 64] = v;
    }
    for (int p = threadIdx.x; p < 64; p += blockDim.x) {
        b2[p] = bf16r(W[O_B2 + p]);
        w3[p] = bf16r(W[O_W3 + p]);
    }
    const float b3 = bf16r(W[O_B3]);
    for (int p = lane; p < 64 * 64; p += 32) aw2[p] = 0.f;
    for (int p = lane; p < 64 * KA; p += 32) aw1[p] = 0.f;
    __syncthreads();

    float dw3[8][2], db2[8][2], db3 = 0.f, loss = 0.f;
#pragma unroll
    for (int nt = 0; nt < 8; ++nt) dw3[nt][0] = dw3[nt][1] = db2[nt][0] = db2[nt][1] = 0.f;

    const int s0 = blockIdx.x * per, s1 = min(n, s0 + per);
    for (int sb = s0 + 16 * warp; sb < s1; sb += 16 * TW) {
        // inputs of the tile (rows past s1 are zero and get dy = 0)
        for (int e = lane; e < 16 * KA; e += 32) {
            const int r = e / KA, i = e % KA, s = sb + r;
            float v = 0.f;
            if (s < s1) v = i < NIN ? X[(size_t)idx[s] * NIN + i] : (i == NIN ? 1.f : 0.f);
            xa[r * TX + i] = v;
        }
        __syncwarp();
        uint32_t ah[4], am[4], al[4];
        // layer 1: H1 = tanh(Xa W1a^T)
        load_a3([&](int r, int c) { return xa[r * TX + c]; }, ah, am, al);
#pragma unroll
        for (int nt = 0; nt < 8; ++nt) {
            float d[4] = {0.f, 0.f, 0.f, 0.f};
            uint32_t b0, b1;
            load_bw(w1a, KA, 8 * nt, 0, b0, b1);
            mma3(d, ah, am, al, b0, b1);
#pragma unroll
            for (int q = 0; q < 4; ++q) h1[(g + 8 * (q >> 1)) * TS + 8 * nt + t2 + (q & 1)] = tanhf(d[q]);
        }
        __syncwarp();
        // layer 2: H2 = tanh(H1 W2^T + b2), kept in the C fragments
        float h2[8][4];
#pragma unroll
        for (int nt = 0; nt < 8; ++nt) h2[nt][0] = h2[nt][1] = h2[nt][2] = h2[nt][3] = 0.f;
#pragma unroll
        for (int kk = 0; kk < 4; ++kk) {
            load_a3([&](int r, int c) { return h1[r * TS + 16 * kk + c]; }, ah, am, al);
#pragma unroll
            for (int nt = 0; nt < 8; ++nt) {
                uint32_t b0, b1;
                load_bw(w2, 64, 8 * nt, 16 * kk, b0, b1);
                mma3(h2[nt], ah, am, al, b0, b1);
            }
        }
        float p0 = 0.f, p1 = 0.f;      // rows g and g + 8: sum of h2 w3 over this lane's columns
#pragma unroll
        for (int nt = 0; nt < 8; ++nt)
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                const int c = 8 * nt + t2 + (q & 1);
                h2[nt][q] = tanhf(h2[nt][q] + b2[c]);
                if (q < 2) p0 = fmaf(h2[nt][q], w3[c], p0);
                else p1 = fmaf(h2[nt][q], w3[c], p1);
            }
        p0 += __shfl_xor_sync(0xffffffffu, p0, 1);
        p0 += __shfl_xor_sync(0xffffffffu, p0, 2);
        p1 += __shfl_xor_sync(0xffffffffu, p1, 1);
        p1 += __shfl_xor_sync(0xffffffffu, p1, 2);
        float dy[2];
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            const int s = sb + g + 8 * h;
            dy[h] = 0.f;
            if (s < s1) {
                const float r = (h ? p1 : p0) + b3 - Y[idx[s]];
                dy[h] = 2.f * r * inv_batch;
                if ((lane & 3) == 0) {
                    loss = fmaf(r, r, loss);
                    db3 += dy[h];
                }
            }
        }
        // output layer's gradients; G2 = dy w3 (1 - H2^2)
#pragma unroll
        for (int nt = 0; nt < 8; ++nt)
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                const int c = 8 * nt + t2 + (q & 1);
                const float d = dy[q >> 1];
                const float gv = d * w3[c] * (1.f - h2[nt][q] * h2[nt][q]);
                dw3[nt][q & 1] = fmaf(d, h2[nt][q], dw3[nt][q & 1]);
                db2[nt][q & 1] += gv;
                g2[(g + 8 * (q >> 1)) * TS + c] = gv;
            }
        __syncwarp();
        // G1 = (G2 W2) (1 - H1^2)
        {
            float z[8][4];
#pragma unroll
            for (int nt = 0; nt < 8; ++nt) z[nt][0] = z[nt][1] = z[nt][2] = z[nt][3] = 0.f;
#pragma unroll
            for (int kk = 0; kk < 4; ++kk) {
                load_a3([&](int r, int c) { return g2[r * TS + 16 * kk + c]; }, ah, am, al);
#pragma unroll
                for (int nt = 0; nt < 8; ++nt) {
                    uint32_t b0, b1;
                    load_bw(w2t, 64, 8 * nt, 16 * kk, b0, b1);
                    mma3(z[nt], ah, am, al, b0, b1);
                }
            }
#pragma unroll
            for (int nt = 0; nt < 8; ++nt)
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    const int o = (g + 8 * (q >> 1)) * TS + 8 * nt + t2 + (q & 1);
                    g1[o] = z[nt][q] * (1.f - h1[o] * h1[o]);
                }
        }
        __syncwarp();
        // dW2 += G2^T H1 (rows: units u; columns: inputs k; K: the 16 samples)
#pragma unroll 1
        for (int mt = 0; mt < 4; ++mt) {
            load_a3([&](int r, int c) { return g2[c * TS + 16 * mt + r]; }, ah, am, al);
#pragma unroll
            for (int nt = 0; nt < 8; ++nt) {
                uint32_t bh[2], bm[2], bl[2];
                load_b3([&](int k, int nn) { return h1[k * TS + 8 * nt + nn]; }, bh, bm, bl);
                float4 *acc = reinterpret_cast<float4 *>(aw2) + (mt * 8 + nt) * 32 + lane;
                const float4 a4 = *acc;
                float d[4] = {a4.x, a4.y, a4.z, a4.w};
                mma6(d, ah, am, al, bh, bm, bl);
                *acc = make_float4(d[0], d[1], d[2], d[3]);
            }
        }
        // dW1a += G1^T Xa
#pragma unroll 1
        for (int mt = 0; mt < 4; ++mt) {
            load_a3([&](int r, int c) { return g1[c * TS + 16 * mt + r]; }, ah, am, al);
#pragma unroll
            for (int nt = 0; nt < 2; ++nt) {
                uint32_t bh[2], bm[2], bl[2];
                load_b3([&](int k, int nn) { return xa[k * TX + 8 * nt + nn]; }, bh, bm, bl);
                float4 *acc = reinterpret_cast<float4 *>(aw1) + (mt * 2 + nt) * 32 + lane;
                const float4 a4 = *acc;
                float d[4] = {a4.x, a4.y, a4.z, a4.w};
                mma6(d, ah, am, al, bh, bm, bl);
                *acc = make_float4(d[0], d[1], d[2], d[3]);
            }
        }
        __syncwarp();
    }

    // column sums of the output layer's gradients over the rows (lanes that
    // share lane % 4), then over the warps in order
#pragma unroll
    for (int nt = 0; nt < 8; ++nt)
#pragma unroll
        for (int c = 0; c < 2; ++c)
#pragma unroll
            for (int m = 4; m <= 16; m <<= 1) {
                dw3[nt][c] += __shfl_xor_sync(0xffffffffu, dw3[nt][c], m);
                db2[nt][c] += __shfl_xor_sync(0xffffffffu, db2[nt][c], m);
            }
    if (g == 0) {
#pragma unroll
        for (int nt = 0; nt < 8; ++nt)
#pragma unroll
            for (int c = 0; c < 2; ++c) {
                vec[(warp * 2 + 0) * 64 + 8 * nt + t2 + c] = dw3[nt][c];
                vec[(warp * 2 + 1) * 64 + 8 * nt + t2 + c] = db2[nt][c];
            }
    }
    for (int m = 16; m >= 1; m >>= 1) {
        db3 += __shfl_xor_sync(0xffffffffu, db3, m);
        loss += __shfl_xor_sync(0xffffffffu, loss, m);
    }
    float *red = vec + TW * 2 * 64;    // [TW][2]
    if (lane == 0) {
        red[warp * 2] = db3;
        red[warp * 2 + 1] = loss;
    }
    __syncthreads();
    float *out = partial + (size_t)blockIdx.x * (NP + 1);
    // fragment element e = ((mt * NT + nt) * 32 + lane) * 4 + q holds row
    // u = 16 mt + lane / 4 + 8 (q / 2), column 8 nt + 2 (lane % 4) + q % 2
    for (int e = threadIdx.x; e < 64 * 64; e += blockDim.x) {
        float sum = 0.f;
        for (int w = 0; w < TW; ++w) sum += (wbase + (size_t)w * TC_WARP_FLOATS + 16 * TX + 3 * 16 * TS)[e];
        const int q = e & 3, ln = (e >> 2) & 31, tile = e >> 7;
        const int u = 16 * (tile >> 3) + (ln >> 2) + 8 * (q >> 1), k = 8 * (tile & 7) + 2 * (ln & 3) + (q & 1);
        out[O_W2 + u * 64 + k] = sum;
    }
    for (int e = threadIdx.x; e < 64 * KA; e += blockDim.x) {
        float sum = 0.f;
        for (int w = 0; w < TW; ++w)
            sum += (wbase + (size_t)w * TC_WARP_FLOATS + 16 * TX + 3 * 16 * TS + 64 * 64)[e];
        const int q = e & 3, ln = (e >> 2) & 31, tile = e >> 7;
        const int u = 16 * (tile >> 1) + (ln >> 2) + 8 * (q >> 1), i = 8 * (tile & 1) + 2 * (ln & 3) + (q & 1);
        if (i < NIN) out[O_W1 + u * NIN + i] = sum;
        else if (i == NIN) out[O_B1 + u] = sum;
    }
    for (int c = threadIdx.x; c < 64; c += blockDim.x) {
        float a = 0.f, b = 0.f;
        for (int w = 0; w < TW; ++w) {
            a += vec[(w * 2) * 64 + c];
            b += vec[(w * 2 + 1) * 64 + c];
        }
        out[O_W3 + c] = a;
        out[O_B2 + c] = b;
    }
    if (threadIdx.x == 0) {
        float a = 0.f, b = 0.f;
        for (int w = 0; w < TW; ++w) {
            a += red[w * 2];
            b += red[w * 2 + 1];
        }
        out[O_B3] = a;
        out[NP] = b;
    }
}

// grad[p] = sum over CTAs in order; loss = sum of squared residuals * inv_batch.
__global__ void mlp_grad_reduce(const float *__restrict__ partial, int ncta, float inv_batch,
                                float *grad, float *loss) {
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p > NP) return;
    float s = 0.f;
    for (int c = 0; c < ncta; ++c) s += partial[(size_t)c * (NP + 1) + p];
    if (p < NP) grad[p] = s;
    else *loss = s * inv_batch;
}

// Adam (Kingma & Ba) on the FP32 master weights; t is the 1-based step.
__global__ void mlp_adam(float *W, float *m, float *v, const float *__restrict__ g, float lr, float b1,
                         float b2, float eps, int t) {
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= NP) return;
    const float gp = g[p];
    const float mp = b1 * m[p] + (1.f - b1) * gp;
    const float vp = b2 * v[p] + (1.f - b2) * gp * gp;
    m[p] = mp;
    v[p] = vp;
    const float mh = mp / (1.f - powf(b1, (float)t));
    const float vh = vp / (1.f - powf(b2, (float)t));
    W[p] -= lr * mh / (sqrtf(vh) + eps);
}

// The controller's work after an attempt, in one launch of CT threads with
// one contiguous output (one copy to the host): the step-doubling norm from
// the per-row sums a row launch with OP_DIFF leaves (summed as
// launch_diff_final sums them), the
// reduction of the per-row statistics (as launch_reduce_stats: the same
// tree, so the same energy), the features, and with W non-null the MLP's
// proposal dz = L_ref exp(f4 - f5/3 + y), clamped to [dz_lo, dz_hi].  With
// the norm, err_prev is taken from it.
// out[0..1] = norm (0 without diff_rows); out[2..5] = the 8 feature floats
// (f0..f5, fE, peak); out[6] = proposal (0 without W); out[7] = energy sum.
constexpr int CT = 256;
__device__ __forceinline__ void step_control(const double *__restrict__ st, int nr, const double *__restrict__ diff_rows,
                                             MlpScalars sc, const float *__restrict__ W, double *out) {
    __shared__ float sw[NP];
    __shared__ float sx[NIN], h1[NH], h2[NH], r[2];
    __shared__ double sh[32];
    const int tid = threadIdx.x;
    // the weights first: their loads overlap the reductions
    if (W) {
        const float4 *W4 = reinterpret_cast<const float4 *>(W);
        for (int p = tid; p < NP / 4; p += CT) {
            const float4 v = W4[p];
            sw[4 * p] = bf16r(v.x);
            sw[4 * p + 1] = bf16r(v.y);
            sw[4 * p + 2] = bf16r(v.z);
            sw[4 * p + 3] = bf16r(v.w);
        }
        for (int p = (NP / 4) * 4 + tid; p < NP; p += CT) sw[p] = bf16r(W[p]);
    }
    double d2 = 0.0, b2 = 0.0;
    if (diff_rows)
        for (int m = tid; m < nr; m += CT) {
            d2 += diff_rows[2 * m];
            b2 += diff_rows[2 * m + 1];
        }
    double e = 0.0, mi = 0.0, mu = 0.0;
    for (int m = tid; m < nr; m += CT) {
        const double *row = st + (size_t)m * NSTAT;
        e += radial_weight(m) * row[ST_SUM_I];
        mi = fmax(mi, row[ST_MAX_I]);
        mu = fmax(mu, row[ST_MAX_U]);
    }
    d2 = block_sum(d2, sh);
    b2 = block_sum(b2, sh);
    e = block_sum(e, sh);
    mi = block_max(mi, sh);
    mu = block_max(mu, sh);
    if (tid == 0) {
        out[0] = d2;
        out[1] = b2;
        if (diff_rows) sc.err_prev = b2 > 0 ? sqrt(d2 / b2) : sqrt(d2);
        const double peak = mi;
        const double f[NIN] = {
            log(fmax(peak, 1e-300) / sc.i_ref),
            log10(mu + 1e-30) / 10.0,
            log(fmax(st[ST_MAX_I], 1e-300) / fmax(peak, 1e-300)),
            sc.peak_prev > 0 ? (peak - sc.peak_prev) / sc.peak_prev : 0.0,
            log(sc.dz_prev / sc.l_ref),
            log(fmax(sc.err_prev, 1e-30) / sc.rtol),
        };
        const double fe = sc.e_prev > 0 ? (e - sc.e_prev) / sc.e_prev : 0.0;
        float *fo = reinterpret_cast<float *>(out + 2);
        for (int k = 0; k < NIN; ++k) fo[k] = (float)f[k];
        fo[NIN] = (float)fe;
        fo[NIN + 1] = (float)peak;
        out[6] = 0.0;
        out[7] = e;
        const double sstep = exp(-f[5] / 3.0);
        sx[0] = (float)f[0];
        sx[1] = (float)f[1];
        sx[2] = (float)f[2];
        sx[3] = (float)(f[3] * sstep);
        sx[4] = (float)(f[4] - f[5] / 3.0);
        sx[5] = (float)(fe * sstep);
    }
    __syncthreads();
    if (!W) return;
    const float y = forward_one(sw, sx, h1, h2, r);
    if (tid == 0) {
        double dz = sc.l_ref * exp((double)sx[4] + (double)y);
        out[6] = fmin(fmax(dz, sc.dz_lo), sc.dz_hi);
    }
}

__global__ void __launch_bounds__(CT)
mlp_step_control(const double *__restrict__ st, int nr, const double *__restrict__ diff_rows, MlpScalars sc,
                 const float *__restrict__ W, double *out) {
    step_control(st, nr, diff_rows, sc, W, out);
}

// The same for the pulses of an adaptive batch on one grid, a CTA per pulse.
__global__ void __launch_bounds__(CT) mlp_step_control_multi(const __grid_constant__ CtlMulti p, const float *W) {
    const int b = blockIdx.x;
    step_control(p.stats[b], p.nr, p.rows[b], p.sc[b], W, p.out + 8 * b);
}

}  // namespace

int mlp_nparam() { return NP; }

cudaError_t launch_mlp_step_control(const double *stats, int nr, const double *diff_rows, const MlpScalars &sc,
                                    const float *W, double *out, cudaStream_t st) {
    mlp_step_control<<<1, CT, 0, st>>>(stats, nr, diff_rows, sc, W, out);
    return cudaGetLastError();
}

cudaError_t launch_mlp_step_control_multi(const CtlMulti &p, const float *W, cudaStream_t st) {
    if (p.n < 1 || p.n > kCtlMulti) return cudaErrorInvalidValue;
    mlp_step_control_multi<<<p.n, CT, 0, st>>>(p, W);
    return cudaGetLastError();
}

cudaError_t launch_mlp_grad(const float *W, const float *X, const float *Y, const int *idx, int n,
                            float *partial, int max_cta, float *grad, float *loss, cudaStream_t st) {
    static_assert(TC_SMEM <= 227 * 1024, "shared memory of the gradient CTA");
    static std::once_flag once;
    static cudaError_t attr = cudaSuccess;
    std::call_once(once, [] {
        attr = cudaFuncSetAttribute(mlp_grad_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)TC_SMEM);
    });
    if (attr != cudaSuccess) return attr;
    const int per_min = 16 * TW;                  // one tile per warp
    int ncta = (n + per_min - 1) / per_min;
    if (ncta > max_cta) ncta = max_cta;
    const int per = (n + ncta - 1) / ncta;
    const float inv_batch = 1.f / (float)n;
    mlp_grad_tc<<<ncta, 32 * TW, TC_SMEM, st>>>(W, X, Y, idx, n, per, inv_batch, partial);
    mlp_grad_reduce<<<(NP + 1 + 255) / 256, 256, 0, st>>>(partial, ncta, inv_batch, grad, loss);
    return cudaGetLastError();
}

cudaError_t launch_mlp_adam(float *W, float *m, float *v, const float *g, float lr, int t, cudaStream_t st) {
    mlp_adam<<<(NP + 255) / 256, 256, 0, st>>>(W, m, v, g, lr, 0.9f, 0.999f, 1e-8f, t);
    return cudaGetLastError();
}

}  // namespace fcn
