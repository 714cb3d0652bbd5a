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
// these kernels (per-CTA gradient partials reduced in a fixed order, then
// Adam).  Not in the paper, which uses a fixed dz; step doubling still
// judges every step.
//
// Parameter layout (floats): W1[64][6], b1[64], W2[64][64], b2[64], W3[64], b3.
//
// Features, all from the FP64 statistics that the closing row launch of an
// attempt computes anyway (launch_reduce_stats), so they cost no pass of
// their own:
//   f0 = log(peak I / I_ref)          f1 = log10(peak rho / rho_nt + 1e-30) / 10
//   f2 = log(on-axis peak I / peak I) f3 = relative change of peak I over the last step
//   f4 = log(dz_prev / L_ref)         f5 = log(err_prev / rtol)
//   fE = relative change of the energy over the last step
// with I_ref taken from the field at the start of the run and
// L_ref = k0 (r_max/5)^2 / 2 (the Rayleigh length of a beam of waist r_max/5).
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include "fcn_device.cuh"

namespace fcn {
namespace {

constexpr int NIN = 6, NH = 64;
constexpr int O_W1 = 0, O_B1 = O_W1 + NH * NIN, O_W2 = O_B1 + NH, O_B2 = O_W2 + NH * NH,
              O_W3 = O_B2 + NH, O_B3 = O_W3 + NH, NP = O_B3 + 1;
constexpr int GT = 256;   // threads of the gradient CTAs

__device__ __forceinline__ float bf16r(float x) { return __bfloat162float(__float2bfloat16_rn(x)); }

// Loads the BF16-rounded weights into shared memory.
__device__ __forceinline__ void load_weights(const float *__restrict__ W, float *sw) {
    for (int p = threadIdx.x; p < NP; p += blockDim.x) sw[p] = bf16r(W[p]);
    __syncthreads();
}

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

// Partial MSE gradient over samples [c*per, min(n, (c+1)*per)) of the
// permutation idx; every thread owns the parameters p = t, t+GT, ... and
// accumulates their gradient over the samples in order (deterministic).
__global__ void __launch_bounds__(GT)
mlp_grad_partial(const float *__restrict__ W, const float *__restrict__ X, const float *__restrict__ Y,
                 const int *__restrict__ idx, int n, int per, float inv_batch, float *partial) {
    __shared__ float sw[NP];
    __shared__ float sx[NIN], h1[NH], h2[NH], g1[NH], g2[NH], red[2];
    load_weights(W, sw);
    constexpr int OWN = (NP + GT - 1) / GT;
    float acc[OWN];
#pragma unroll
    for (int i = 0; i < OWN; ++i) acc[i] = 0.f;
    float loss = 0.f;
    const int s0 = blockIdx.x * per, s1 = min(n, s0 + per);
    for (int s = s0; s < s1; ++s) {
        const int j = idx[s];
        if (threadIdx.x < NIN) sx[threadIdx.x] = X[(size_t)j * NIN + threadIdx.x];
        __syncthreads();
        const float y = forward_one(sw, sx, h1, h2, red);
        const float r = y - Y[j];
        const float dy = 2.f * r * inv_batch;       // d(mean squared error)/dy
        loss += r * r;
        const int u = threadIdx.x;
        if (u < NH) g2[u] = dy * sw[O_W3 + u] * (1.f - h2[u] * h2[u]);
        __syncthreads();
        if (u < NH) {
            float a = 0.f;
#pragma unroll 8
            for (int k = 0; k < NH; ++k) a = fmaf(sw[O_W2 + k * NH + u], g2[k], a);
            g1[u] = a * (1.f - h1[u] * h1[u]);
        }
        __syncthreads();
#pragma unroll
        for (int i = 0; i < OWN; ++i) {
            const int p = threadIdx.x + i * GT;
            if (p >= NP) break;
            float g;
            if (p < O_B1) g = g1[p / NIN] * sx[p % NIN];
            else if (p < O_W2) g = g1[p - O_B1];
            else if (p < O_B2) g = g2[(p - O_W2) / NH] * h1[(p - O_W2) % NH];
            else if (p < O_W3) g = g2[p - O_B2];
            else if (p < O_B3) g = dy * h2[p - O_W3];
            else g = dy;
            acc[i] += g;
        }
        __syncthreads();
    }
    float *out = partial + (size_t)blockIdx.x * (NP + 1);
#pragma unroll
    for (int i = 0; i < OWN; ++i) {
        const int p = threadIdx.x + i * GT;
        if (p < NP) out[p] = acc[i];
    }
    if (threadIdx.x == 0) out[NP] = loss;
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

// Features of the current field from the diagnostic reduction `red` (see
// launch_reduce_stats) and the controller's scalars; with W non-null also
// the MLP's proposal dz = L_ref exp(f4 - f5/3 + y), clamped to [lo, hi].
__global__ void mlp_propose(const double *__restrict__ red, MlpScalars sc, const float *__restrict__ W,
                            float *features, double *dz_out, const double *__restrict__ norm) {
    __shared__ float sw[NP];
    __shared__ float sx[NIN], h1[NH], h2[NH], r[2];
    if (threadIdx.x == 0) {
        if (norm) sc.err_prev = norm[1] > 0 ? sqrt(norm[0] / norm[1]) : sqrt(norm[0]);
        const double peak = red[1];
        const double f[NIN] = {
            log(fmax(peak, 1e-300) / sc.i_ref),
            log10(red[2] + 1e-30) / 10.0,
            log(fmax(red[3], 1e-300) / fmax(peak, 1e-300)),
            sc.peak_prev > 0 ? (peak - sc.peak_prev) / sc.peak_prev : 0.0,
            log(sc.dz_prev / sc.l_ref),
            log(fmax(sc.err_prev, 1e-30) / sc.rtol),
        };
        const double fe = sc.e_prev > 0 ? (red[0] - sc.e_prev) / sc.e_prev : 0.0;
        for (int k = 0; k < NIN; ++k) features[k] = (float)f[k];
        features[NIN] = (float)fe;
        features[NIN + 1] = (float)peak;
        const double g = f[4] - f[5] / 3.0;
        const double sstep = exp(-f[5] / 3.0);
        sx[0] = (float)f[0];
        sx[1] = (float)f[1];
        sx[2] = (float)f[2];
        sx[3] = (float)(f[3] * sstep);
        sx[4] = (float)g;
        sx[5] = (float)(fe * sstep);
    }
    __syncthreads();
    if (!W) return;
    load_weights(W, sw);
    const float y = forward_one(sw, sx, h1, h2, r);
    if (threadIdx.x == 0) {
        double dz = sc.l_ref * exp((double)sx[4] + (double)y);
        dz = fmin(fmax(dz, sc.dz_lo), sc.dz_hi);
        *dz_out = dz;
    }
}

}  // namespace

int mlp_nparam() { return NP; }

cudaError_t launch_mlp_grad(const float *W, const float *X, const float *Y, const int *idx, int n,
                            float *partial, int max_cta, float *grad, float *loss, cudaStream_t st) {
    const int per = 32;
    int ncta = (n + per - 1) / per;
    if (ncta > max_cta) ncta = max_cta;
    const int per_cta = (n + ncta - 1) / ncta;
    const float inv_batch = 1.f / (float)n;
    mlp_grad_partial<<<ncta, GT, 0, st>>>(W, X, Y, idx, n, per_cta, inv_batch, partial);
    mlp_grad_reduce<<<(NP + 1 + 255) / 256, 256, 0, st>>>(partial, ncta, inv_batch, grad, loss);
    return cudaGetLastError();
}

cudaError_t launch_mlp_adam(float *W, float *m, float *v, const float *g, float lr, int t, cudaStream_t st) {
    mlp_adam<<<(NP + 255) / 256, 256, 0, st>>>(W, m, v, g, lr, 0.9f, 0.999f, 1e-8f, t);
    return cudaGetLastError();
}

cudaError_t launch_mlp_propose(const double *red, const MlpScalars &sc, const float *W, float *features,
                               double *dz_out, cudaStream_t st, const double *norm) {
    mlp_propose<<<1, NH, 0, st>>>(red, sc, W, features, dz_out, norm);
    return cudaGetLastError();
}

}  // namespace fcn
