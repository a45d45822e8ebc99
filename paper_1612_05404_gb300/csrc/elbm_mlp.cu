// elbm_mlp.cu -- training and inference of the learned alpha proposal:
// features, FP32 forward / analytic backward / Adam (training, master
// weights) and BF16 tensor-core forward (inference). The network and its
// parameter layout are described in elbm_mlp.cuh.
#include <cuda_runtime.h>

#include "elbm.h"
#include "elbm_device.cuh"
#include "elbm_mlp.cuh"

namespace elbm {
namespace {

constexpr int TB = 128;       // samples per training block
constexpr int TBP = TB + 1;   // padded stride of the per-sample activation rows
constexpr int NPART = MLP_NPARAM + 1;  // gradient + loss per block partial

struct TrainSmem {
    float th[MLP_NPARAM];
    float x[MLP_NIN * TBP];
    float z1[MLP_NH * TBP];   // z1, then dL/dz1
    float h1[MLP_NH * TBP];
    float z2[MLP_NH * TBP];   // z2, then dL/dz2
    float h2[MLP_NH * TBP];
    float dout[TB];
    float red[TB / 32];
};

__device__ __forceinline__ float gelu_f(float z)
{
    return 0.5f * z * (1.f + tanhf(0.7978845608028654f * fmaf(0.044715f * z * z, z, z)));
}
__device__ __forceinline__ float gelu_prime_f(float z)
{
    const float tt = tanhf(0.7978845608028654f * fmaf(0.044715f * z * z, z, z));
    return 0.5f * (1.f + tt) + 0.5f * z * (1.f - tt * tt) * 0.7978845608028654f * fmaf(3.f * 0.044715f, z * z, 1.f);
}

// splitmix64 (Steele, Lea & Flood 2014): minibatch sample indices
__device__ __forceinline__ unsigned long long splitmix64(unsigned long long z)
{
    z += 0x9e3779b97f4a7c15ull;
    z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ull;
    z = (z ^ (z >> 27)) * 0x94d049bb133111ebull;
    return z ^ (z >> 31);
}

// Per block: forward and backward of TB samples in FP32, then the block's sum
// of per-sample parameter gradients (of the batch-mean squared error) and of
// the squared residuals, written to part[block * NPART + k]. Samples: rows
// base + i of X (feature-major, X[j * n + s]) when `seed` is 0, else rows
// splitmix64(seed + step * batch + i) mod n.
__global__ void __launch_bounds__(TB) k_mlp_grad(const float *__restrict__ X, const float *__restrict__ y,
                                                 long long n, long long batch, unsigned long long seed,
                                                 long long step, const float *__restrict__ theta,
                                                 float *__restrict__ part)
{
    extern __shared__ __align__(16) unsigned char smraw[];
    TrainSmem &sm = *reinterpret_cast<TrainSmem *>(smraw);
    const int tid = threadIdx.x;
    for (int k = tid; k < MLP_NPARAM; k += TB) sm.th[k] = theta[k];
    const long long pos = (long long)blockIdx.x * TB + tid;
    const bool valid = pos < batch;
    long long s = pos;
    if (seed && valid) s = (long long)(splitmix64(seed + (unsigned long long)(step * batch + pos)) % (unsigned long long)n);
    float x[MLP_NIN];
#pragma unroll
    for (int j = 0; j < MLP_NIN; j++) {
        x[j] = valid ? X[(long long)j * n + s] : 0.f;
        sm.x[j * TBP + tid] = x[j];
    }
    __syncthreads();
    const float *W1 = sm.th + MLP_OFF_W1, *b1 = sm.th + MLP_OFF_B1, *W2 = sm.th + MLP_OFF_W2;
    const float *b2 = sm.th + MLP_OFF_B2, *W3 = sm.th + MLP_OFF_W3;
    // forward
#pragma unroll 4
    for (int i = 0; i < MLP_NH; i++) {
        float z = b1[i];
#pragma unroll
        for (int j = 0; j < MLP_NIN; j++) z = fmaf(W1[i * MLP_NIN + j], x[j], z);
        sm.z1[i * TBP + tid] = z;
        sm.h1[i * TBP + tid] = gelu_f(z);
    }
    float o = sm.th[MLP_OFF_B3];
#pragma unroll 2
    for (int i = 0; i < MLP_NH; i++) {
        float z = b2[i];
#pragma unroll 8
        for (int j = 0; j < MLP_NH; j++) z = fmaf(W2[i * MLP_NH + j], sm.h1[j * TBP + tid], z);
        const float h = gelu_f(z);
        sm.z2[i * TBP + tid] = z;
        sm.h2[i * TBP + tid] = h;
        o = fmaf(W3[i], h, o);
    }
    const float r = valid ? o - y[s] : 0.f;
    const float dout = 2.f * r / float(batch);
    sm.dout[tid] = dout;
    // backward: dz2 = dout W3 gelu'(z2); dz1 = (W2^T dz2) gelu'(z1)
    for (int i = 0; i < MLP_NH; i++)
        sm.z2[i * TBP + tid] = dout * W3[i] * gelu_prime_f(sm.z2[i * TBP + tid]);
#pragma unroll 2
    for (int j = 0; j < MLP_NH; j++) {
        float a = 0.f;
#pragma unroll 8
        for (int i = 0; i < MLP_NH; i++) a = fmaf(W2[i * MLP_NH + j], sm.z2[i * TBP + tid], a);
        sm.z1[j * TBP + tid] = a * gelu_prime_f(sm.z1[j * TBP + tid]);
    }
    // squared residuals of the block
    float l2 = r * r;
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) l2 += __shfl_down_sync(0xffffffffu, l2, off);
    if ((tid & 31) == 0) sm.red[tid >> 5] = l2;
    __syncthreads();
    // parameter gradients summed over the block's samples
    float *out = part + (long long)blockIdx.x * NPART;
    for (int k = tid; k < MLP_NPARAM; k += TB) {
        float g = 0.f;
        if (k < MLP_OFF_B1) {
            const int i = k / MLP_NIN, j = k - i * MLP_NIN;
            for (int q = 0; q < TB; q++) g = fmaf(sm.z1[i * TBP + q], sm.x[j * TBP + q], g);
        } else if (k < MLP_OFF_W2) {
            const int i = k - MLP_OFF_B1;
            for (int q = 0; q < TB; q++) g += sm.z1[i * TBP + q];
        } else if (k < MLP_OFF_B2) {
            const int i = (k - MLP_OFF_W2) / MLP_NH, j = (k - MLP_OFF_W2) - i * MLP_NH;
            for (int q = 0; q < TB; q++) g = fmaf(sm.z2[i * TBP + q], sm.h1[j * TBP + q], g);
        } else if (k < MLP_OFF_W3) {
            const int i = k - MLP_OFF_B2;
            for (int q = 0; q < TB; q++) g += sm.z2[i * TBP + q];
        } else if (k < MLP_OFF_B3) {
            const int i = k - MLP_OFF_W3;
            for (int q = 0; q < TB; q++) g = fmaf(sm.dout[q], sm.h2[i * TBP + q], g);
        } else {
            for (int q = 0; q < TB; q++) g += sm.dout[q];
        }
        out[k] = g;
    }
    if (tid == 0) {
        float t = 0.f;
        for (int w = 0; w < TB / 32; w++) t += sm.red[w];
        out[MLP_NPARAM] = t;
    }
}

// grad[k] = sum over blocks of the partials (fixed order: reproducible);
// grad[NPARAM] = mean squared error of the batch
__global__ void k_mlp_reduce(const float *__restrict__ part, int nblocks, long long batch, float *__restrict__ grad,
                             float *__restrict__ loss_out)
{
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= NPART) return;
    float g = 0.f;
    for (int b = 0; b < nblocks; b++) g += part[(long long)b * NPART + k];
    if (k < MLP_NPARAM) grad[k] = g;
    else if (loss_out) *loss_out = g / float(batch);
}

// Adam (Kingma & Ba 2015, Algorithm 1), step t >= 1
__global__ void k_mlp_adam(float *__restrict__ th, const float *__restrict__ g, float *__restrict__ m,
                           float *__restrict__ v, int t, float lr, float b1, float b2, float eps)
{
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= MLP_NPARAM) return;
    const float gk = g[k];
    const float mk = b1 * m[k] + (1.f - b1) * gk;
    const float vk = b2 * v[k] + (1.f - b2) * gk * gk;
    m[k] = mk;
    v[k] = vk;
    // 1 - beta^t as -expm1(t ln beta), ln beta = log1p(-(1 - beta)): no cancellation for beta near 1
    const float mh = mk / -expm1f(float(t) * log1pf(-(1.f - b1)));
    const float vh = vk / -expm1f(float(t) * log1pf(-(1.f - b2)));
    th[k] -= lr * mh / (sqrtf(vh) + eps);
}

// FP32 forward (the training arithmetic), one thread per sample
__global__ void __launch_bounds__(128) k_mlp_fwd_fp32(const float *__restrict__ X, long long n,
                                                      const float *__restrict__ th, float *__restrict__ o)
{
    __shared__ float sth[MLP_NPARAM];
    for (int k = threadIdx.x; k < MLP_NPARAM; k += blockDim.x) sth[k] = th[k];
    __syncthreads();
    const long long s = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= n) return;
    float x[MLP_NIN], h1[MLP_NH];
#pragma unroll
    for (int j = 0; j < MLP_NIN; j++) x[j] = X[(long long)j * n + s];
#pragma unroll
    for (int i = 0; i < MLP_NH; i++) {
        float z = sth[MLP_OFF_B1 + i];
#pragma unroll
        for (int j = 0; j < MLP_NIN; j++) z = fmaf(sth[MLP_OFF_W1 + i * MLP_NIN + j], x[j], z);
        h1[i] = gelu_f(z);
    }
    float out = sth[MLP_OFF_B3];
    for (int i = 0; i < MLP_NH; i++) {
        float z = sth[MLP_OFF_B2 + i];
#pragma unroll
        for (int j = 0; j < MLP_NH; j++) z = fmaf(sth[MLP_OFF_W2 + i * MLP_NH + j], h1[j], z);
        out = fmaf(sth[MLP_OFF_W3 + i], gelu_f(z), out);
    }
    o[s] = out;
}

// BF16 tensor-core forward: 4 warps per block, 32 samples per warp and pass,
// grid-stride over warp tiles (the block loads the weights once)
__global__ void __launch_bounds__(128) k_mlp_fwd_bf16(const float *__restrict__ X, long long n,
                                                      const float *__restrict__ th, float *__restrict__ o)
{
    __shared__ MlpSmem sm;
    __shared__ __align__(16) __nv_bfloat16 xs[4][32 * MLP_XS];
    __shared__ float os[4][32];
    mlp_load_smem(th, sm);
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const long long ntiles = (n + 31) / 32;
    for (long long tile = (long long)blockIdx.x * 4 + w; tile < ntiles; tile += (long long)gridDim.x * 4) {
        const long long s = tile * 32 + lane;
        __nv_bfloat16 *row = xs[w] + lane * MLP_XS;
#pragma unroll
        for (int c = 0; c < 32; c += 2) {
            const float v0 = (s < n && c < MLP_NIN) ? X[(long long)c * n + s] : 0.f;
            const float v1 = (s < n && c + 1 < MLP_NIN) ? X[(long long)(c + 1) * n + s] : 0.f;
            *reinterpret_cast<unsigned *>(row + c) = pack_bf16x2(v0, v1);
        }
        __syncwarp();
        mlp_warp_bf16(sm, xs[w], os[w]);
        if (s < n) o[s] = os[w][lane];
        __syncwarp();
    }
}

// features X (feature-major) and S of sites given by FP32 deviations
__global__ void __launch_bounds__(128) k_alpha_features(const float *__restrict__ dev, long long n,
                                                        float *__restrict__ X, float *__restrict__ Sout)
{
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    float d[Q], f[Q], D[Q], drho, du, umax;
#pragma unroll
    for (int p = 0; p < Q; p++) d[p] = dev[(long long)p * n + i];
    site_delta(d, f, D, &drho, &du, &umax);
    float S = 0.f;
#pragma unroll
    for (int p = 0; p < Q; p++) S = fmaxf(S, fabsf(D[p] / f[p]));
    if (!(S > 0.f)) S = 1.f;
#pragma unroll
    for (int p = 0; p < Q; p++) X[(long long)p * n + i] = (D[p] / f[p]) / S;
    X[(long long)19 * n + i] = (log2f(S) + 9.f) * 0.125f;
    if (Sout) Sout[i] = S;
}

}  // namespace
}  // namespace elbm

using namespace elbm;

extern "C" long long elbm_mlp_workspace_floats(long long batch)
{
    if (batch <= 0) return 0;
    return ((batch + TB - 1) / TB) * (long long)NPART + NPART;
}

static elbm_status mlp_grad_enqueue(const float *X, const float *y, long long n, long long batch,
                                    unsigned long long seed, long long step, const float *theta, float *grad,
                                    float *loss, float *work, cudaStream_t s)
{
    const int nb = (int)((batch + TB - 1) / TB);
    if (cudaFuncSetAttribute(k_mlp_grad, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sizeof(TrainSmem)) !=
        cudaSuccess)
        return ELBM_E_CUDA;
    k_mlp_grad<<<nb, TB, sizeof(TrainSmem), s>>>(X, y, n, batch, seed, step, theta, work);
    k_mlp_reduce<<<(NPART + 255) / 256, 256, 0, s>>>(work, nb, batch, grad, loss);
    return cudaGetLastError() == cudaSuccess ? ELBM_OK : ELBM_E_CUDA;
}

extern "C" elbm_status elbm_alpha_features(const float *d, long long n, float *X, float *S, void *stream)
{
    if (n < 0 || (n > 0 && (!d || !X))) return ELBM_E_INVAL;
    if (n == 0) return ELBM_OK;
    k_alpha_features<<<(unsigned)((n + 127) / 128), 128, 0, (cudaStream_t)stream>>>(d, n, X, S);
    return cudaGetLastError() == cudaSuccess ? ELBM_OK : ELBM_E_CUDA;
}

extern "C" elbm_status elbm_mlp_forward(const float *X, long long n, const float *theta, int arith, float *o,
                                        void *stream)
{
    if (n < 0 || (n > 0 && (!X || !theta || !o))) return ELBM_E_INVAL;
    if (arith != ELBM_MLP_FP32 && arith != ELBM_MLP_BF16_TC) return ELBM_E_INVAL;
    if (n == 0) return ELBM_OK;
    cudaStream_t s = (cudaStream_t)stream;
    if (arith == ELBM_MLP_FP32) {
        k_mlp_fwd_fp32<<<(unsigned)((n + 127) / 128), 128, 0, s>>>(X, n, theta, o);
    } else {
        const long long tiles = (n + 31) / 32;
        const long long blocks = (tiles + 3) / 4;
        k_mlp_fwd_bf16<<<(unsigned)(blocks < 4 * 152 ? blocks : 4 * 152), 128, 0, s>>>(X, n, theta, o);
    }
    return cudaGetLastError() == cudaSuccess ? ELBM_OK : ELBM_E_CUDA;
}

extern "C" elbm_status elbm_mlp_grad(const float *X, const float *y, long long n, const float *theta, float *grad,
                                     float *loss, float *work, void *stream)
{
    if (n <= 0 || !X || !y || !theta || !grad || !work) return ELBM_E_INVAL;
    return mlp_grad_enqueue(X, y, n, n, 0ull, 0, theta, grad, loss, work, (cudaStream_t)stream);
}

extern "C" elbm_status elbm_mlp_adam(float *theta, const float *grad, float *m, float *v, int t, float lr,
                                     float beta1, float beta2, float eps, void *stream)
{
    if (!theta || !grad || !m || !v || t < 1 || !(lr > 0.f) || !(beta1 >= 0.f && beta1 < 1.f) ||
        !(beta2 >= 0.f && beta2 < 1.f) || !(eps > 0.f))
        return ELBM_E_INVAL;
    k_mlp_adam<<<(MLP_NPARAM + 255) / 256, 256, 0, (cudaStream_t)stream>>>(theta, grad, m, v, t, lr, beta1, beta2,
                                                                           eps);
    return cudaGetLastError() == cudaSuccess ? ELBM_OK : ELBM_E_CUDA;
}

extern "C" elbm_status elbm_mlp_train(const float *X, const float *y, long long n, float *theta, float *m, float *v,
                                      int t0, int steps, long long batch, float lr, unsigned long long seed,
                                      float *loss_hist, float *work, void *stream)
{
    if (n <= 0 || !X || !y || !theta || !m || !v || !work || t0 < 0 || steps < 0 || batch <= 0 || !(lr > 0.f) ||
        seed == 0)
        return ELBM_E_INVAL;
    cudaStream_t s = (cudaStream_t)stream;
    float *grad = work + ((batch + TB - 1) / TB) * (long long)NPART;
    for (int k = 0; k < steps; k++) {
        elbm_status st = mlp_grad_enqueue(X, y, n, batch, seed, t0 + k, theta, grad, loss_hist ? loss_hist + k : nullptr,
                                          work, s);
        if (st != ELBM_OK) return st;
        k_mlp_adam<<<(MLP_NPARAM + 255) / 256, 256, 0, s>>>(theta, grad, m, v, t0 + k + 1, lr, 0.9f, 0.999f, 1e-8f);
    }
    return cudaGetLastError() == cudaSuccess ? ELBM_OK : ELBM_E_CUDA;
}
