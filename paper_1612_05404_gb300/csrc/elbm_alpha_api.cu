// elbm_alpha_api.cu -- elbm_alpha_eval: the entropic alpha of Eq. (entropic)
// for independent sites outside a simulation (tests of the root's H-error
// against an FP64 evaluation; (f, alpha) pairs for the learned proposal).
#include <cuda_runtime.h>

#include "elbm.h"
#include "elbm_device.cuh"
#include "elbm_mlp.cuh"

namespace elbm {
namespace {

template <int AP>
__global__ void __launch_bounds__(128, AP == ELBM_APREC_FP64 ? 1 : 4)
k_alpha_eval(const float *__restrict__ dev, long long n, float eq_tol_f, double eq_tol_d,
             double *__restrict__ alpha, float *__restrict__ herr, int *__restrict__ status,
             float *__restrict__ delta)
{
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    float d[Q];
#pragma unroll
    for (int p = 0; p < Q; p++) d[p] = dev[(long long)p * n + i];
    // moments and Eq. (2) in FP32, as the FP32 collision forms them
    float D[Q], f[Q], drho, du, umax;
    const float r = site_delta(d, f, D, &drho, &du, &umax);
    if (delta)
        for (int p = 0; p < Q; p++) delta[(long long)p * n + i] = D[p];
    double a;
    float he;
    int st;
    if (AP == ELBM_APREC_FP64) {
        double fd[Q], dd[Q];
#pragma unroll
        for (int p = 0; p < Q; p++) {
            fd[p] = double(f[p]);
            dd[p] = double(D[p]);
        }
        AlphaOut ao = alpha_fp64(fd, dd, double(r), eq_tol_d);
        a = ao.alpha;
        he = float(ao.herr);
        st = ao.status;
    } else {
        AlphaOutF ao = alpha_fp32(f, D, d, r, drho, eq_tol_f, du, umax, AP == ELBM_APREC_FP32);
        a = double(ao.alpha) + double(ao.alpha_lo);
        he = ao.herr;
        st = (ao.status == 0 && ao.iters > 1) ? 5 : ao.status;
    }
    alpha[i] = a;
    if (herr) herr[i] = he;
    if (status) status[i] = st;
}

// The learned proposal: series start, features and the BF16 tensor-core
// network for the 32 sites of each warp, then the FP32 Newton iteration from
// alpha = alpha_c + S^3 o(X) where S >= 2^-5, else alpha_c (status 5: the lane needed more than one
// evaluation, i.e. fell back to the full iteration) and the same float-float
// guard.
template <int AP>
__global__ void __launch_bounds__(128) k_alpha_eval_learned(const float *__restrict__ dev, long long n,
                                                            float eq_tol_f, const float *__restrict__ th,
                                                            double *__restrict__ alpha, float *__restrict__ herr,
                                                            int *__restrict__ status, float *__restrict__ delta)
{
    __shared__ MlpSmem sm;
    __shared__ __align__(16) __nv_bfloat16 xs[4][32 * MLP_XS];
    __shared__ float os[4][32];
    mlp_load_smem(th, sm);
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const bool valid = i < n;
    float d[Q], f[Q], D[Q], drho, du, umax;
#pragma unroll
    for (int p = 0; p < Q; p++) d[p] = valid ? dev[(long long)p * n + i] : 0.f;
    const float r = site_delta(d, f, D, &drho, &du, &umax);
    if (delta && valid)
        for (int p = 0; p < Q; p++) delta[(long long)p * n + i] = D[p];
    AlphaSetupF st;
    alpha_fp32_setup(f, D, d, r, drho, eq_tol_f, du, umax, st);
    mlp_site_features(st.x, st.S > 0.f ? st.S : 1.f, xs[w] + lane * MLP_XS);
    __syncwarp();
    mlp_warp_bf16(sm, xs[w], os[w]);
    const float am = st.S >= 0x1p-5f ? st.ac + st.S * st.S * st.S * os[w][lane] : st.ac;
    if (!valid) return;
    AlphaOutF ao = alpha_fp32_solve(f, D, d, r, st, AP == ELBM_APREC_FP32, am);
    alpha[i] = double(ao.alpha) + double(ao.alpha_lo);
    if (herr) herr[i] = ao.herr;
    if (status) status[i] = (ao.status == 0 && ao.iters > 1) ? 5 : ao.status;
}

// Training pairs: the guarded FP32 root alpha* (|h| <= 1e-10 rho), features X
// (feature-major), target y = (alpha* - alpha_c)/S^3 clipped to [-8, 8], keep =
// 1 for a root with S >= 2^-5 (below, S^3 o is under the FP32 resolution of
// alpha_c, the proposal is alpha_c itself, and the target would be rounding
// noise of alpha_c divided by S^3).
__global__ void __launch_bounds__(128) k_alpha_harvest(const float *__restrict__ dev, long long n, float eq_tol_f,
                                                       float *__restrict__ X, float *__restrict__ y,
                                                       int *__restrict__ keep)
{
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    float d[Q], f[Q], D[Q], drho, du, umax;
#pragma unroll
    for (int p = 0; p < Q; p++) d[p] = dev[(long long)p * n + i];
    const float r = site_delta(d, f, D, &drho, &du, &umax);
    AlphaSetupF st;
    alpha_fp32_setup(f, D, d, r, drho, eq_tol_f, du, umax, st);
    const float S = st.S > 0.f ? st.S : 1.f;
    const float iS = 1.f / S;
#pragma unroll
    for (int p = 0; p < Q; p++) X[(long long)p * n + i] = st.x[p] * iS;
    X[(long long)19 * n + i] = (__log2f(S) + 9.f) * 0.125f;
    AlphaOutF ao = alpha_fp32_solve(f, D, d, r, st, true, -1.f);
    const bool ok = ao.status == 0 && st.S >= 0x1p-5f;
    const double t = ok ? ((double(ao.alpha) - double(st.ac)) + double(ao.alpha_lo)) / (double(S) * S * S) : 0.0;
    y[i] = float(fmin(8.0, fmax(-8.0, t)));
    keep[i] = ok ? 1 : 0;
}

}  // namespace
}  // namespace elbm

extern "C" elbm_status elbm_alpha_harvest(const float *d, long long n, double eq_tol, float *X, float *y, int *keep,
                                          void *stream)
{
    using namespace elbm;
    if (n < 0 || (n > 0 && (!d || !X || !y || !keep)) || !(eq_tol >= 0x1p-18)) return ELBM_E_INVAL;
    if (n == 0) return ELBM_OK;
    k_alpha_harvest<<<(unsigned)((n + 127) / 128), 128, 0, (cudaStream_t)stream>>>(d, n, float(eq_tol), X, y, keep);
    return cudaGetLastError() == cudaSuccess ? ELBM_OK : ELBM_E_CUDA;
}

extern "C" elbm_status elbm_alpha_eval(const float *d, long long n, int aprec, double eq_tol,
                                       const float *mlp, double *alpha, float *herr, int *status,
                                       float *delta, void *stream)
{
    using namespace elbm;
    if (n < 0 || (n > 0 && (!d || !alpha))) return ELBM_E_INVAL;
    if (aprec < ELBM_APREC_FP64 || aprec > ELBM_APREC_FP32_FAST) return ELBM_E_INVAL;
    if (!(eq_tol >= 0.0) || (aprec != ELBM_APREC_FP64 && eq_tol < 0x1p-18)) return ELBM_E_INVAL;
    if (mlp && aprec == ELBM_APREC_FP64) return ELBM_E_INVAL;  // the proposal starts the FP32 iteration
    if (n == 0) return ELBM_OK;
    const unsigned blocks = (unsigned)((n + 127) / 128);
    cudaStream_t s = (cudaStream_t)stream;
    const float tf = float(eq_tol);
    if (mlp) {
        if (aprec == ELBM_APREC_FP32)
            k_alpha_eval_learned<ELBM_APREC_FP32><<<blocks, 128, 0, s>>>(d, n, tf, mlp, alpha, herr, status, delta);
        else
            k_alpha_eval_learned<ELBM_APREC_FP32_FAST><<<blocks, 128, 0, s>>>(d, n, tf, mlp, alpha, herr, status, delta);
        return cudaGetLastError() == cudaSuccess ? ELBM_OK : ELBM_E_CUDA;
    }
    if (aprec == ELBM_APREC_FP64)
        k_alpha_eval<ELBM_APREC_FP64><<<blocks, 128, 0, s>>>(d, n, tf, eq_tol, alpha, herr, status, delta);
    else if (aprec == ELBM_APREC_FP32)
        k_alpha_eval<ELBM_APREC_FP32><<<blocks, 128, 0, s>>>(d, n, tf, eq_tol, alpha, herr, status, delta);
    else
        k_alpha_eval<ELBM_APREC_FP32_FAST><<<blocks, 128, 0, s>>>(d, n, tf, eq_tol, alpha, herr, status, delta);
    return cudaGetLastError() == cudaSuccess ? ELBM_OK : ELBM_E_CUDA;
}
