// elbm_alpha_api.cu -- elbm_alpha_eval: the entropic alpha of Eq. (entropic)
// for independent sites outside a simulation (tests of the root's H-error
// against an FP64 evaluation; (f, alpha) pairs for the learned proposal).
#include <cuda_runtime.h>

#include "elbm.h"
#include "elbm_device.cuh"

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
    // moments and Eq. (2) in FP32, in the order of the FP32 collision
    float rs = 0.f, jx = 0.f, jy = 0.f, jz = 0.f;
#pragma unroll
    for (int p = 0; p < Q; p++) {
        rs += d[p];
        jx += float(cx(p)) * d[p];
        jy += float(cy(p)) * d[p];
        jz += float(cz(p)) * d[p];
    }
    const float r = 1.f + rs, drho = rs;
    const float ir = 1.f / r;
    const float ux = jx * ir, uy = jy * ir, uz = jz * ir;
    const float usq = ux * ux + uy * uy + uz * uz;
    float D[Q], f[Q];
#pragma unroll
    for (int p = 0; p < Q; p++) {
        const float P = Ppoly<float>(p, ux, uy, uz, usq);
        D[p] = float(wq(p)) * (drho + r * P) - d[p];
        f[p] = float(wq(p)) + d[p];
        if (delta) delta[(long long)p * n + i] = D[p];
    }
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
        AlphaOutF ao = alpha_fp32(f, D, d, r, drho, eq_tol_f, AP == ELBM_APREC_FP32);
        a = double(ao.alpha) + double(ao.alpha_lo);
        he = ao.herr;
        st = ao.status;
    }
    alpha[i] = a;
    if (herr) herr[i] = he;
    if (status) status[i] = st;
}

}  // namespace
}  // namespace elbm

extern "C" elbm_status elbm_alpha_eval(const float *d, long long n, int aprec, double eq_tol,
                                       const float *mlp, double *alpha, float *herr, int *status,
                                       float *delta, void *stream)
{
    using namespace elbm;
    if (n < 0 || (n > 0 && (!d || !alpha))) return ELBM_E_INVAL;
    if (aprec < ELBM_APREC_FP64 || aprec > ELBM_APREC_FP32_FAST) return ELBM_E_INVAL;
    if (!(eq_tol >= 0.0) || (aprec != ELBM_APREC_FP64 && eq_tol < 0x1p-18)) return ELBM_E_INVAL;
    if (mlp) return ELBM_E_INVAL;  // the learned proposal is not available through this entry point yet
    if (n == 0) return ELBM_OK;
    const unsigned blocks = (unsigned)((n + 127) / 128);
    cudaStream_t s = (cudaStream_t)stream;
    const float tf = float(eq_tol);
    if (aprec == ELBM_APREC_FP64)
        k_alpha_eval<ELBM_APREC_FP64><<<blocks, 128, 0, s>>>(d, n, tf, eq_tol, alpha, herr, status, delta);
    else if (aprec == ELBM_APREC_FP32)
        k_alpha_eval<ELBM_APREC_FP32><<<blocks, 128, 0, s>>>(d, n, tf, eq_tol, alpha, herr, status, delta);
    else
        k_alpha_eval<ELBM_APREC_FP32_FAST><<<blocks, 128, 0, s>>>(d, n, tf, eq_tol, alpha, herr, status, delta);
    return cudaGetLastError() == cudaSuccess ? ELBM_OK : ELBM_E_CUDA;
}
