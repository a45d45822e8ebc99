// elbm_mlp.cuh -- the learned alpha proposal on the GPU: site features and
// BF16 tensor-core inference of the 20 -> 64 -> 64 -> 1 gelu network.
//
// The paper computes alpha as the root of Eq. (entropic) and has no learned
// part. The proposal alpha = alpha_c + S^3 o(X) starts the Newton iteration
// on the paper's h(alpha), alpha_c being the moment-series start (the root of
// the cubic truncation of h, whose error is O(S^3)); a lane that is not
// converged after one evaluation falls back to the full Newton iteration, and
// the float-float guard certifies the H-error as for the plain root. Features
// of a site, x_p = Delta_p / f_p, S = max |x_p|:
// X = (x_0/S, ..., x_18/S, (log2 S + 9)/8).
//
// Parameters: one FP32 vector (the training master copy), in the order W1
// (64 x 20, out x in), b1 (64), W2 (64 x 64), b2 (64), W3 (64), b3 (1).
//
// Inference: one warp evaluates the network for 32 sites with
// mma.sync.m16n8k16 (BF16 operands, FP32 accumulation): layer 1 is
// [32 x 32 (20 features, zero padded)] x [32 x 64], layer 2 [32 x 64] x
// [64 x 64]; layer 3 (64 -> 1) is an FP32 dot product. The layer-1
// accumulator fragments, after bias and gelu, are exactly the A fragments of
// layer 2 (two n8 tiles form one k16 slice), so activations stay in
// registers. Weights sit in shared memory as BF16 with padded rows (40 and
// 72 elements) so that the fragment loads are free of bank conflicts.
#pragma once

#include <cuda_bf16.h>

#include "elbm_device.cuh"

namespace elbm {
ELBM_VS_BEGIN

constexpr int MLP_NIN = 20, MLP_NH = 64;
constexpr int MLP_OFF_W1 = 0, MLP_OFF_B1 = MLP_NH * MLP_NIN, MLP_OFF_W2 = MLP_OFF_B1 + MLP_NH,
              MLP_OFF_B2 = MLP_OFF_W2 + MLP_NH * MLP_NH, MLP_OFF_W3 = MLP_OFF_B2 + MLP_NH,
              MLP_OFF_B3 = MLP_OFF_W3 + MLP_NH, MLP_NPARAM = MLP_OFF_B3 + 1;
constexpr int MLP_W1S = 40, MLP_W2S = 72, MLP_XS = 40;  // padded row strides (BF16 elements)

struct __align__(16) MlpSmem {
    __nv_bfloat16 w1[MLP_NH * MLP_W1S];
    __nv_bfloat16 w2[MLP_NH * MLP_W2S];
    float b1[MLP_NH], b2[MLP_NH], w3[MLP_NH], b3, pad[3];
};
static_assert(sizeof(MlpSmem) % 16 == 0, "MlpSmem is copied as 16-byte words");

// FP32 master parameters -> BF16 padded layout (whole block; ends with a barrier)
__device__ __forceinline__ void mlp_load_smem(const float *__restrict__ th, MlpSmem &sm)
{
    for (int i = threadIdx.x; i < MLP_NH * MLP_W1S; i += blockDim.x) {
        const int r = i / MLP_W1S, c = i - r * MLP_W1S;
        sm.w1[i] = __float2bfloat16_rn(c < MLP_NIN ? th[MLP_OFF_W1 + r * MLP_NIN + c] : 0.f);
    }
    for (int i = threadIdx.x; i < MLP_NH * MLP_W2S; i += blockDim.x) {
        const int r = i / MLP_W2S, c = i - r * MLP_W2S;
        sm.w2[i] = __float2bfloat16_rn(c < MLP_NH ? th[MLP_OFF_W2 + r * MLP_NH + c] : 0.f);
    }
    for (int i = threadIdx.x; i < MLP_NH; i += blockDim.x) {
        sm.b1[i] = th[MLP_OFF_B1 + i];
        sm.b2[i] = th[MLP_OFF_B2 + i];
        sm.w3[i] = th[MLP_OFF_W3 + i];
    }
    if (threadIdx.x == 0) sm.b3 = th[MLP_OFF_B3];
    __syncthreads();
}

// gelu, tanh form (Hendrycks & Gimpel 2016); tanh.approx.f32 for inference
__device__ __forceinline__ float tanh_approx(float x)
{
    float y;
    asm("tanh.approx.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}
__device__ __forceinline__ float gelu_fast(float z)
{
    const float u = 0.7978845608028654f * fmaf(0.044715f * z * z, z, z);
    return 0.5f * z * (1.f + tanh_approx(u));
}

__device__ __forceinline__ unsigned pack_bf16x2(float lo, float hi)
{
    const __nv_bfloat162 v = __floats2bfloat162_rn(lo, hi);  // .x = lo (lower address)
    return *reinterpret_cast<const unsigned *>(&v);
}

__device__ __forceinline__ void mma_bf16_16816(float (&d)[4], const unsigned (&a)[4], unsigned b0, unsigned b1)
{
    asm volatile(
        "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
        "{%0,%1,%2,%3};\n"
        : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
        : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}

__device__ __forceinline__ unsigned lds32(const __nv_bfloat16 *p)
{
    return *reinterpret_cast<const unsigned *>(p);
}

// The network for the 32 sites of a warp. xs: the warp's feature tile in
// shared memory, 32 rows (sites) x MLP_XS BF16 (columns 20..31 zero); o: 32
// outputs (shared memory). Every lane of the warp must call it.
__device__ __forceinline__ void mlp_warp_bf16(const MlpSmem &sm, const __nv_bfloat16 *xs, float *o)
{
    unsigned lane;  // the lane in the warp (not threadIdx.x: blocks may be two-dimensional)
    asm("mov.u32 %0, %%laneid;" : "=r"(lane));
    const int g = int(lane >> 2), t = int(lane & 3);
#pragma unroll 1
    for (int mt = 0; mt < 2; mt++) {
        const __nv_bfloat16 *xr0 = xs + (mt * 16 + g) * MLP_XS;
        const __nv_bfloat16 *xr1 = xr0 + 8 * MLP_XS;
        // layer 1: acc[nt] = X W1^T + b1
        float acc[8][4];
#pragma unroll
        for (int nt = 0; nt < 8; nt++) {
            const float c0 = sm.b1[nt * 8 + 2 * t], c1 = sm.b1[nt * 8 + 2 * t + 1];
            acc[nt][0] = c0; acc[nt][1] = c1; acc[nt][2] = c0; acc[nt][3] = c1;
        }
#pragma unroll
        for (int ks = 0; ks < 2; ks++) {
            const int k0 = ks * 16 + 2 * t;
            const unsigned a[4] = {lds32(xr0 + k0), lds32(xr1 + k0), lds32(xr0 + k0 + 8), lds32(xr1 + k0 + 8)};
#pragma unroll
            for (int nt = 0; nt < 8; nt++) {
                const __nv_bfloat16 *wr = sm.w1 + (nt * 8 + g) * MLP_W1S + k0;
                mma_bf16_16816(acc[nt], a, lds32(wr), lds32(wr + 8));
            }
        }
        // gelu; the accumulators of n tiles 2j, 2j+1 are the A fragment of k slice j
        unsigned a2[4][4];
#pragma unroll
        for (int j = 0; j < 4; j++) {
            a2[j][0] = pack_bf16x2(gelu_fast(acc[2 * j][0]), gelu_fast(acc[2 * j][1]));
            a2[j][1] = pack_bf16x2(gelu_fast(acc[2 * j][2]), gelu_fast(acc[2 * j][3]));
            a2[j][2] = pack_bf16x2(gelu_fast(acc[2 * j + 1][0]), gelu_fast(acc[2 * j + 1][1]));
            a2[j][3] = pack_bf16x2(gelu_fast(acc[2 * j + 1][2]), gelu_fast(acc[2 * j + 1][3]));
        }
        // layer 2
#pragma unroll
        for (int nt = 0; nt < 8; nt++) {
            const float c0 = sm.b2[nt * 8 + 2 * t], c1 = sm.b2[nt * 8 + 2 * t + 1];
            acc[nt][0] = c0; acc[nt][1] = c1; acc[nt][2] = c0; acc[nt][3] = c1;
        }
#pragma unroll
        for (int j = 0; j < 4; j++) {
            const int k0 = j * 16 + 2 * t;
#pragma unroll
            for (int nt = 0; nt < 8; nt++) {
                const __nv_bfloat16 *wr = sm.w2 + (nt * 8 + g) * MLP_W2S + k0;
                mma_bf16_16816(acc[nt], a2[j], lds32(wr), lds32(wr + 8));
            }
        }
        // layer 3 (FP32): rows g and g + 8 of this m tile
        float s0 = 0.f, s1 = 0.f;
#pragma unroll
        for (int nt = 0; nt < 8; nt++) {
            const float w0 = sm.w3[nt * 8 + 2 * t], w1 = sm.w3[nt * 8 + 2 * t + 1];
            s0 = fmaf(w0, gelu_fast(acc[nt][0]), fmaf(w1, gelu_fast(acc[nt][1]), s0));
            s1 = fmaf(w0, gelu_fast(acc[nt][2]), fmaf(w1, gelu_fast(acc[nt][3]), s1));
        }
        s0 += __shfl_xor_sync(0xffffffffu, s0, 1);
        s0 += __shfl_xor_sync(0xffffffffu, s0, 2);
        s1 += __shfl_xor_sync(0xffffffffu, s1, 1);
        s1 += __shfl_xor_sync(0xffffffffu, s1, 2);
        if (t == 0) {
            o[mt * 16 + g] = s0 + sm.b3;
            o[mt * 16 + g + 8] = s1 + sm.b3;
        }
    }
    __syncwarp();
}

// features of one site (x_p = Delta_p / f_p, S = max |x_p| > 0) into its row
// of a warp tile
__device__ __forceinline__ void mlp_site_features(const float *x, float S, __nv_bfloat16 *xrow)
{
    const float iS = 1.f / S;
#pragma unroll
    for (int p = 0; p < Q; p += 2) {
        const float v1 = p + 1 < Q ? x[p + 1] * iS : (__log2f(S) + 9.f) * 0.125f;
        *reinterpret_cast<unsigned *>(xrow + p) = pack_bf16x2(x[p] * iS, v1);
    }
#pragma unroll
    for (int c = 20; c < 32; c += 2) *reinterpret_cast<unsigned *>(xrow + c) = 0u;
}

ELBM_VS_END
}  // namespace elbm
