// elbm_internal.h -- host-side state of a handle and the per-precision kernel
// launchers (implemented in k_fp64.cu / k_fp32.cu / k_bf16.cu, and for the
// D2Q9 set in k_fp64_d2q9.cu / k_fp32_d2q9.cu).
#pragma once

#include <cuda_runtime.h>
#include "elbm.h"
#include "elbm_device.cuh"

namespace elbm {

// slots of the device scalar array
enum {
    S_QSUM = 0, S_Q2, S_QMEAN, S_SA, S_SB, S_R2, S_RQ2, S_RB2, S_RESID, S_CONV,
    S_PHISUM, S_PHIMEAN,
    S_ITER,        // Poisson units (V-cycles, or groups of SOR sweeps) of this step
    S_PREV,        // residual norm at the previous convergence test
    S_NOCONV,      // solves that hit the cap without converging (cumulative)
    S_ITER_TOTAL,  // Poisson units over all steps
    S_STEPS,       // completed steps
    S_KEEP,        // 1 while the Poisson loop must go on
    S_HAVE_OLD,    // 1 once phi(t-1) is recorded for the extrapolated warm start
    S_INRATIO,     // adaptive inlet: scale of the initial inlet profile for the next step
    S_NSCAL = 24
};
// per-block partial slots of the collision diagnostics
enum {
    D_MASS = 0, D_MX, D_MY, D_MZ, D_Q, D_AMIN, D_AMAX, D_ASUM, D_NSHORT, D_NNOROOT,
    D_NCLIP, D_HERR, D_UMAX, D_NBAD, D_NFLUID, D_NGUARD, D_NGFAIL, D_NLFALL, D_NPART = 18,
    D_UIN = 18     // adaptive inlet: per-block sum of u . d over the region (every step)
};

struct Phys {
    Cst<double> cd;                   // constants in FP64
    Cst<float> cf;                    // the same constants rounded to FP32
    double tol, rho_in, rho_out;      // host / reduction-side values
    double n_fluid, n_unknown;
    int charge_model, force_el, alpha_mode, aprec, store_macro, neutralize, newtonian;
    int eps_face, carreau_lagged;
    // adaptive inlet: direction d, mean of the initial profile along d, region sites
    int adaptive, n_inlet;
    double in_d[3], in_m0, n_region;
};

template <typename T> __host__ __device__ __forceinline__ const Cst<T> &cst(const Phys &ph);
template <> __host__ __device__ __forceinline__ const Cst<double> &cst<double>(const Phys &ph) { return ph.cd; }
template <> __host__ __device__ __forceinline__ const Cst<float> &cst<float>(const Phys &ph) { return ph.cf; }

struct Bufs {
    void *fA, *fB, *gA, *gB;          // populations (current A, next B)
    float *rA, *rB;                   // BF16 storage: reference density of each stored site (A/B)
    void *rho, *q, *phi;              // scalar planes
    void *psi, *sig;                  // psi(rho) of the Shan-Chen force; sigma(rho) (transport mode)
    void *ux, *uy, *uz, *alpha, *nu;  // optional macroscopic planes
    float *alpha_lo;                  // reduced precision: low part of a guarded alpha (with store_macro)
    unsigned char *mask;              // node kinds (NULL when all fluid)
    // per site, bit p set when the pull of population p comes back from a
    // wall face or a solid node (bits 0..6 also serve the D3Q7 pull, whose
    // directions are D3Q19's first seven); NULL when every pull is a plain
    // gather (all faces periodic, no solid node)
    const unsigned *bbits;
    void *E2;                         // FULL electric force: |E|^2 per site
    const unsigned char *region;      // adaptive inlet: sites of the nozzle mean (NULL: fixed inlet)
    const int *inlet_idx;             // adaptive inlet: the inlet nodes
    const double *inlet_u0;           // adaptive inlet: their initial velocities (3 each)
    void *nh;                         // paper-mode charge: 4 planes n_x, n_y, n_z, |grad rho|^2
    void *ab;                         // conserved paper-mode charge: 2 planes a, b (NULL otherwise)
    double *part;                     // per-block partial sums
    double *scal;                     // device scalars (S_*)
    float *scalf;                     // the same scalars rounded to FP32
    double *colres;                   // per-column results of the finalize kernel
    unsigned int *ticket;             // last-block-done counter of the finalize kernel
    // sticky record of the steps without diagnostics since the last ones:
    // [0] their max H-error (order-preserving bits of a float >= 0),
    // [1] their flags (1 non-finite or non-positive density, 2 guard failure)
    unsigned int *sticky;
    double *diag;                     // ELBM_NDIAG diagnostics
    const void *mlpimg;               // learned alpha: BF16 shared-memory image of the network
    void *phi_old;                    // potential of the previous step (extrapolated warm start)
};

struct Launch {
    dim3 block, grid;
    int nblocks;
};

// Per-precision launchers. All enqueue on `s` and never synchronise.
struct Ops {
    void (*init_pop)(const Geom &, const Phys &, const Bufs &, const double *rho0,
                     const double *u0, const double *f0, const double *u_in,
                     const double *q0, const Launch &, cudaStream_t);
    void (*moments)(const Geom &, const Phys &, const Bufs &, const Launch &, cudaStream_t);
    // stage 0: gradient/normal and the per-site a, b with their block sums;
    // stage 1: q from the finalised sums, with block sums of q and q^2
    void (*charge)(const Geom &, const Phys &, const Bufs &, int stage, const Launch &, cudaStream_t);
    void (*sor)(const Geom &, const Phys &, const Bufs &, int color, const Launch &, cudaStream_t);
    // zc: the colour whose residual is taken as 0 (the one a Gauss-Seidel
    // sweep updated last), or -1
    void (*resid)(const Geom &, const Phys &, const Bufs &, int zc, const Launch &, cudaStream_t);
    // stage 0: block sums of phi over non-solid nodes; stage 1: subtract S_PHIMEAN
    void (*phi_mean)(const Geom &, const Phys &, const Bufs &, int stage, const Launch &, cudaStream_t);
    void (*collide)(const Geom &, const Phys &, const Bufs &, int diag, const Launch &, cudaStream_t);
    // FULL electric force: |E|^2 of every site into the E2 plane, before the collision
    void (*efield2)(const Geom &, const Phys &, const Bufs &, const Launch &, cudaStream_t);
    // adaptive inlet: the rescaled inlet equilibria into the buffer of the next step
    void (*inlet)(const Geom &, const Phys &, const Bufs &, cudaStream_t);
    // warm start of the Poisson solve: phi <- 2 phi - phi_old, phi_old <- phi
    void (*phi_extrap)(const Geom &, const Bufs &, cudaStream_t);
    void (*export_pop)(const Geom &, const Bufs &, double *out, const Launch &, cudaStream_t);
    void (*export_gpop)(const Geom &, const Bufs &, double *out, const Launch &, cudaStream_t);
    void (*export_plane)(const void *plane, double *out, long long n, cudaStream_t);
    // out[i] += lo[i] (the low part of a float-float plane)
    void (*add_plane)(const float *lo, double *out, long long n, cudaStream_t);
    // the bounce bits of every site (Bufs.bbits), once at elbm_init
    void (*bounce_bits)(const Geom &, const Bufs &, const Launch &, cudaStream_t);
    // the site-wide compute kernels (the collision variants): in a batch
    // graph every other kernel runs at a higher priority
    const void *heavy[5];
};

struct MGLevel;  // elbm_kernels.cuh
struct MGTail;   // elbm_kernels.cuh
struct MGOps {
    void (*tail)(const Geom &, const MGTail &, int nu, cudaStream_t);
    void (*prepare)();  // kernel attributes (shared-memory opt-in), before any capture
    void (*smooth)(const Geom &, const Phys &, const Bufs &, const MGLevel &, int level, int color,
                   const Launch &fine_half, cudaStream_t);
    void (*restrict_)(const Geom &, const Phys &, const Bufs &, const MGLevel &F, const MGLevel &C, int level,
                      int zc, cudaStream_t);
    void (*eps)(const Geom &, const Phys &, const Bufs &, const MGLevel &F, const MGLevel &C, int level,
                cudaStream_t);
    void (*prolong)(const Geom &, const Bufs &, const MGLevel &F, const MGLevel &C, int level, cudaStream_t);
};

Ops ops_fp64();
Ops ops_fp32();
Ops ops_bf16();
// the same kernels for the D2Q9 set (k_fp64_d2q9.cu / k_fp32_d2q9.cu)
Ops ops_fp64_d2q9();
Ops ops_fp32_d2q9();
// public population order and weights of D2Q9 (c: 3 per population)
int vset_d2q9(int *c, double *w);
MGOps mgops_fp64();
MGOps mgops_fp32();

}  // namespace elbm
