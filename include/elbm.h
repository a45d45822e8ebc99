/*
 * elbm.h -- C ABI of the GB300 (sm_103a) charged entropic lattice Boltzmann
 * library: one time step of Lauricella et al., "Entropic Lattice Boltzmann
 * Model for Charged Leaky Dielectric Multiphase Fluids in Electrified Jets"
 * (arXiv:1612.05404), Sec. II, on a 3-D D3Q19 lattice, or on the paper's own
 * 2-D D2Q9 lattice (params.velset; the paper's experiments, Sec. III, are 2-D).
 *
 * One step (Sec. II C) is: moments; free charge (Eqs. surface-q2 / surface-q3,
 * or the transported D3Q7 charge); neutralisation and the variable-permittivity
 * Poisson equation div(eps grad phi) = -q (Sec. II); Shan-Chen force Eq. (sc);
 * electric force Eq. (force_el2); entropic alpha Eq. (entropic) with Eq. (H);
 * Carreau viscosity Eqs. (stress), (strain2), (carreau), (beta); the update
 * Eq. (lattice-b) with the exact-difference source Eq. (add); streaming.
 *
 * Conventions
 *  - Every call returns an elbm_status (0 = success). Nothing is printed, no
 *    call exits the process. elbm_strerror() names a status.
 *  - Lattice arrays are flat, x fastest: site = x + nx*(y + ny*z). Host arrays
 *    passed in are FP64 (fields) or uint8 (node kinds), owned by the caller and
 *    only read during the call. Population arrays are planes: f[p*N + site],
 *    in the velocity order reported by elbm_velocity_set_of(params.velset).
 *  - The handle owns every byte of device memory it uses (one arena, plus
 *    the export scratch of elbm_fields); elbm_free releases it. Work is
 *    issued on the caller's CUDA stream (params.cuda_stream, NULL = the
 *    legacy default stream).
 *  - Invalid parameters return ELBM_E_INVAL and allocate nothing.
 */
#ifndef ELBM_H
#define ELBM_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct elbm_handle elbm_handle;

typedef enum {
    ELBM_OK = 0,
    ELBM_W_POISSON_NOCONV = 1, /* a Poisson solve hit poisson_maxit; last iterate kept */
    ELBM_E_INVAL = -1,         /* invalid argument or parameter set */
    ELBM_E_NOMEM = -2,         /* device or pinned host allocation failed */
    ELBM_E_CUDA = -3,          /* a CUDA runtime call failed */
    ELBM_E_NUMERIC = -4,       /* a non-finite value or rho <= 0 appeared */
    ELBM_E_STATE = -5          /* request not possible in this handle's state */
} elbm_status;

/* node kinds of the geometry mask */
enum { ELBM_NODE_FLUID = 0, ELBM_NODE_SOLID = 1, ELBM_NODE_INLET = 2, ELBM_NODE_OUTLET = 3 };
/* flow boundary of a domain face (faces: -x,+x,-y,+y,-z,+z) */
enum { ELBM_FACE_PERIODIC = 0, ELBM_FACE_WALL = 1 };
/* potential boundary of a domain face */
enum { ELBM_PHI_PERIODIC = 0, ELBM_PHI_DIRICHLET = 1, ELBM_PHI_NEUMANN = 2 };
/* free-charge model: none, Eq. (surface-q2), Eq. (surface-q3), D3Q7 transport */
enum { ELBM_CHARGE_NONE = 0, ELBM_CHARGE_CONSERVED = 1, ELBM_CHARGE_XI = 2,
       ELBM_CHARGE_TRANSPORT = 3 };
/* electric force: q E, or Eq. (force_el2) q E + (eps-1)/2 grad|E|^2 (|E|^2 of
 * the fluid face neighbours by central differences; a neighbour that is not
 * fluid takes the site's own |E|^2) */
enum { ELBM_FEL_QE = 0, ELBM_FEL_FULL = 1 };
/* velocity set of the populations: D3Q19 (3-D), or the paper's D2Q9 (Sec. II:
 * rest 4/9, axis 1/9, diagonals 1/36) on a lattice one site thick (nz = 1) */
enum { ELBM_VSET_D3Q19 = 0, ELBM_VSET_D2Q9 = 1 };
/* face permittivity of the Poisson operator: arithmetic or harmonic mean of
 * the two sites (a Dirichlet face couples with the site's own eps) */
enum { ELBM_EPS_FACE_ARITH = 0, ELBM_EPS_FACE_HARMONIC = 1 };
/* Poisson solver: red-black SOR as the paper states it, or geometric
 * multigrid (red-black Gauss-Seidel smoothing) on the same fine operator with
 * the same stopping rule; interior solid nodes are conductors held at
 * phi_solid on the fine level (the coarse levels correct the other nodes);
 * multigrid needs lattice extents that halve at least once (even, and even
 * on periodic axes) and a level of at most 4096 cells */
enum { ELBM_POISSON_SOR = 0, ELBM_POISSON_MG = 1 };
/* relaxation: entropic alpha (Eq. entropic), alpha = 2 (BGK), or the
 * entropic alpha with its Newton iteration started from the learned proposal
 * (elbm_params.mlp; FP32 or BF16 storage with FP32 alpha arithmetic) */
enum { ELBM_ALPHA_ENTROPIC = 0, ELBM_ALPHA_BGK = 1, ELBM_ALPHA_LEARNED = 2 };
/* population storage / arithmetic:
 *   FP64: f stored and computed in FP64, potential in FP64;
 *   FP32: f stored as FP32 deviations d = f - w, FP32 arithmetic;
 *   BF16: f stored in BF16 as f - w rho_ref, rho_ref the density of the
 *         site that wrote the value (kept beside the populations), FP32
 *         arithmetic. */
enum { ELBM_PREC_FP64 = 0, ELBM_PREC_FP32 = 1, ELBM_PREC_BF16 = 2 };
/* arithmetic of the alpha root:
 *   FP64: Newton in FP64;
 *   FP32: Newton in FP32 (the same equation written without cancellation),
 *         then a float-float guard at the sites where FP32 rounding cannot
 *         certify |h(alpha)| <= 1e-10 rho: h'(0) and h re-evaluated as pairs
 *         of FP32 values and at most three more Newton steps;
 *   FP32_FAST: the FP32 Newton root alone (|h| at the FP32 rounding level). */
enum { ELBM_APREC_FP64 = 0, ELBM_APREC_FP32 = 1, ELBM_APREC_FP32_FAST = 2 };

/* selectors for elbm_fields; selected blocks are written back to back in
 * this bit order */
#define ELBM_F_RHO   (1u << 0) /* N: density at the last completed step */
#define ELBM_F_U     (1u << 1) /* 3N: half-step velocity (j + F/2)/rho, xyz per site */
#define ELBM_F_PHI   (1u << 2) /* N: potential */
#define ELBM_F_Q     (1u << 3) /* N: free charge (before neutralisation) */
#define ELBM_F_ALPHA (1u << 4) /* N: entropic alpha */
#define ELBM_F_NU    (1u << 5) /* N: Carreau viscosity */
#define ELBM_F_POP   (1u << 6) /* 19N: populations f(r, t) after streaming */
#define ELBM_F_GPOP  (1u << 7) /* 7N: charge populations g(r, t) (transport mode) */
#define ELBM_F_DIAG  (1u << 8) /* ELBM_NDIAG diagnostics of the last step */

/* diagnostics (FP64): 0 mass, 1-3 momentum sum (j + F/2), 4 total charge,
 * 5 alpha min, 6 alpha max, 7 alpha mean, 8 near-equilibrium shortcuts,
 * 9 no-root fallbacks, 10 clipped at the positivity bound, 11 Poisson
 * sweeps, 12 Poisson relative residual, 13 max |h(alpha)|/rho as evaluated
 * on the device, 14 max |u|, 15 non-finite count, 16 subtracted mean charge,
 * 17 step counter, 18 Poisson sweeps summed over all steps, 19 sites whose
 * alpha took the float-float guard, 20 sites where the guard ended above
 * 1e-10 rho, 21 learned-alpha sites that fell back to the Newton root,
 * 22 scale of the inlet profile set by the adaptive inlet (0 without it),
 * 23 flags of the steps without diagnostics since the previous ones (the
 * earlier steps of a k-step batch graph, or of diag_every > 1): bit 0 a
 * non-finite value or non-positive density, bit 1 a guard failure.
 * 5-12, 14, 16, 19 and 21 are those of the last step; 13 is the maximum
 * over the last step and those steps; 15 and 20 add 1 when bit 0 resp.
 * bit 1 of 23 is set, so that a failure on any step reaches the status
 * elbm_step returns. */
#define ELBM_NDIAG 24

typedef struct elbm_params {
    int nx, ny, nz;              /* lattice; nz = 1 for D2Q9; nx*ny*nz < 2^31 (ELBM_E_INVAL otherwise) */
    int face_bc[6];              /* ELBM_FACE_* ; opposite faces must agree when periodic */
    int phi_bc[6];               /* ELBM_PHI_* ; PERIODIC exactly where face_bc is */
    int phi_axis;                /* axis normal to the electrode planes (0,1,2) */
    int charge_model;            /* ELBM_CHARGE_* */
    int force_el;                /* ELBM_FEL_* */
    int neutralize;              /* subtract the mean free charge before Poisson */
    int poisson_solver;          /* ELBM_POISSON_* */
    int poisson_maxit;           /* cap on SOR sweeps (multigrid: V-cycles) per step */
    int poisson_fixed_sweeps;    /* > 0: exactly this many sweeps (V-cycles), no test */
    int poisson_check_every;     /* convergence test every k sweeps (>= 1); with FP32
                                    potentials a test interval without progress
                                    (residual above 0.97 of the previous test)
                                    ends the solve at its rounding floor */
    int alpha_mode;              /* ELBM_ALPHA_* */
    int precision;               /* ELBM_PREC_* */
    int alpha_precision;         /* ELBM_APREC_* (FP64 precision forces FP64) */
    int store_macro;             /* keep u, alpha, nu planes for elbm_fields */
    int diag_every;              /* diagnostics every k steps (0 = never) */
    int profile;                 /* time each pass with CUDA events (elbm_pass_times) */
    int graph;                   /* run each step as one CUDA graph, the Poisson loop a
                                    device-side while node (needs diag_every = 1);
                                    0: issue from the host, one sync per test */
    int autotune;                /* 1: choose the block shape of the site kernels by
                                    timing the collision at elbm_init (cached per
                                    lattice size for the process); 0: fixed shape */
    double phi_lo, phi_hi;       /* potential on the ghost planes at axis coord -1 and n */
    double phi_solid;            /* potential of interior solid (conductor) nodes */
    double nu0, nu_inf, lambda, n_carreau;  /* Carreau law; n = 1 is Newtonian nu0 */
    double G, Gw, rho0;          /* Shan-Chen couplings, psi = rho0 (1 - exp(-rho/rho0)) */
    double eps_kappa;            /* permittivity eps = 1 + kappa rho / rho0 */
    double sigma_liq, sigma_gas; /* conductivity per phase (transport mode) */
    double Dq;                   /* charge diffusivity (transport mode) */
    double E_ext[3];             /* uniform applied field */
    double Q_b, Q_s, K_d;        /* Eq. (surface-q2) totals and curvature scale */
    double xi_b, xi_s;           /* Eq. (surface-q3) coefficients */
    double theta_width;          /* width of the smoothed Heaviside theta(rho; rho0) */
    double sor_omega, poisson_tol;
    double alpha_eq_tol;         /* max |Delta_p/f_p| below which alpha = 2; must be
                                    >= 2^-18 when the arithmetic is FP32 */
    double rho_in, rho_out;      /* densities of inlet / outlet nodes */
    void *cuda_stream;           /* cudaStream_t of the caller (NULL: default stream) */
    const float *mlp;            /* ELBM_ALPHA_LEARNED: device FP32 parameters of the
                                    proposal (ELBM_MLP_NPARAM values), read once by
                                    elbm_init (kept as BF16 by the handle); else NULL */
    int eps_face;                /* ELBM_EPS_FACE_*: permittivity of a face of the Poisson
                                    operator between two sites (the paper is silent) */
    int carreau_lagged;          /* 0: gdot as the root of Eq. (strain2) each step; 1: Eq.
                                    (strain2) with tau from the previous step's nu ("a slow
                                    variation of nu over the time step", Sec. II B), no root */
    double alpha_h_tol;          /* H-error target |h(alpha)|/rho that the FP32 root
                                    certifies (float-float guard), 0 = 1e-10; below
                                    the guard's resolution (~1e-11) sites end as
                                    guard failures (diag 20); ignored in FP64 */
    int velset;                  /* ELBM_VSET_* (0 = D3Q19). D2Q9 needs nz = 1 and phi_axis
                                    0 or 1; the z faces take no part (no link crosses them,
                                    the potential has no z flux: face_bc[4..5] and
                                    phi_bc[4..5] only pass the checks every set makes,
                                    E_ext[2] must be 0). It runs
                                    FP64 or FP32 populations with the FP64 or the guarded
                                    FP32 root, the paper's charge models (not transport) and
                                    SOR; other choices return ELBM_E_INVAL */
} elbm_params;

/* Initial state, all host arrays of N = nx*ny*nz sites (caller-owned):
 *   mask  uint8 node kinds (NULL = all fluid);
 *   rho0  FP64 initial density (required);
 *   u0    FP64 3N initial velocity, xyz per site (NULL = at rest);
 *   q0    FP64 initial free charge, transport mode (NULL = 0);
 *   u_in  FP64 3N inlet velocity, read at inlet nodes (NULL = 0);
 *   f0    FP64 19N populations f(r, 0) overriding the equilibrium start
 *         (NULL = f^eq(rho0, u0), Eq. 2);
 *   inlet_region  uint8 N (NULL = the inlet profile stays as given): the
 *         adaptive inlet of the jet (Sec. III B). After the collision of each
 *         step, the mean over the fluid sites with inlet_region != 0 of the
 *         half-step velocity along d (the direction of the summed initial
 *         inlet velocities), over the initial profile's own mean along d,
 *         rescales the initial inlet velocities; the next step pulls
 *         f^eq(rho_in, rescaled u_in) from the inlet nodes. Needs u_in with a
 *         nonzero mean and at least one fluid region site (ELBM_E_INVAL). */
typedef struct elbm_init_fields {
    const unsigned char *mask;
    const double *rho0, *u0, *q0, *u_in, *f0;
    const unsigned char *inlet_region;
} elbm_init_fields;

/* Validate the parameters, allocate the device state, build f(r, 0) (and
 * g(r, 0) = w_i q0 (1 + c_i.u0/c_s^2) in transport mode), set phi = 0.
 * n_instances must be 1. On success *out owns the new handle. */
elbm_status elbm_init(const elbm_params *p, const elbm_init_fields *init, int n_instances,
                      elbm_handle **out);

/* Advance nsteps >= 0 time steps on the handle's stream. Returns after the
 * work is done; ELBM_E_NUMERIC if a non-finite value or rho <= 0 appeared,
 * ELBM_W_POISSON_NOCONV if a Poisson solve hit its cap. */
elbm_status elbm_step(elbm_handle *h, int nsteps);

/* Copy the selected fields (ELBM_F_* bits) to the caller's host buffer out of
 * out_len doubles, blocks back to back in bit order, converted to FP64.
 * U, ALPHA and NU need store_macro = 1 (else ELBM_E_STATE); GPOP needs
 * transport mode. ELBM_E_INVAL if out_len is too small. After a step run as
 * a CUDA graph (alone or in a batch) DIAG comes from a pinned-memory copy
 * that the graph made, without touching the device; the FP64 conversion of
 * the other fields goes through a device scratch buffer that the handle
 * keeps (grown on demand, freed by elbm_free). */
elbm_status elbm_fields(elbm_handle *h, unsigned mask, double *out, size_t out_len);

/* Number of doubles elbm_fields writes for this selector (0 on error). */
size_t elbm_fields_size(const elbm_handle *h, unsigned mask);

/* Per-pass device time accumulated since elbm_init when params.profile = 1,
 * measured with CUDA events on the handle's stream around each pass:
 * out[0] moments + charge ms, out[1] Poisson ms, out[2] collision ms,
 * out[3] reductions ms, out[4] steps timed, out[5] collision launches,
 * out[6] Poisson sweeps, out[7] kernel launches of all passes.
 * Writes min(n, 8) values; ELBM_E_STATE when profiling is off. Not part of
 * the paper's method: instrumentation for measuring the method's kernels. */
elbm_status elbm_pass_times(const elbm_handle *h, double *out, int n);

/* elbm_batch_create flags */
#define ELBM_BATCH_PIPELINE 1 /* instances at odd positions run half a step ahead */
#define ELBM_BATCH_SPAN(k) ((k) << 8) /* graphs of k steps (1..16) for elbm_step(batch, >= k) */

/* Batched lattices (not in the paper: an execution form). One batch handle
 * advances n existing instance handles (each made by elbm_init, with
 * diag_every = 1 and profile = 0) by one CUDA graph launch per step: each
 * instance's whole step, its Poisson loop a device-side while node of its
 * own, is a parallel branch of that graph, so instances of uneven size and
 * uneven Poisson work run side by side.
 *   inst   array of n distinct instance handles (not batches); the batch
 *          keeps the pointers: free the batch before its instances, and step
 *          the instances only through the batch while it exists (elbm_step
 *          on the batch returns ELBM_E_STATE if one was stepped alone);
 *   flags  0, or ELBM_BATCH_PIPELINE: each graph launch runs the instances
 *          at odd positions half a step ahead (their collision of the step,
 *          then the moments and potential solve of the next), so that the
 *          latency-bound potential solves of one half overlap the collisions
 *          of the other. The populations and the step counter of every
 *          instance are as without the flag; an instance running ahead holds
 *          the density, charge and potential of the populations it stores
 *          (one step later than an instance not ahead). Its first moments
 *          and solve run once here. After the batch is freed, such an
 *          instance stepped alone repeats that solve (warm-started);
 *          | ELBM_BATCH_SPAN(k), k in 1..16: besides the one-step graphs,
 *          graphs of k consecutive steps, each instance's k steps one chain
 *          of its branch: elbm_step(batch, n) launches n / k of them and the
 *          rest one step at a time. The branches meet once per k steps
 *          instead of every step, so one instance's latency-bound solves
 *          overlap the others' collisions across step boundaries; every
 *          instance runs the same kernels in the same order (bit for bit
 *          the populations and fields of one-step launches), except that
 *          the diagnostics (ELBM_F_DIAG) are formed on the last of the k
 *          steps only;
 *   stream cudaStream_t on which elbm_step(batch) launches the graphs.
 * elbm_step(batch, k) advances every instance k steps and returns the worst
 * status of the instances (non-finite state, Poisson non-convergence; the
 * non-finite count is that of the last step, a NaN persisting);
 * elbm_fields and elbm_pass_times on a batch return ELBM_E_STATE (read each
 * instance); elbm_free(batch) frees the batch only. */
elbm_status elbm_batch_create(elbm_handle *const *inst, int n, int flags, void *stream, elbm_handle **out);

/* The entropic alpha of Eq. (entropic) for n independent sites outside a
 * simulation: the root the collision step computes, for checking its H-error
 * against an FP64 evaluation and for harvesting (f, alpha) pairs. Per site,
 * from FP32 deviations d_p = f_p - w_p (FP32 arithmetic, in the order the
 * FP32 collision uses): rho = 1 + sum d, u = sum d c / rho,
 * Delta_p = w_p (sum d + rho P_p(u)) - d_p with P_p the velocity polynomial
 * of Eq. (2) (formed so that sum_p Delta_p = 0 as for the exact Delta: sum d
 * compensated, w_p sum d - d_p in one rounding, the residual taken off
 * Delta_0), f_p = w_p + d_p rounded to FP32.
 *   d       device FP32 deviations, planes d[p*n + i], p = 0..18;
 *   n       number of sites (0: nothing is enqueued);
 *   aprec   ELBM_APREC_* arithmetic of the root;
 *   eq_tol  near-equilibrium shortcut (alpha = 2) when max|Delta/f| < eq_tol;
 *           >= 2^-18 for the FP32 modes;
 *   mlp     NULL: Newton from the moment-series start; else device FP32
 *           parameters of the learned proposal (ELBM_MLP_NPARAM values, see
 *           elbm_mlp_forward): Newton starts from alpha_c + S^3 o(X); FP32
 *           modes only;
 *   alpha   device FP64 out [n]: the root (high + low part of a guarded root);
 *   herr    device FP32 out [n] or NULL: |h(alpha)|/rho as the method
 *           reports it (evaluated, or the FP32 rounding bound);
 *   status  device int32 out [n] or NULL: 0 root, 1 shortcut, 2 no root
 *           (alpha = 2), 3 clipped at the positivity bound, 4 guard ended
 *           above 1e-10 rho, 5 root after more than one FP32 evaluation of h
 *           (with a learned proposal: the lane fell back to the full Newton
 *           iteration);
 *   delta   device FP32 out [19*n] or NULL: the Delta_p planes used;
 *   stream  cudaStream_t (NULL: legacy default stream).
 * Buffers are the caller's; returns after enqueueing (ELBM_E_INVAL on a
 * bad argument, nothing enqueued). */
elbm_status elbm_alpha_eval(const float *d, long long n, int aprec, double eq_tol, const float *mlp,
                            double *alpha, float *herr, int *status, float *delta, void *stream);

/* ---- learned alpha proposal (not in the paper: an addition that starts the
 * Newton iteration of Eq. (entropic); the root and its H-error stay the
 * method's) ----
 * Features of a site (populations f_p, Delta_p = f^eq_p - f_p), x_p =
 * Delta_p/f_p, S = max|x_p|: X = (x_0/S .. x_18/S, (log2 S + 9)/8). Network
 * o(X) = W3 . gelu(W2 gelu(W1 X + b1) + b2) + b3, 20 -> 64 -> 64 -> 1, gelu in
 * the tanh form; proposal alpha = alpha_c + S^3 o where S >= 2^-5 (else
 * alpha_c), alpha_c the moment-series start (root of h(a)/a truncated after
 * a^3 M4/12, M_k = sum f x^k; error O(S^3)). Parameters: one FP32 vector of
 * ELBM_MLP_NPARAM values, W1 (64 x 20, row-major out x in), b1 (64), W2
 * (64 x 64), b2 (64), W3 (64), b3 (1). Sample arrays are feature-major:
 * X[j*n + i]. All pointers are device memory owned by the caller; calls
 * return after enqueueing on `stream`; bad arguments give ELBM_E_INVAL with
 * nothing enqueued. */
#define ELBM_MLP_NIN 20
#define ELBM_MLP_NPARAM 5569
enum { ELBM_MLP_FP32 = 0, ELBM_MLP_BF16_TC = 1 };
/* features of n sites from FP32 deviations d[p*n + i] (as elbm_alpha_eval
 * computes Delta): X out [20*n], S out [n] or NULL */
elbm_status elbm_alpha_features(const float *d, long long n, float *X, float *S, void *stream);
/* training pairs from FP32 deviations: X out [20*n] (features), y out [n] =
 * (alpha* - alpha_c)/S^3 clipped to [-8, 8] with alpha* the guarded FP32 root
 * (|h| <= 1e-10 rho), keep out [n] = 1 for a root with S >= 2^-5 (else 0,
 * y = 0); eq_tol >= 2^-18 as for elbm_alpha_eval */
elbm_status elbm_alpha_harvest(const float *d, long long n, double eq_tol, float *X, float *y, int *keep,
                               void *stream);
/* o[i] = network output for sample i: ELBM_MLP_FP32 (training arithmetic,
 * CUDA cores) or ELBM_MLP_BF16_TC (BF16 operands and FP32 accumulation on
 * the tensor cores, as the learned proposal runs) */
elbm_status elbm_mlp_forward(const float *X, long long n, const float *theta, int arith, float *o, void *stream);
/* floats of workspace elbm_mlp_grad / elbm_mlp_train need for a batch */
long long elbm_mlp_workspace_floats(long long batch);
/* gradient of the mean squared error mean_i (o(X_i) - y_i)^2 over all n
 * samples (FP32 forward and analytic backward; deterministic reduction):
 * grad out [ELBM_MLP_NPARAM], loss out [1] or NULL, work of
 * elbm_mlp_workspace_floats(n) floats */
elbm_status elbm_mlp_grad(const float *X, const float *y, long long n, const float *theta, float *grad, float *loss,
                          float *work, void *stream);
/* one Adam step (Kingma & Ba 2015) at step t >= 1: theta, m, v updated in place */
elbm_status elbm_mlp_adam(float *theta, const float *grad, float *m, float *v, int t, float lr, float beta1,
                          float beta2, float eps, void *stream);
/* `steps` minibatch Adam steps (beta 0.9 / 0.999, eps 1e-8), steps t0+1 ..
 * t0+steps; minibatch k draws `batch` samples with replacement, sample i at
 * splitmix64(seed + (t0 + k) * batch + i) mod n (seed != 0); loss_hist out
 * [steps] (minibatch MSE before each step) or NULL; work of
 * elbm_mlp_workspace_floats(batch) floats */
elbm_status elbm_mlp_train(const float *X, const float *y, long long n, float *theta, float *m, float *v, int t0,
                           int steps, long long batch, float lr, unsigned long long seed, float *loss_hist, float *work,
                           void *stream);

/* Allocation-free density and mass of a population array. The paper has no
 * counterpart: this serves callers that may not allocate device memory
 * (code running during CUDA stream capture, hosts that give the device to
 * their own memory pool, latency-bound loops that forbid allocator calls).
 *   f      device FP64 populations, planes f[p*n_sites + site], p = 0..18 (the
 *          layout elbm_fields(ELBM_F_POP) returns);
 *   mask   device uint8 node kinds, or NULL for all fluid;
 *   rho    device FP64 out: sum_p f_p at fluid sites, 0 elsewhere;
 *   mass   device FP64 out (one value): sum of rho;
 *   stream cudaStream_t (NULL: the legacy default stream).
 * All pointers are the caller's; nothing is allocated or freed. Scratch is a
 * fixed device array of ELBM_NOALLOC_MAX_BLOCKS doubles inside the library,
 * held by every GPU that loads it until the process exits, so
 * n_sites <= ELBM_NOALLOC_MAX_SITES (else ELBM_E_INVAL). The first call on a
 * device looks up that array's device address (cudaGetSymbolAddress); make
 * the first call on each device before any stream capture. The address is
 * kept for the life of the device's primary context: after a
 * cudaDeviceReset the entry point must not be called again in that process.
 * A CUDA error left pending on the calling thread by earlier work is cleared,
 * not reported as this call's. Every call uses
 * the same scratch and leaves its contents behind (each call overwrites the
 * slots it reads, so nothing needs clearing); calls whose kernels overlap on
 * the GPU (several streams at once) race on it and must be serialised by the
 * caller. Returns after enqueueing the work on `stream`. */
#define ELBM_NOALLOC_MAX_BLOCKS 16384
#define ELBM_NOALLOC_MAX_SITES (ELBM_NOALLOC_MAX_BLOCKS * 1024LL)
elbm_status elbm_density_noalloc(const double *f, const unsigned char *mask, long long n_sites,
                                 double *rho, double *mass, void *stream);

/* Release the handle and its device memory. NULL is a no-op. */
void elbm_free(elbm_handle *h);

/* Static text for a status code. */
const char *elbm_strerror(int status);

/* The D3Q19 velocity set of the library (host call, no GPU needed):
 * c[3*p + a] and w[p] for p = 0..18; returns 19. */
int elbm_velocity_set(int *c, double *w);

/* The velocity set `velset` (ELBM_VSET_*; host call, no GPU needed): c[3*p + a]
 * and w[p] for p = 0..Q-1 (either pointer may be NULL); returns Q (19 or 9),
 * or ELBM_E_INVAL for an unknown set. */
int elbm_velocity_set_of(int velset, int *c, double *w);

#ifdef __cplusplus
}
#endif
#endif /* ELBM_H */
