/*
 * elbm_oracle.h -- plain FP64 CPU oracle of the charged entropic lattice
 * Boltzmann (ELBM) time step of Lauricella et al., "Entropic Lattice Boltzmann
 * Model for Charged Leaky Dielectric Multiphase Fluids in Electrified Jets"
 * (arXiv:1612.05404).
 *
 * TEST INFRASTRUCTURE. Only the test suite, the smoke check and the CPU
 * baseline leg of the benchmark load this library. The product path (the CUDA
 * library under paper_1612_05404_gb300/) never includes, links or calls it,
 * and this oracle includes nothing from the product path.
 *
 * Every array is a flat FP64 (or uint8) array over the lattice with x fastest:
 * site index = x + nx*(y + ny*z). Populations are stored as planes:
 * f[p*N + site]. 2-D problems use dim = 2, nz = 1 and the D2Q9 set; 3-D
 * problems use D3Q19.
 */
#ifndef ELBM_ORACLE_H
#define ELBM_ORACLE_H

#ifdef __cplusplus
extern "C" {
#endif

/* node kinds in the geometry mask */
enum { ORC_FLUID = 0, ORC_SOLID = 1, ORC_INLET = 2, ORC_OUTLET = 3 };
/* flow boundary per domain face (-x,+x,-y,+y,-z,+z) */
enum { ORC_FACE_PERIODIC = 0, ORC_FACE_WALL = 1 };
/* potential boundary per domain face */
enum { ORC_PHI_PERIODIC = 0, ORC_PHI_DIRICHLET = 1, ORC_PHI_NEUMANN = 2 };
/* charge models */
enum { ORC_CHARGE_NONE = 0, ORC_CHARGE_CONSERVED = 1, ORC_CHARGE_XI = 2,
       ORC_CHARGE_TRANSPORT = 3 };
/* electric force */
enum { ORC_FEL_QE = 0, ORC_FEL_FULL = 1 };
/* relaxation */
enum { ORC_ALPHA_ENTROPIC = 0, ORC_ALPHA_BGK = 1 };
/* face permittivity: arithmetic or harmonic mean of the two sites */
enum { ORC_EPS_FACE_ARITH = 0, ORC_EPS_FACE_HARMONIC = 1 };
/* alpha status codes */
enum { ORC_A_ROOT = 0, ORC_A_SHORTCUT = 1, ORC_A_NOROOT = 2, ORC_A_CLIPPED = 3 };

typedef struct orc_params {
    int dim;                 /* 2 (D2Q9) or 3 (D3Q19) */
    int nx, ny, nz;
    int face_bc[6];          /* ORC_FACE_* per face -x,+x,-y,+y,-z,+z */
    int phi_bc[6];           /* ORC_PHI_* per face */
    int phi_axis;            /* axis normal to the electrodes (0,1,2) */
    int charge_model;        /* ORC_CHARGE_* */
    int force_el;            /* ORC_FEL_* */
    int neutralize;          /* 1: subtract the mean charge before Poisson */
    int poisson_maxit;       /* cap on SOR sweeps */
    int poisson_fixed_sweeps;/* >0: run exactly this many sweeps, no test */
    int alpha_mode;          /* ORC_ALPHA_* */
    int eps_face;            /* ORC_EPS_FACE_*: face permittivity of the Poisson operator */
    int carreau_lagged;      /* 1: gdot from the previous step's nu (no root of Eq. strain2) */
    int pad1;
    double phi_lo, phi_hi;   /* ghost-plane potentials at axis coord -1, n */
    double phi_solid;        /* potential of interior solid (conductor) nodes */
    double nu0, nu_inf, lambda, n_carreau;   /* Carreau law, Eq. (carreau) */
    double G, Gw, rho0;      /* Shan-Chen couplings and psi scale, Eq. (sc) */
    double eps_kappa;        /* eps = 1 + kappa*rho/rho0 */
    double sigma_liq, sigma_gas, Dq;          /* transport-mode charge */
    double E_ext[3];         /* uniform applied field */
    double Q_b, Q_s, K_d, xi_b, xi_s, theta_width;
    double sor_omega, poisson_tol;
    double alpha_eq_tol;     /* max|x_p| below which alpha = 2 */
    double rho_in, rho_out;  /* densities of inlet / outlet nodes */
} orc_params;

/* number of diagnostics written by orc_step */
#define ORC_NDIAG 20

/* threads of the site-parallel loops (OpenMP; n <= 0 keeps the setting);
 * returns the number in use. Results are the same for any number. */
int orc_set_threads(int n);

/* ---------------- per-site building blocks ---------------- */
int    orc_Q(int dim);
void   orc_lattice(int dim, int *c /* Q*3 */, double *w /* Q */, double *cs2);
void   orc_feq(int dim, double rho, const double *u, double *feq);
double orc_H(int dim, const double *f);
double orc_h(int dim, const double *f, const double *delta, double alpha);
double orc_h_prime0(int dim, const double *f, const double *delta);
int    orc_alpha(int dim, const double *f, const double *delta, double eq_tol,
                 double *alpha);
double orc_alpha_bisect(int dim, const double *f, const double *delta);
double orc_spectral_norm(int dim, const double *Pi /* 3x3 row-major */);
int    orc_carreau(const orc_params *p, double Pi_norm, double alpha, double rho,
                   double *gdot, double *nu);
void   orc_carreau_lagged(const orc_params *p, double Pi_norm, double alpha, double rho,
                          double nu_prev, double *gdot, double *nu);

/* ---------------- field-level building blocks ---------------- */
void orc_sc_force(const orc_params *p, const unsigned char *mask,
                  const double *rho, double *F /* 3N */);
void orc_charge_field(const orc_params *p, const unsigned char *mask,
                      const double *rho, double *q, double *K, double *sums);
int  orc_poisson_solve(const orc_params *p, const unsigned char *mask,
                       const double *rho, const double *qn, double qmean,
                       double *phi, int *iters, double *resid);
int  orc_poisson_system(const orc_params *p, const unsigned char *mask,
                        const double *rho, const double *qn,
                        double *A, double *b, long *index, int *n_unknown);
void orc_efield(const orc_params *p, const unsigned char *mask,
                const double *phi, double *E /* 3N */);

void orc_stream(const orc_params *p, const unsigned char *mask, const double *u_in,
                const double *rho, const double *fs, const double *gs,
                double *f_out, double *g_out);

/* ---------------- whole step ---------------- */
int orc_init(const orc_params *p, const unsigned char *mask,
             const double *rho0_field, const double *u0_field,
             const double *q0_field, const double *u_in, double *f, double *g,
             double *phi);
void orc_apply_io(const orc_params *p, const unsigned char *mask, const double *u_in,
                  double *f);
/* u_in: inlet velocities (3 per site, read at inlet nodes); with region
 * (uint8 per site: the nozzle sites whose mean velocity rescales the inlet
 * profile) and u_in0 (the initial inlet velocities) not NULL, u_in is
 * rewritten each step (the adaptive inlet); else it is only read. */
int orc_step(const orc_params *p, const unsigned char *mask,
             double *u_in, const unsigned char *region, const double *u_in0,
             double *f, double *g, double *phi,
             double *rho, double *u, double *q, double *alpha_out,
             double *nu_out, double *diag);

#ifdef __cplusplus
}
#endif
#endif
