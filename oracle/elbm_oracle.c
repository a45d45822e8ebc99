/*
 * elbm_oracle.c -- plain, slow, FP64 CPU oracle of the charged entropic
 * lattice Boltzmann step of Lauricella et al. (arXiv:1612.05404), Sec. II.
 *
 * TEST INFRASTRUCTURE. Loaded only by the test suite, the smoke check and the
 * benchmark's CPU-baseline leg. It shares no code, header, table or helper
 * with the CUDA library; the velocity tables below are written out here from
 * the definitions of the D2Q9 / D3Q19 / D3Q7 sets.
 *
 * The code follows the paper's statement of the model, one step of the
 * summary in Sec. II C at a time, with plain loops over sites and
 * populations. Where the paper is silent the reading used is stated at the
 * point of use. Compiled without fast-math and without FP contraction.
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif
#include "elbm_oracle.h"

/* ------------------------------------------------------------------------
 * Threads. Loops whose sites are independent (each iteration writes only its
 * own site's outputs) run in parallel over sites when compiled with OpenMP;
 * every global sum is taken serially in site order afterwards, so the
 * results are bit for bit those of one thread.
 * ---------------------------------------------------------------------- */
int orc_set_threads(int n)
{
#ifdef _OPENMP
    if (n > 0) omp_set_num_threads(n);
    return omp_get_max_threads();
#else
    (void)n;
    return 1;
#endif
}

/* ------------------------------------------------------------------------
 * Velocity sets. D2Q9 (Sec. II, Eq. 2 and the text after it): rest weight
 * 4/9, axis 1/9, diagonal 1/36, c_s^2 = 1/3. D3Q19 (the 3-D set with the
 * same c_s^2): rest 1/3, the 6 axis links 1/18, the 12 face diagonals 1/36.
 * D3Q7 for the charge advection-diffusion: rest 1/4, axis 1/8, c_s^2 = 1/4.
 * ---------------------------------------------------------------------- */
static const int C9[9][3] = {
    {0, 0, 0}, {1, 0, 0}, {-1, 0, 0}, {0, 1, 0}, {0, -1, 0},
    {1, 1, 0}, {-1, -1, 0}, {1, -1, 0}, {-1, 1, 0}};
static const double W9[9] = {4.0 / 9, 1.0 / 9, 1.0 / 9, 1.0 / 9, 1.0 / 9,
                             1.0 / 36, 1.0 / 36, 1.0 / 36, 1.0 / 36};
static const int C19[19][3] = {
    {0, 0, 0},
    {1, 0, 0}, {-1, 0, 0}, {0, 1, 0}, {0, -1, 0}, {0, 0, 1}, {0, 0, -1},
    {1, 1, 0}, {-1, -1, 0}, {1, -1, 0}, {-1, 1, 0},
    {1, 0, 1}, {-1, 0, -1}, {1, 0, -1}, {-1, 0, 1},
    {0, 1, 1}, {0, -1, -1}, {0, 1, -1}, {0, -1, 1}};
static const double W19[19] = {
    1.0 / 3,
    1.0 / 18, 1.0 / 18, 1.0 / 18, 1.0 / 18, 1.0 / 18, 1.0 / 18,
    1.0 / 36, 1.0 / 36, 1.0 / 36, 1.0 / 36, 1.0 / 36, 1.0 / 36,
    1.0 / 36, 1.0 / 36, 1.0 / 36, 1.0 / 36, 1.0 / 36, 1.0 / 36};
static const int C7[7][3] = {
    {0, 0, 0}, {1, 0, 0}, {-1, 0, 0}, {0, 1, 0}, {0, -1, 0}, {0, 0, 1}, {0, 0, -1}};
static const double W7[7] = {0.25, 0.125, 0.125, 0.125, 0.125, 0.125, 0.125};
static const double CS2 = 1.0 / 3.0;
static const double CS2_Q = 0.25;

typedef struct {
    const orc_params *p;
    int dim, nx, ny, nz, Q;
    long N;
    int c[19][3];
    double w[19];
    int opp[19];
} ctx_t;

int orc_Q(int dim) { return dim == 2 ? 9 : 19; }

static void lattice_tables(int dim, int c[19][3], double w[19], int opp[19])
{
    int Q = orc_Q(dim);
    for (int p = 0; p < Q; p++) {
        for (int a = 0; a < 3; a++) c[p][a] = (dim == 2) ? C9[p][a] : C19[p][a];
        w[p] = (dim == 2) ? W9[p] : W19[p];
    }
    /* opposite direction: the q with c_q = -c_p */
    for (int p = 0; p < Q; p++)
        for (int q = 0; q < Q; q++)
            if (c[q][0] == -c[p][0] && c[q][1] == -c[p][1] && c[q][2] == -c[p][2])
                opp[p] = q;
}

void orc_lattice(int dim, int *c, double *w, double *cs2)
{
    int cc[19][3], opp[19];
    double ww[19];
    lattice_tables(dim, cc, ww, opp);
    for (int p = 0; p < orc_Q(dim); p++) {
        for (int a = 0; a < 3; a++) c[3 * p + a] = cc[p][a];
        w[p] = ww[p];
    }
    *cs2 = CS2;
}

static void ctx_init(ctx_t *C, const orc_params *p)
{
    C->p = p;
    C->dim = p->dim;
    C->nx = p->nx;
    C->ny = p->ny;
    C->nz = p->nz;
    C->Q = orc_Q(p->dim);
    C->N = (long)p->nx * p->ny * p->nz;
    lattice_tables(p->dim, C->c, C->w, C->opp);
}

/* Site reached from (x,y,z) by (dx,dy,dz). Periodic faces wrap. Returns -1
 * when the move leaves the domain through a non-periodic face; *face is then
 * the face index (0..5 = -x,+x,-y,+y,-z,+z). */
static long nbr(const ctx_t *C, int x, int y, int z, int dx, int dy, int dz, int *face)
{
    int n[3] = {C->nx, C->ny, C->nz};
    int r[3] = {x + dx, y + dy, z + dz};
    *face = -1;
    for (int a = 0; a < 3; a++) {
        if (r[a] < 0) {
            if (C->p->face_bc[2 * a] == ORC_FACE_PERIODIC) r[a] += n[a];
            else { *face = 2 * a; return -1; }
        } else if (r[a] >= n[a]) {
            if (C->p->face_bc[2 * a + 1] == ORC_FACE_PERIODIC) r[a] -= n[a];
            else { *face = 2 * a + 1; return -1; }
        }
    }
    return r[0] + (long)n[0] * (r[1] + (long)n[1] * r[2]);
}

static void coords(const ctx_t *C, long s, int *x, int *y, int *z)
{
    *x = (int)(s % C->nx);
    *y = (int)((s / C->nx) % C->ny);
    *z = (int)(s / ((long)C->nx * C->ny));
}

/* Material laws of Sec. II. */
static double psi_of(const orc_params *p, double rho)   /* after Eq. (sc) */
{
    return p->rho0 * (1.0 - exp(-rho / p->rho0));
}
static double theta_of(const orc_params *p, double rho) /* smoothed Heaviside */
{
    return 0.5 * (1.0 + tanh((rho - p->rho0) / p->theta_width));
}
static double eps_of(const orc_params *p, double rho)   /* eps = 1 + kappa rho/rho0 */
{
    return 1.0 + p->eps_kappa * rho / p->rho0;
}
static double sigma_of(const orc_params *p, double rho) /* conductivity per phase */
{
    return p->sigma_gas + (p->sigma_liq - p->sigma_gas) * theta_of(p, rho);
}
/* permittivity of the face between two sites: the arithmetic mean (the
 * default reading), or the harmonic mean (the series value of two half-cells) */
static double eps_face(const orc_params *p, double ea, double eb)
{
    if (p->eps_face == ORC_EPS_FACE_HARMONIC) return 2.0 * ea * eb / (ea + eb);
    return 0.5 * (ea + eb);
}

/* ------------------------------------------------------------------------
 * Eq. (2): second-order Mach expansion of the equilibrium.
 * ---------------------------------------------------------------------- */
void orc_feq(int dim, double rho, const double *u, double *feq)
{
    int c[19][3], opp[19];
    double w[19];
    lattice_tables(dim, c, w, opp);
    double uz = (dim == 2) ? 0.0 : u[2];
    double usq = u[0] * u[0] + u[1] * u[1] + uz * uz;
    for (int p = 0; p < orc_Q(dim); p++) {
        double cu = c[p][0] * u[0] + c[p][1] * u[1] + c[p][2] * uz;
        feq[p] = w[p] * rho *
                 (1.0 + cu / CS2 + (cu * cu - CS2 * usq) / (2.0 * CS2 * CS2));
    }
}

/* Eq. (H): H(f) = sum_p f_p ln(f_p / w_p). */
double orc_H(int dim, const double *f)
{
    int c[19][3], opp[19];
    double w[19];
    lattice_tables(dim, c, w, opp);
    double s = 0.0;
    for (int p = 0; p < orc_Q(dim); p++) s += f[p] * log(f[p] / w[p]);
    return s;
}

/* h(alpha) = H(f + alpha*Delta) - H(f), Eq. (entropic), written as
 *   sum_p [ (f_p + a D_p) log1p(a D_p / f_p) + a D_p ln(f_p / w_p) ],
 * which is the same quantity rearranged exactly (no use of sum D = 0) and
 * free of the cancellation between the two H values near the root.
 * A population driven to exactly zero contributes its limit 0 ln 0 = 0. */
double orc_h(int dim, const double *f, const double *d, double a)
{
    int c[19][3], opp[19];
    double w[19];
    lattice_tables(dim, c, w, opp);
    double s = 0.0;
    for (int p = 0; p < orc_Q(dim); p++) {
        double y = a * d[p] / f[p];
        double t = (1.0 + y <= 0.0) ? 0.0 : (f[p] + a * d[p]) * log1p(y);
        s += t + a * d[p] * log(f[p] / w[p]);
    }
    return s;
}

/* dh/dalpha = sum_p D_p [1 + ln(f_p/w_p) + log1p(a D_p/f_p)]. */
static double h_prime(int dim, const double *f, const double *d, double a)
{
    int c[19][3], opp[19];
    double w[19];
    lattice_tables(dim, c, w, opp);
    double s = 0.0;
    for (int p = 0; p < orc_Q(dim); p++)
        s += d[p] * (1.0 + log(f[p] / w[p]) + log1p(a * d[p] / f[p]));
    return s;
}

double orc_h_prime0(int dim, const double *f, const double *d)
{
    return h_prime(dim, f, d, 0.0);
}

/* Bracket [lo, hi] around the nontrivial root of h, or a status when there
 * is none. h(0) = 0 and h is convex in alpha (h'' = sum D^2/(f + a D) > 0),
 * so with h'(0) < 0 there is exactly one root in (0, alpha_max], where
 * alpha_max keeps every f_p + alpha D_p non-negative. */
static int alpha_bracket(int dim, const double *f, const double *d, double eq_tol,
                         double *lo, double *hi, double *alpha)
{
    int Q = orc_Q(dim);
    double maxabs = 0.0, amax = INFINITY;
    for (int p = 0; p < Q; p++) {
        double x = d[p] / f[p];
        if (fabs(x) > maxabs) maxabs = fabs(x);
        if (d[p] < 0.0 && -f[p] / d[p] < amax) amax = -f[p] / d[p];
    }
    /* reading: at (numerical) equilibrium the collision is plain BGK */
    if (!(maxabs >= eq_tol)) { *alpha = 2.0; return ORC_A_SHORTCUT; }
    /* reading: with h'(0) >= 0 no positive alpha keeps H from rising;
     * fall back to the BGK value alpha = 2 */
    if (h_prime(dim, f, d, 0.0) >= 0.0) { *alpha = 2.0; return ORC_A_NOROOT; }
    double h_hi;
    if (isinf(amax)) {
        *hi = 4.0;
        while ((h_hi = orc_h(dim, f, d, *hi)) < 0.0 && *hi < 1e30) *hi *= 2.0;
    } else {
        *hi = amax * (1.0 - 1e-15);
        h_hi = orc_h(dim, f, d, *hi);
    }
    /* root beyond the positivity limit: clip there */
    if (h_hi < 0.0) { *alpha = *hi; return ORC_A_CLIPPED; }
    *lo = 0.5 * (*hi);
    for (int k = 0; k < 4000 && orc_h(dim, f, d, *lo) >= 0.0; k++) *lo *= 0.5;
    return ORC_A_ROOT;
}

/* Eq. (entropic): the nontrivial root of H(f + alpha (f^eq - f)) = H(f).
 * Safeguarded Newton inside the sign bracket, started at the BGK value 2,
 * run until the update is at rounding level. */
int orc_alpha(int dim, const double *f, const double *d, double eq_tol, double *alpha)
{
    double lo = 0.0, hi = 0.0;
    int st = alpha_bracket(dim, f, d, eq_tol, &lo, &hi, alpha);
    if (st != ORC_A_ROOT) return st;
    double x = 2.0;
    if (!(x > lo && x < hi)) x = 0.5 * (lo + hi);
    for (int it = 0; it < 300; it++) {
        double hx = orc_h(dim, f, d, x);
        if (hx == 0.0) break;
        if (hx < 0.0) lo = x; else hi = x;
        double xn = x - hx / h_prime(dim, f, d, x);
        if (!(xn > lo && xn < hi)) xn = 0.5 * (lo + hi);
        if (fabs(xn - x) <= 4e-16 * fabs(x) || hi - lo <= 4e-16 * hi) { x = xn; break; }
        x = xn;
    }
    *alpha = x;
    return ORC_A_ROOT;
}

/* The same root by plain bisection, to the last representable bit. */
double orc_alpha_bisect(int dim, const double *f, const double *d)
{
    double lo = 0.0, hi = 0.0, a = 0.0;
    int st = alpha_bracket(dim, f, d, 0.0, &lo, &hi, &a);
    if (st != ORC_A_ROOT) return a;
    for (int it = 0; it < 5000; it++) {
        double mid = lo + 0.5 * (hi - lo);
        if (mid <= lo || mid >= hi) break;
        if (orc_h(dim, f, d, mid) < 0.0) lo = mid; else hi = mid;
    }
    return 0.5 * (lo + hi);
}

/* Matrix 2-norm of a symmetric tensor (Sec. II B): the largest |eigenvalue|.
 * Cyclic Jacobi rotations until the off-diagonal part vanishes. */
double orc_spectral_norm(int dim, const double *Pi)
{
    int n = dim;
    double a[3][3];
    for (int i = 0; i < 3; i++)
        for (int j = 0; j < 3; j++) a[i][j] = Pi[3 * i + j];
    for (int sweep = 0; sweep < 100; sweep++) {
        double off = 0.0, diag = 0.0;
        for (int i = 0; i < n; i++) {
            diag += a[i][i] * a[i][i];
            for (int j = i + 1; j < n; j++) off += a[i][j] * a[i][j];
        }
        if (off <= 1e-34 * diag || off == 0.0) break;
        for (int p = 0; p < n; p++)
            for (int q = p + 1; q < n; q++) {
                if (a[p][q] == 0.0) continue;
                double theta = (a[q][q] - a[p][p]) / (2.0 * a[p][q]);
                double t = (theta >= 0.0 ? 1.0 : -1.0) /
                           (fabs(theta) + sqrt(theta * theta + 1.0));
                double cth = 1.0 / sqrt(t * t + 1.0), sth = t * cth;
                /* a <- J^T a J with J the rotation in the (p,q) plane */
                double J[3][3] = {{1, 0, 0}, {0, 1, 0}, {0, 0, 1}}, tmp[3][3];
                J[p][p] = cth; J[q][q] = cth; J[p][q] = sth; J[q][p] = -sth;
                for (int i = 0; i < 3; i++)
                    for (int j = 0; j < 3; j++) {
                        double s = 0.0;
                        for (int k = 0; k < 3; k++) s += a[i][k] * J[k][j];
                        tmp[i][j] = s;
                    }
                for (int i = 0; i < 3; i++)
                    for (int j = 0; j < 3; j++) {
                        double s = 0.0;
                        for (int k = 0; k < 3; k++) s += J[k][i] * tmp[k][j];
                        a[i][j] = s;
                    }
            }
    }
    double m = 0.0;
    for (int i = 0; i < n; i++)
        if (fabs(a[i][i]) > m) m = fabs(a[i][i]);
    return m;
}

/* ------------------------------------------------------------------------
 * Carreau law, Eq. (carreau), and Eq. (beta).
 * ---------------------------------------------------------------------- */
static double nu_carreau(const orc_params *p, double g)
{
    double lg = p->lambda * g;
    return p->nu_inf + (p->nu0 - p->nu_inf) * pow(1.0 + lg * lg, 0.5 * (p->n_carreau - 1.0));
}
static double dnu_carreau(const orc_params *p, double g)
{
    double lg = p->lambda * g;
    return (p->nu0 - p->nu_inf) * (p->n_carreau - 1.0) * p->lambda * p->lambda * g *
           pow(1.0 + lg * lg, 0.5 * (p->n_carreau - 3.0));
}
static double beta_of(double nu) { return CS2 / (2.0 * nu + CS2); }

/* Eq. (strain2): gdot = Pi / (rho tau(gdot) c_s^2) with 1/tau = alpha beta(nu(gdot)).
 * Reading: the root is sought in [A beta(nu0), A beta(nu_inf)], A = Pi alpha/(rho c_s^2),
 * where g(gdot) = gdot - A beta(nu(gdot)) changes sign; safeguarded Newton from
 * the left end of that bracket. */
int orc_carreau(const orc_params *p, double Pn, double alpha, double rho,
                double *gdot, double *nu)
{
    if (p->n_carreau == 1.0 || p->lambda == 0.0 || p->nu0 == p->nu_inf) {
        *nu = p->nu0;
        *gdot = Pn * alpha * beta_of(p->nu0) / (rho * CS2);
        return 0;
    }
    double A = Pn * alpha / (rho * CS2);
    if (A == 0.0) { *gdot = 0.0; *nu = p->nu0; return 0; }
    double lo = A * beta_of(p->nu0), hi = A * beta_of(p->nu_inf);
    double x = lo;
    int it;
    for (it = 0; it < 300; it++) {
        double nux = nu_carreau(p, x);
        double gx = x - A * beta_of(nux);
        if (gx == 0.0) break;
        if (gx < 0.0) lo = x; else hi = x;
        double bp = -2.0 * CS2 / ((2.0 * nux + CS2) * (2.0 * nux + CS2));
        double gp = 1.0 - A * bp * dnu_carreau(p, x);
        double xn = x - gx / gp;
        if (!(xn > lo && xn < hi)) xn = 0.5 * (lo + hi);
        if (fabs(xn - x) <= 4e-16 * fabs(x) || hi - lo <= 4e-16 * hi) { x = xn; break; }
        x = xn;
    }
    *gdot = x;
    *nu = nu_carreau(p, x);
    return it;
}

/* The lagged reading of the same passage ("a slow variation of nu over the
 * time step"): Eq. (strain2) evaluated with tau from the previous step's
 * viscosity, gdot = Pi alpha beta(nu_prev) / (rho c_s^2), no root; then
 * nu = nu(gdot) by Eq. (carreau). A fixed point of this map is the root of
 * Eq. (strain2). */
void orc_carreau_lagged(const orc_params *p, double Pn, double alpha, double rho, double nu_prev,
                        double *gdot, double *nu)
{
    if (p->n_carreau == 1.0 || p->lambda == 0.0 || p->nu0 == p->nu_inf) {
        *nu = p->nu0;
        *gdot = Pn * alpha * beta_of(p->nu0) / (rho * CS2);
        return;
    }
    *gdot = Pn * alpha * beta_of(nu_prev) / (rho * CS2);
    *nu = nu_carreau(p, *gdot);
}

/* ------------------------------------------------------------------------
 * Shan-Chen force, Eq. (sc). Fluid, inlet and outlet neighbours enter the
 * first sum with their own psi; solid nodes and the nodes beyond a wall face
 * enter the wall sum, which (as the equation is printed) carries psi of the
 * site itself.
 * ---------------------------------------------------------------------- */
void orc_sc_force(const orc_params *p, const unsigned char *mask,
                  const double *rho, double *F)
{
    ctx_t C;
    ctx_init(&C, p);
#pragma omp parallel for schedule(static)
    for (long s = 0; s < C.N; s++) {
        F[3 * s] = F[3 * s + 1] = F[3 * s + 2] = 0.0;
        if (mask[s] != ORC_FLUID) continue;
        int x, y, z, face;
        coords(&C, s, &x, &y, &z);
        double ps = psi_of(p, rho[s]);
        double sf[3] = {0, 0, 0}, sw[3] = {0, 0, 0};
        for (int q = 1; q < C.Q; q++) {
            long nb = nbr(&C, x, y, z, C.c[q][0], C.c[q][1], C.c[q][2], &face);
            for (int a = 0; a < 3; a++) {
                if (nb < 0 || mask[nb] == ORC_SOLID) sw[a] += C.w[q] * ps * C.c[q][a];
                else sf[a] += C.w[q] * psi_of(p, rho[nb]) * C.c[q][a];
            }
        }
        for (int a = 0; a < 3; a++) F[3 * s + a] = -p->G * ps * sf[a] - p->Gw * ps * sw[a];
    }
}

/* ------------------------------------------------------------------------
 * Free charge, Eqs. (surface-q2) (conserved) and (surface-q3) (xi form).
 * Readings: gradients use the isotropic lattice stencil
 *   grad X = (1/c_s^2) sum_p w_p X(r + c_p) c_p,
 * with a node that is solid or beyond a wall face taking the value of the
 * site itself; n = grad rho / max(|grad rho|, 1e-12); the mean curvature is
 * K = -div n, the sign that makes a convex liquid drop positive (the paper
 * prints K_max > 0 on the drop's protruding tip); (K/K_d)^(1/4) is taken
 * as max(K,0)^(1/4).
 * ---------------------------------------------------------------------- */
void orc_charge_field(const orc_params *p, const unsigned char *mask,
                      const double *rho, double *q, double *K, double *sums)
{
    ctx_t C;
    ctx_init(&C, p);
    double *grad = calloc(3 * C.N, sizeof(double));
    double *nh = calloc(3 * C.N, sizeof(double));
    double *a = calloc(C.N, sizeof(double));
    double *b = calloc(C.N, sizeof(double));
#pragma omp parallel for schedule(static)
    for (long s = 0; s < C.N; s++) {
        if (mask[s] == ORC_SOLID) continue;
        int x, y, z, face;
        coords(&C, s, &x, &y, &z);
        for (int qq = 1; qq < C.Q; qq++) {
            long nb = nbr(&C, x, y, z, C.c[qq][0], C.c[qq][1], C.c[qq][2], &face);
            double v = (nb < 0 || mask[nb] == ORC_SOLID) ? rho[s] : rho[nb];
            for (int k = 0; k < 3; k++) grad[3 * s + k] += C.w[qq] * v * C.c[qq][k] / CS2;
        }
        double g2 = grad[3 * s] * grad[3 * s] + grad[3 * s + 1] * grad[3 * s + 1] +
                    grad[3 * s + 2] * grad[3 * s + 2];
        double gn = sqrt(g2);
        if (gn < 1e-12) gn = 1e-12;
        for (int k = 0; k < 3; k++) nh[3 * s + k] = grad[3 * s + k] / gn;
    }
#pragma omp parallel for schedule(static)
    for (long s = 0; s < C.N; s++) {
        if (K) K[s] = 0.0;
        if (mask[s] != ORC_FLUID) continue;
        int x, y, z, face;
        coords(&C, s, &x, &y, &z);
        double div = 0.0;
        for (int qq = 1; qq < C.Q; qq++) {
            long nb = nbr(&C, x, y, z, C.c[qq][0], C.c[qq][1], C.c[qq][2], &face);
            long src = (nb < 0 || mask[nb] == ORC_SOLID) ? s : nb;
            for (int k = 0; k < 3; k++) div += C.w[qq] * nh[3 * src + k] * C.c[qq][k] / CS2;
        }
        double Kc = -div;
        if (K) K[s] = Kc;
        double g2 = grad[3 * s] * grad[3 * s] + grad[3 * s + 1] * grad[3 * s + 1] +
                    grad[3 * s + 2] * grad[3 * s + 2];
        double kp = Kc > 0.0 ? Kc : 0.0;
        a[s] = rho[s] * theta_of(p, rho[s]);
        b[s] = g2 * (1.0 + pow(kp / p->K_d, 0.25));
    }
    double Sa = 0.0, Sb = 0.0;
    for (long s = 0; s < C.N; s++) {
        if (mask[s] != ORC_FLUID) continue;
        Sa += a[s];
        Sb += b[s];
    }
#pragma omp parallel for schedule(static)
    for (long s = 0; s < C.N; s++) {
        q[s] = 0.0;
        if (mask[s] != ORC_FLUID) continue;
        if (p->charge_model == ORC_CHARGE_CONSERVED)
            q[s] = (Sa > 0.0 ? p->Q_b * a[s] / Sa : 0.0) + (Sb > 0.0 ? p->Q_s * b[s] / Sb : 0.0);
        else
            q[s] = p->xi_b * a[s] + p->xi_s * b[s];
    }
    if (sums) { sums[0] = Sa; sums[1] = Sb; }
    free(grad); free(nh); free(a); free(b);
}

/* ------------------------------------------------------------------------
 * Potential boundary values. A face normal to phi_axis carries phi_lo (low
 * side) or phi_hi (high side), placed one spacing outside the lattice; the
 * other Dirichlet faces carry the linear profile between them. Interior solid
 * nodes are conductors at phi_solid.
 * ---------------------------------------------------------------------- */
enum { PN_UNKNOWN = 0, PN_DIRICHLET = 1, PN_NONE = 2 };

static double phi_ghost(const ctx_t *C, int face, int x, int y, int z)
{
    const orc_params *p = C->p;
    int axis = face / 2, hi = face & 1;
    if (axis == p->phi_axis) return hi ? p->phi_hi : p->phi_lo;
    int r[3] = {x, y, z}, n[3] = {C->nx, C->ny, C->nz};
    return p->phi_lo + (r[p->phi_axis] + 1.0) * (p->phi_hi - p->phi_lo) / (n[p->phi_axis] + 1.0);
}

/* Neighbour of site s along +-axis for the potential stencil. */
static int pois_nb(const ctx_t *C, const unsigned char *mask, int x, int y, int z,
                   int axis, int sign, long *idx, double *val)
{
    int d[3] = {0, 0, 0}, face;
    d[axis] = sign;
    long nb = nbr(C, x, y, z, d[0], d[1], d[2], &face);
    if (nb < 0) {
        if (C->p->phi_bc[face] == ORC_PHI_DIRICHLET) {
            *val = phi_ghost(C, face, x, y, z);
            return PN_DIRICHLET;
        }
        return PN_NONE;
    }
    if (mask[nb] == ORC_SOLID) { *val = C->p->phi_solid; return PN_DIRICHLET; }
    *idx = nb;
    return PN_UNKNOWN;
}

static int has_dirichlet(const ctx_t *C, const unsigned char *mask)
{
    for (int f = 0; f < 2 * C->dim; f++)
        if (C->p->phi_bc[f] == ORC_PHI_DIRICHLET) return 1;
    for (long s = 0; s < C->N; s++)
        if (mask[s] == ORC_SOLID) return 1;
    return 0;
}

/* Residual r = div(eps grad phi) + qn (7-point / 5-point finite volume with
 * the arithmetic mean of eps on each face) and its reference norm. */
static void pois_residual(const ctx_t *C, const unsigned char *mask, const double *eps,
                          const double *qn, double qmean, const double *phi, double *rn,
                          double *ref, double *t3 /* 3N scratch: per site r^2, q^2, b^2 */)
{
#pragma omp parallel for schedule(static)
    for (long s = 0; s < C->N; s++) {
        t3[3 * s] = t3[3 * s + 1] = t3[3 * s + 2] = 0.0;
        if (mask[s] == ORC_SOLID) continue;
        int x, y, z;
        coords(C, s, &x, &y, &z);
        double r = qn[s], bs = 0.0;
        for (int a = 0; a < C->dim; a++)
            for (int sg = -1; sg <= 1; sg += 2) {
                long nb = 0;
                double v = 0.0;
                int k = pois_nb(C, mask, x, y, z, a, sg, &nb, &v);
                if (k == PN_UNKNOWN) r += eps_face(C->p, eps[s], eps[nb]) * (phi[nb] - phi[s]);
                else if (k == PN_DIRICHLET) { r += eps[s] * (v - phi[s]); bs += eps[s] * v; }
            }
        t3[3 * s] = r * r;
        if (mask[s] == ORC_FLUID) t3[3 * s + 1] = (qn[s] + qmean) * (qn[s] + qmean);
        t3[3 * s + 2] = bs * bs;
    }
    double r2 = 0.0, q2 = 0.0, b2 = 0.0;
    for (long s = 0; s < C->N; s++) {
        if (mask[s] == ORC_SOLID) continue;
        r2 += t3[3 * s];
        if (mask[s] == ORC_FLUID) q2 += t3[3 * s + 1];
        b2 += t3[3 * s + 2];
    }
    *rn = sqrt(r2);
    *ref = sqrt(q2) + sqrt(b2);
}

/* Colour of a site in the SOR sweep. (x + y + z) mod 2 (red-black) colours
 * every face neighbour differently unless a periodic extent is odd: there
 * the two sites across the wrap, x = 0 and x = n - 1, have the same parity.
 * With an odd periodic extent the sweep takes three colours, (c(x) + c(y) +
 * c(z)) mod 3 with c(i) = i mod 2 except c = 2 at i = n - 1 on an odd
 * periodic axis: c differs by 1 or 2 between face neighbours on every axis
 * (the wrap included), so the sum mod 3 does too. The sweep order is the
 * paper's free choice (it states SOR, not an ordering); the converged
 * potential is the solution of the same discrete system. */
static int odd_periodic(const ctx_t *C, int a)
{
    const int n = a == 0 ? C->nx : (a == 1 ? C->ny : C->nz);
    return C->p->face_bc[2 * a] == ORC_FACE_PERIODIC && (n & 1) && n > 1;
}
static int sor_ncolors(const ctx_t *C)
{
    for (int a = 0; a < C->dim; a++)
        if (odd_periodic(C, a)) return 3;
    return 2;
}
static int col3_axis(const ctx_t *C, int a, int i)
{
    const int n = a == 0 ? C->nx : (a == 1 ? C->ny : C->nz);
    return (odd_periodic(C, a) && i == n - 1) ? 2 : (i & 1);
}
static int sor_color(const ctx_t *C, int ncol, int x, int y, int z)
{
    if (ncol == 2) return (x + y + z) & 1;
    return (col3_axis(C, 0, x) + col3_axis(C, 1, y) + (C->dim == 3 ? col3_axis(C, 2, z) : 0)) % 3;
}

/* Poisson equation div(eps grad phi) = -qn (Sec. II) by SOR with the site
 * ordering of sor_color, warm-started from phi. qn is the charge
 * after neutralisation, qmean the uniform charge that was subtracted. The
 * iteration stops when ||r||_2 <= tol (||q||_2 + ||b||_2), q = qn + qmean the
 * free charge on fluid nodes and b the Dirichlet data, or after a fixed
 * number of sweeps when poisson_fixed_sweeps > 0. With no Dirichlet data the
 * solution is defined up to a constant: it is shifted to zero mean. */
int orc_poisson_solve(const orc_params *p, const unsigned char *mask, const double *rho,
                      const double *qn, double qmean, double *phi, int *iters,
                      double *resid)
{
    ctx_t C;
    ctx_init(&C, p);
    double *eps = malloc(C.N * sizeof(double));
    double *t3 = malloc(3 * C.N * sizeof(double));
#pragma omp parallel for schedule(static)
    for (long s = 0; s < C.N; s++) eps[s] = eps_of(p, rho[s]);
    double w = p->sor_omega, rn = 0.0, ref = 0.0;
    const int ncol = sor_ncolors(&C);
    int k = 0;
    for (;;) {
        if (p->poisson_fixed_sweeps > 0) {
            if (k >= p->poisson_fixed_sweeps) break;
        } else {
            pois_residual(&C, mask, eps, qn, qmean, phi, &rn, &ref, t3);
            if (rn <= p->poisson_tol * ref || k >= p->poisson_maxit) break;
        }
        /* the sites of one colour read only the other colours */
        for (int color = 0; color < ncol; color++)
#pragma omp parallel for schedule(static)
            for (long s = 0; s < C.N; s++) {
                int x, y, z;
                coords(&C, s, &x, &y, &z);
                if (sor_color(&C, ncol, x, y, z) != color || mask[s] == ORC_SOLID) continue;
                double num = qn[s], den = 0.0;
                for (int a = 0; a < C.dim; a++)
                    for (int sg = -1; sg <= 1; sg += 2) {
                        long nb = 0;
                        double v = 0.0;
                        int kk = pois_nb(&C, mask, x, y, z, a, sg, &nb, &v);
                        if (kk == PN_UNKNOWN) {
                            double ef = eps_face(p, eps[s], eps[nb]);
                            num += ef * phi[nb];
                            den += ef;
                        } else if (kk == PN_DIRICHLET) {
                            num += eps[s] * v;
                            den += eps[s];
                        }
                    }
                if (den > 0.0) phi[s] = (1.0 - w) * phi[s] + w * num / den;
            }
        k++;
    }
    if (!has_dirichlet(&C, mask)) {
        double m = 0.0;
        long n = 0;
        for (long s = 0; s < C.N; s++)
            if (mask[s] != ORC_SOLID) { m += phi[s]; n++; }
        m /= (double)n;
        for (long s = 0; s < C.N; s++)
            if (mask[s] != ORC_SOLID) phi[s] -= m;
    }
    pois_residual(&C, mask, eps, qn, qmean, phi, &rn, &ref, t3);
    if (iters) *iters = k;
    if (resid) *resid = ref > 0.0 ? rn / ref : rn;
    free(eps);
    free(t3);
    return 0;
}

/* Dense form A phi = b of the same discrete Poisson problem, for a direct
 * solve on tiny lattices. index[s] = unknown number of site s (or -1). With
 * no Dirichlet data the last row is replaced by the zero-mean condition. */
int orc_poisson_system(const orc_params *p, const unsigned char *mask, const double *rho,
                       const double *qn, double *A, double *b, long *index, int *n_unknown)
{
    ctx_t C;
    ctx_init(&C, p);
    long n = 0;
    for (long s = 0; s < C.N; s++) index[s] = (mask[s] == ORC_SOLID) ? -1 : n++;
    *n_unknown = (int)n;
    for (long i = 0; i < n * n; i++) A[i] = 0.0;
    for (long s = 0; s < C.N; s++) {
        if (index[s] < 0) continue;
        long i = index[s];
        int x, y, z;
        coords(&C, s, &x, &y, &z);
        double es = eps_of(p, rho[s]);
        b[i] = -qn[s];
        for (int a = 0; a < C.dim; a++)
            for (int sg = -1; sg <= 1; sg += 2) {
                long nb = 0;
                double v = 0.0;
                int k = pois_nb(&C, mask, x, y, z, a, sg, &nb, &v);
                if (k == PN_UNKNOWN) {
                    double ef = eps_face(p, es, eps_of(p, rho[nb]));
                    A[i * n + i] -= ef;
                    A[i * n + index[nb]] += ef;
                } else if (k == PN_DIRICHLET) {
                    A[i * n + i] -= es;
                    b[i] -= es * v;
                }
            }
    }
    if (!has_dirichlet(&C, mask)) {
        for (long j = 0; j < n; j++) A[(n - 1) * n + j] = 1.0;
        b[n - 1] = 0.0;
    }
    return 0;
}

/* E = -grad phi by central differences plus the applied field (Sec. II).
 * Across a Neumann face the neighbour takes the site's own potential. */
void orc_efield(const orc_params *p, const unsigned char *mask, const double *phi, double *E)
{
    ctx_t C;
    ctx_init(&C, p);
#pragma omp parallel for schedule(static)
    for (long s = 0; s < C.N; s++) {
        E[3 * s] = E[3 * s + 1] = E[3 * s + 2] = 0.0;
        if (mask[s] != ORC_FLUID) continue;
        int x, y, z;
        coords(&C, s, &x, &y, &z);
        for (int a = 0; a < 3; a++) {
            if (a >= C.dim) { E[3 * s + a] = p->E_ext[a]; continue; }
            double pv[2];
            for (int k = 0; k < 2; k++) {
                long nb = 0;
                double v = 0.0;
                int kind = pois_nb(&C, mask, x, y, z, a, k ? 1 : -1, &nb, &v);
                pv[k] = (kind == PN_UNKNOWN) ? phi[nb] : (kind == PN_DIRICHLET ? v : phi[s]);
            }
            E[3 * s + a] = -(pv[1] - pv[0]) / 2.0 + p->E_ext[a];
        }
    }
}

/* Ohmic term R = div(sigma grad phi), same face rule as the Poisson operator. */
static double ohmic(const ctx_t *C, const unsigned char *mask, const double *rho,
                    const double *phi, long s)
{
    int x, y, z;
    coords(C, s, &x, &y, &z);
    double ss = sigma_of(C->p, rho[s]), R = 0.0;
    for (int a = 0; a < C->dim; a++)
        for (int sg = -1; sg <= 1; sg += 2) {
            long nb = 0;
            double v = 0.0;
            int k = pois_nb(C, mask, x, y, z, a, sg, &nb, &v);
            if (k == PN_UNKNOWN) R += 0.5 * (ss + sigma_of(C->p, rho[nb])) * (phi[nb] - phi[s]);
            else if (k == PN_DIRICHLET) R += ss * (v - phi[s]);
        }
    return R;
}

static int validate(const orc_params *p)
{
    if (p->dim != 2 && p->dim != 3) return -1;
    if (p->nx < 1 || p->ny < 1 || p->nz < 1) return -1;
    if (p->dim == 2 && p->nz != 1) return -1;
    if (p->charge_model == ORC_CHARGE_TRANSPORT && p->dim != 3) return -1;
    for (int f = 0; f < 2 * p->dim; f++)
        if ((p->face_bc[f] == ORC_FACE_PERIODIC) != (p->phi_bc[f] == ORC_PHI_PERIODIC)) return -1;
    if (p->nu0 <= 0.0 || p->nu_inf <= 0.0 || p->rho0 <= 0.0) return -1;
    return 0;
}

/* Populations of fluid sites that arrive from inlet / outlet nodes carry the
 * boundary equilibria at every time level, the initial one included (the
 * boundary nodes are sources of f^eq(rho_in, u_in) and f^eq(rho_out, 0)). */
void orc_apply_io(const orc_params *p, const unsigned char *mask, const double *u_in, double *f)
{
    ctx_t C;
    ctx_init(&C, p);
#pragma omp parallel for schedule(static)
    for (long s = 0; s < C.N; s++) {
        if (mask[s] != ORC_FLUID) continue;
        int x, y, z, face;
        coords(&C, s, &x, &y, &z);
        for (int k = 0; k < C.Q; k++) {
            long src = nbr(&C, x, y, z, -C.c[k][0], -C.c[k][1], -C.c[k][2], &face);
            if (src < 0 || (mask[src] != ORC_INLET && mask[src] != ORC_OUTLET)) continue;
            double uio[3] = {0, 0, 0}, fe[19];
            if (mask[src] == ORC_INLET && u_in)
                for (int a = 0; a < 3; a++) uio[a] = u_in[3 * src + a];
            orc_feq(p->dim, mask[src] == ORC_INLET ? p->rho_in : p->rho_out, uio, fe);
            f[k * C.N + s] = fe[k];
        }
    }
}

int orc_init(const orc_params *p, const unsigned char *mask, const double *rho0_field,
             const double *u0_field, const double *q0_field, const double *u_in,
             double *f, double *g, double *phi)
{
    if (validate(p)) return -1;
    ctx_t C;
    ctx_init(&C, p);
#pragma omp parallel for schedule(static)
    for (long s = 0; s < C.N; s++) {
        double feq[19];
        double u[3] = {0, 0, 0};
        if (u0_field) { u[0] = u0_field[3 * s]; u[1] = u0_field[3 * s + 1]; u[2] = u0_field[3 * s + 2]; }
        if (mask[s] == ORC_FLUID) {
            orc_feq(p->dim, rho0_field[s], u, feq);
            for (int q = 0; q < C.Q; q++) f[q * C.N + s] = feq[q];
        } else {
            for (int q = 0; q < C.Q; q++) f[q * C.N + s] = 0.0;
        }
        if (g) {
            for (int i = 0; i < 7; i++) {
                double cu = C7[i][0] * u[0] + C7[i][1] * u[1] + C7[i][2] * u[2];
                double q0 = q0_field ? q0_field[s] : 0.0;
                g[i * C.N + s] = (mask[s] == ORC_FLUID) ? W7[i] * q0 * (1.0 + cu / CS2_Q) : 0.0;
            }
        }
        phi[s] = 0.0;
    }
    orc_apply_io(p, mask, u_in, f);
    return 0;
}

/* ------------------------------------------------------------------------
 * Streaming, the left side of Eq. (lattice-b): f_p(r + c_p, t+1) = f*_p(r, t),
 * periodic faces wrapping, with halfway bounce-back where r + c_p is a solid
 * node or lies beyond a wall face (f_opp(p)(r, t+1) = f*_p(r, t)). Populations
 * arriving from an inlet node carry the inlet equilibrium f^eq(rho_in, u_in);
 * from an outlet node, the reservoir equilibrium f^eq(rho_out, 0). The D3Q7
 * charge populations stream the same way; inlet / outlet nodes carry no charge.
 * f_out / g_out must not alias fs / gs.
 * ---------------------------------------------------------------------- */
void orc_stream(const orc_params *p, const unsigned char *mask, const double *u_in,
                const double *rho, const double *fs, const double *gs,
                double *f_out, double *g_out)
{
    ctx_t C;
    ctx_init(&C, p);
    long N = C.N;
    int Q = C.Q;
    double *fn = calloc((size_t)Q * N, sizeof(double));
    double *gn = gs ? calloc(7 * N, sizeof(double)) : NULL;
    /* each destination (population, site) is written by one source site:
     * streaming is a permutation, bounce-back writes the site's own entry,
     * and inlet / outlet nodes do not push */
#pragma omp parallel for schedule(static)
    for (long s = 0; s < N; s++) {
        if (mask[s] != ORC_FLUID) continue;
        int x, y, z, face;
        coords(&C, s, &x, &y, &z);
        for (int k = 0; k < Q; k++) {
            long nb = nbr(&C, x, y, z, C.c[k][0], C.c[k][1], C.c[k][2], &face);
            if (nb < 0 || mask[nb] == ORC_SOLID) fn[C.opp[k] * N + s] = fs[k * N + s];
            else if (mask[nb] == ORC_FLUID) fn[k * N + nb] = fs[k * N + s];
        }
        for (int k = 0; k < Q; k++) {
            long src = nbr(&C, x, y, z, -C.c[k][0], -C.c[k][1], -C.c[k][2], &face);
            if (src < 0) continue;
            if (mask[src] == ORC_INLET || mask[src] == ORC_OUTLET) {
                double uio[3] = {0, 0, 0}, fe[19];
                if (mask[src] == ORC_INLET && u_in)
                    for (int a = 0; a < 3; a++) uio[a] = u_in[3 * src + a];
                orc_feq(p->dim, mask[src] == ORC_INLET ? p->rho_in : p->rho_out, uio, fe);
                fn[k * N + s] = fe[k];
            }
        }
        if (gs) {
            for (int i = 0; i < 7; i++) {
                long nb = nbr(&C, x, y, z, C7[i][0], C7[i][1], C7[i][2], &face);
                int opp = (i == 0) ? 0 : ((i & 1) ? i + 1 : i - 1);
                if (nb < 0 || mask[nb] == ORC_SOLID) gn[opp * N + s] = gs[i * N + s];
                else if (mask[nb] == ORC_FLUID) gn[i * N + nb] = gs[i * N + s];
            }
        }
    }
    memcpy(f_out, fn, (size_t)Q * N * sizeof(double));
    if (gs) memcpy(g_out, gn, 7 * N * sizeof(double));
    free(fn);
    if (gn) free(gn);
}

/* ------------------------------------------------------------------------
 * One time step (Sec. II C): alpha (Eq. entropic), gdot / nu / beta (Eqs.
 * strain2, carreau, beta), charge and Poisson, Shan-Chen force, then the
 * update Eq. (lattice-b) with the exact-difference source Eq. (add),
 * followed by streaming.
 *
 * State in/out: f (post-streaming populations at time t), g (D3Q7 charge
 * populations, transport mode), phi (potential, warm start). Outputs at
 * time t: rho, u (half-step velocity), q (free charge), alpha, nu, diag.
 * ---------------------------------------------------------------------- */
/* The adaptive inlet of the jet (Sec. III B): at each time step the mean
 * velocity of the fluid inside the nozzle sets the Poiseuille profile of the
 * inlet nodes. Reading: after the collision of the step, the mean over the
 * `region` sites of the half-step velocity along the inlet direction d (the
 * direction of the summed initial inlet velocities), divided by the initial
 * inlet profile's own mean along d, rescales that initial profile; the
 * populations that the inlet nodes send in the streaming of this step (those
 * of the next time level) carry the rescaled profile. */
static void inlet_rescale(const ctx_t *C, const unsigned char *mask, const unsigned char *region,
                          const double *u, const double *u_in0, double *u_in)
{
    double d[3] = {0, 0, 0}, mu = 0.0, m0 = 0.0;
    long nr = 0, ni = 0;
    for (long s = 0; s < C->N; s++)
        if (mask[s] == ORC_INLET)
            for (int a = 0; a < 3; a++) d[a] += u_in0[3 * s + a];
    double dn = sqrt(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]);
    if (dn == 0.0) return;
    for (int a = 0; a < 3; a++) d[a] /= dn;
    for (long s = 0; s < C->N; s++) {
        if (mask[s] == ORC_INLET) {
            m0 += u_in0[3 * s] * d[0] + u_in0[3 * s + 1] * d[1] + u_in0[3 * s + 2] * d[2];
            ni++;
        }
        if (region[s] && mask[s] == ORC_FLUID) {
            mu += u[3 * s] * d[0] + u[3 * s + 1] * d[1] + u[3 * s + 2] * d[2];
            nr++;
        }
    }
    if (ni == 0 || nr == 0 || m0 == 0.0) return;
    double ratio = (mu / (double)nr) / (m0 / (double)ni);
    for (long s = 0; s < C->N; s++)
        if (mask[s] == ORC_INLET)
            for (int a = 0; a < 3; a++) u_in[3 * s + a] = ratio * u_in0[3 * s + a];
}

int orc_step(const orc_params *p, const unsigned char *mask, double *u_in,
             const unsigned char *region, const double *u_in0,
             double *f, double *g, double *phi, double *rho, double *u, double *q,
             double *alpha_out, double *nu_out, double *diag)
{
    int vr = validate(p);
    if (vr) return vr;
    ctx_t C;
    ctx_init(&C, p);
    long N = C.N;
    int Q = C.Q;
    double *j = calloc(3 * N, sizeof(double));
    double *qn = calloc(N, sizeof(double));
    double *Fint = calloc(3 * N, sizeof(double));
    double *E = calloc(3 * N, sizeof(double));
    double *E2 = calloc(N, sizeof(double));
    double *fs = calloc((size_t)Q * N, sizeof(double));
    double *gs = g ? calloc(7 * N, sizeof(double)) : NULL;
    for (int k = 0; k < ORC_NDIAG; k++) diag[k] = 0.0;
    diag[5] = INFINITY;
    diag[6] = -INFINITY;

    /* moments: rho = sum f, rho u = sum f c */
    long nfluid = 0;
    for (long s = 0; s < N; s++)
        if (mask[s] == ORC_FLUID) nfluid++;
#pragma omp parallel for schedule(static)
    for (long s = 0; s < N; s++) {
        rho[s] = 0.0;
        q[s] = 0.0;
        if (mask[s] == ORC_FLUID) {
            for (int k = 0; k < Q; k++) {
                double fk = f[k * N + s];
                rho[s] += fk;
                for (int a = 0; a < 3; a++) j[3 * s + a] += fk * C.c[k][a];
            }
        } else if (mask[s] == ORC_INLET) rho[s] = p->rho_in;
        else if (mask[s] == ORC_OUTLET) rho[s] = p->rho_out;
    }

    /* free charge */
    if (p->charge_model == ORC_CHARGE_TRANSPORT) {
#pragma omp parallel for schedule(static)
        for (long s = 0; s < N; s++)
            if (mask[s] == ORC_FLUID)
                for (int i = 0; i < 7; i++) q[s] += g[i * N + s];
    } else if (p->charge_model == ORC_CHARGE_CONSERVED || p->charge_model == ORC_CHARGE_XI) {
        orc_charge_field(p, mask, rho, q, NULL, NULL);
    }
    double qsum = 0.0;
    for (long s = 0; s < N; s++)
        if (mask[s] == ORC_FLUID) qsum += q[s];
    double qmean = (p->neutralize && nfluid > 0) ? qsum / (double)nfluid : 0.0;
    for (long s = 0; s < N; s++) qn[s] = (mask[s] == ORC_FLUID) ? q[s] - qmean : 0.0;

    /* potential */
    int iters = 0;
    double resid = 0.0;
    if (p->charge_model != ORC_CHARGE_NONE)
        orc_poisson_solve(p, mask, rho, qn, qmean, phi, &iters, &resid);

    /* forces */
    orc_sc_force(p, mask, rho, Fint);
    orc_efield(p, mask, phi, E);
    if (p->force_el == ORC_FEL_FULL)
        for (long s = 0; s < N; s++)
            E2[s] = E[3 * s] * E[3 * s] + E[3 * s + 1] * E[3 * s + 1] + E[3 * s + 2] * E[3 * s + 2];

    /* per-site records of the collision, summed serially below: alpha
     * status, H-error, |u|, H(f), body force */
    int *ast = calloc(N, sizeof(int));
    double *aherr = calloc(N, sizeof(double));
    double *umag = calloc(N, sizeof(double));
    double *Hs = calloc(N, sizeof(double));
    double *Fs = calloc(3 * N, sizeof(double));
    double tau_q = 0.5 + p->Dq / CS2_Q;
#pragma omp parallel for schedule(static)
    for (long s = 0; s < N; s++) {
        /* the lagged Carreau reading takes the previous step's viscosity (in
         * nu_out; 0 before the first step means nu0) */
        const double nu_prev = nu_out[s] > 0.0 ? nu_out[s] : p->nu0;
        alpha_out[s] = 0.0;
        nu_out[s] = 0.0;
        u[3 * s] = u[3 * s + 1] = u[3 * s + 2] = 0.0;
        if (mask[s] != ORC_FLUID) continue;
        int x, y, z;
        coords(&C, s, &x, &y, &z);
        double r = rho[s], fl[19], feq[19], d[19], feq2[19];
        for (int k = 0; k < Q; k++) fl[k] = f[k * N + s];
        double F[3];
        for (int a = 0; a < 3; a++) F[a] = Fint[3 * s + a] + q[s] * E[3 * s + a];
        if (p->force_el == ORC_FEL_FULL) {
            /* Eq. (force_el2): + (eps - 1)/2 grad|E|^2, central differences,
             * a non-fluid neighbour taking the site's own |E|^2 */
            double e = eps_of(p, r);
            for (int a = 0; a < C.dim; a++) {
                double ev[2];
                for (int k = 0; k < 2; k++) {
                    int dd[3] = {0, 0, 0}, face;
                    dd[a] = k ? 1 : -1;
                    long nb = nbr(&C, x, y, z, dd[0], dd[1], dd[2], &face);
                    ev[k] = (nb < 0 || mask[nb] != ORC_FLUID) ? E2[s] : E2[nb];
                }
                F[a] += 0.5 * (e - 1.0) * (ev[1] - ev[0]) / 2.0;
            }
        }
        double ub[3];
        for (int a = 0; a < 3; a++) ub[a] = j[3 * s + a] / r;
        orc_feq(p->dim, r, ub, feq);
        for (int k = 0; k < Q; k++) d[k] = feq[k] - fl[k];

        double alpha = 2.0;
        int st = ORC_A_ROOT;
        if (p->alpha_mode == ORC_ALPHA_ENTROPIC) st = orc_alpha(p->dim, fl, d, p->alpha_eq_tol, &alpha);
        ast[s] = st;
        if (st == ORC_A_ROOT && p->alpha_mode == ORC_ALPHA_ENTROPIC)
            aherr[s] = fabs(orc_h(p->dim, fl, d, alpha)) / r;

        /* Eq. (stress): Pi = sum (f - feq) c c */
        double Pi[9] = {0};
        for (int k = 0; k < Q; k++)
            for (int a = 0; a < 3; a++)
                for (int b2 = 0; b2 < 3; b2++) Pi[3 * a + b2] -= d[k] * C.c[k][a] * C.c[k][b2];
        double Pn = orc_spectral_norm(p->dim, Pi);
        double gdot = 0.0, nu = p->nu0;
        if (p->carreau_lagged) orc_carreau_lagged(p, Pn, alpha, r, nu_prev, &gdot, &nu);
        else orc_carreau(p, Pn, alpha, r, &gdot, &nu);
        double beta = beta_of(nu);

        /* Eq. (add): S = feq(rho, u + F/rho) - feq(rho, u) */
        double u2[3];
        for (int a = 0; a < 3; a++) u2[a] = ub[a] + F[a] / r;
        orc_feq(p->dim, r, u2, feq2);
        /* Eq. (lattice-b): f* = f - alpha beta (f - feq) + S */
        for (int k = 0; k < Q; k++)
            fs[k * N + s] = fl[k] + alpha * beta * d[k] + (feq2[k] - feq[k]);

        double up[3];
        for (int a = 0; a < 3; a++) up[a] = (j[3 * s + a] + 0.5 * F[a]) / r;
        for (int a = 0; a < 3; a++) u[3 * s + a] = up[a];
        alpha_out[s] = alpha;
        nu_out[s] = nu;

        if (p->charge_model == ORC_CHARGE_TRANSPORT) {
            /* D3Q7 advection-diffusion of the free charge with the Ohmic source */
            double R = ohmic(&C, mask, rho, phi, s);
            for (int i = 0; i < 7; i++) {
                double cu = C7[i][0] * up[0] + C7[i][1] * up[1] + C7[i][2] * up[2];
                double geq = W7[i] * q[s] * (1.0 + cu / CS2_Q);
                double gi = g[i * N + s];
                gs[i * N + s] = gi - (gi - geq) / tau_q + W7[i] * R;
            }
        }

        umag[s] = sqrt(up[0] * up[0] + up[1] * up[1] + up[2] * up[2]);
        Hs[s] = orc_H(p->dim, fl);
        for (int a = 0; a < 3; a++) Fs[3 * s + a] = F[a];
    }
    /* diagnostics: sums in site order */
    double asum = 0.0;
    for (long s = 0; s < N; s++) {
        if (mask[s] != ORC_FLUID) continue;
        int st = ast[s];
        if (st == ORC_A_SHORTCUT) diag[8] += 1;
        else if (st == ORC_A_NOROOT) diag[9] += 1;
        else if (st == ORC_A_CLIPPED) diag[10] += 1;
        if (aherr[s] > diag[13]) diag[13] = aherr[s];
        double alpha = alpha_out[s];
        diag[0] += rho[s];
        for (int a = 0; a < 3; a++) diag[1 + a] += j[3 * s + a] + 0.5 * Fs[3 * s + a];
        diag[4] += q[s];
        if (alpha < diag[5]) diag[5] = alpha;
        if (alpha > diag[6]) diag[6] = alpha;
        asum += alpha;
        if (umag[s] > diag[14]) diag[14] = umag[s];
        diag[15] += Hs[s];
        for (int a = 0; a < 3; a++) diag[17 + a] += Fs[3 * s + a];
    }
    diag[7] = nfluid ? asum / (double)nfluid : 0.0;
    diag[11] = iters;
    diag[12] = resid;
    diag[16] = qmean;
    free(ast); free(aherr); free(umag); free(Hs); free(Fs);

    if (region && u_in0 && u_in) inlet_rescale(&C, mask, region, u, u_in0, u_in);
    orc_stream(p, mask, u_in, rho, fs, gs, f, g);

    free(j); free(qn); free(Fint); free(E); free(E2); free(fs);
    if (gs) free(gs);
    return 0;
}
