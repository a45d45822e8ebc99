// elbm_device.cuh -- device-side building blocks of the charged entropic
// lattice Boltzmann step of Lauricella et al. (arXiv:1612.05404), Sec. II:
// precision traits, the D3Q19 / D3Q7 velocity sets, and the per-site physics
// (Eq. 2 equilibrium, Eq. entropic alpha root, Eq. strain2 / carreau / beta
// viscosity, the matrix 2-norm of the stress).
#pragma once

#include <cuda_runtime.h>
#include <cuda_bf16.h>
#include <stdint.h>

#include "elbm.h"

namespace elbm {

// ---------------------------------------------------------------------------
// Velocity set of the populations. A translation unit compiles the kernels
// for one set: D3Q19 by default, the paper's D2Q9 (Sec. II, the set its
// Eq. 2 is written for) where ELBM_D2Q9 is defined. Everything that depends
// on the set (the tables, the per-site physics, the kernels and their
// launchers) sits in an inline namespace named after it, so that the two
// builds link into one library side by side; the problem description, the
// constants and the buffer tables below are common to both. Components are
// encoded as characters '0'/'1'/'2' for -1/0/+1 so that an unrolled loop
// folds them to constants; opposite links are consecutive (p = 2k-1, 2k) in
// both orders, which are the library's public population orders
// (elbm_velocity_set_of).
// ---------------------------------------------------------------------------
#ifdef ELBM_D2Q9
#define ELBM_VS_BEGIN inline namespace d2q9 {
#else
#define ELBM_VS_BEGIN inline namespace d3q19 {
#endif
#define ELBM_VS_END }

ELBM_VS_BEGIN
#ifdef ELBM_D2Q9
// D2Q9: rest 4/9, the 4 axis links 1/9, the 4 diagonals 1/36, c_s^2 = 1/3;
// lattices of this set are one site thick in z (nz = 1).
constexpr int Q = 9;
__host__ __device__ constexpr int cx(int p) { return "120112020"[p] - '1'; }
__host__ __device__ constexpr int cy(int p) { return "111202002"[p] - '1'; }
__host__ __device__ constexpr int cz(int p) { return "111111111"[p] - '1'; }
__host__ __device__ constexpr double wq(int p) { return p == 0 ? 4.0 / 9.0 : (p < 5 ? 1.0 / 9.0 : 1.0 / 36.0); }
#else
// D3Q19 (the 3-D set with the c_s^2 = 1/3 of the paper's D2Q9): rest 1/3, the
// 6 axis links 1/18, the 12 face diagonals 1/36.
constexpr int Q = 19;
__host__ __device__ constexpr int cx(int p) { return "1201111202020201111"[p] - '1'; }
__host__ __device__ constexpr int cy(int p) { return "1112011200211112020"[p] - '1'; }
__host__ __device__ constexpr int cz(int p) { return "1111120111120022002"[p] - '1'; }
__host__ __device__ constexpr double wq(int p) { return p == 0 ? 1.0 / 3.0 : (p < 7 ? 1.0 / 18.0 : 1.0 / 36.0); }
#endif
// number of the axis links (the rest population is 0, they are 1..NAX)
constexpr int NAX = Q == 9 ? 4 : 6;
__host__ __device__ constexpr int opp(int p) { return p == 0 ? 0 : ((p & 1) ? p + 1 : p - 1); }
constexpr double CS2 = 1.0 / 3.0;
ELBM_VS_END

// D3Q7 for the charge advection-diffusion: rest 1/4, axis links 1/8, c_s^2 = 1/4.
constexpr int Q7 = 7;
__host__ __device__ constexpr int c7x(int i) { return "1201111"[i] - '1'; }
__host__ __device__ constexpr int c7y(int i) { return "1112011"[i] - '1'; }
__host__ __device__ constexpr int c7z(int i) { return "1111120"[i] - '1'; }
__host__ __device__ constexpr double w7(int i) { return i == 0 ? 0.25 : 0.125; }
constexpr double CS2Q = 0.25;

// ---------------------------------------------------------------------------
// Precision traits: storage type of the populations, arithmetic type, type
// of the scalar planes (rho, q, phi), and whether populations are handled as
// deviations d_p = f_p - w_p from the rest-state equilibrium (dev). BF16
// storage (rel) keeps f_p - w_p rho_ref instead, rho_ref the density of the
// site that wrote the value (a plane beside the populations, A/B like them):
// at a gas-phase site (rho ~ 0.16) f_p - w_p is about -0.84 w_p, whose 8-bit
// significand would leave ~1 % of f_p as noise, while f_p - w_p rho is of
// the order of the Mach number.
// ---------------------------------------------------------------------------
template <int PR> struct Tr;
template <> struct Tr<ELBM_PREC_FP64> {
    typedef double st; typedef double ct; typedef double sc; typedef double gt;
    static constexpr bool dev = false, rel = false;
};
template <> struct Tr<ELBM_PREC_FP32> {
    typedef float st; typedef float ct; typedef float sc; typedef float gt;
    static constexpr bool dev = true, rel = false;
};
template <> struct Tr<ELBM_PREC_BF16> {
    typedef __nv_bfloat16 st; typedef float ct; typedef float sc; typedef float gt;
    static constexpr bool dev = true, rel = true;
};

__device__ __forceinline__ float to_ct(float v) { return v; }
__device__ __forceinline__ double to_ct(double v) { return v; }
__device__ __forceinline__ float to_ct(__nv_bfloat16 v) { return __bfloat162float(v); }
template <typename S> __device__ __forceinline__ S from_ct(float v);
template <> __device__ __forceinline__ float from_ct<float>(float v) { return v; }
template <> __device__ __forceinline__ __nv_bfloat16 from_ct<__nv_bfloat16>(float v) { return __float2bfloat16_rn(v); }
template <typename S> __device__ __forceinline__ S from_ct(double v);
template <> __device__ __forceinline__ double from_ct<double>(double v) { return v; }

// ---------------------------------------------------------------------------
// Problem description passed by value to every kernel.
// ---------------------------------------------------------------------------
struct Geom {
    int nx, ny, nz;
    long long N;
    int per[3];          // axis periodic (both faces)
    int phi_kind[6];     // ELBM_PHI_* per face
    int phi_axis;
    int has_mask;        // any non-fluid node
    int phi_lin;         // the potential plane holds psi = phi - phi_lin, phi_lin(c) = phi_lo + (c+1) slope
                         // along phi_axis (reduced precision, both electrode faces Dirichlet)
    int ncol;            // colours of the Poisson sweep ordering: 2 (red-black) or 3 (an odd periodic extent)
};

// Colour of a cell in the Poisson sweep ordering. Red-black, (x + y + z) mod
// 2, gives every face neighbour the other colour unless a periodic extent is
// odd: the two cells across the wrap then share a parity. There the ordering
// takes three colours, (c(x) + c(y) + c(z)) mod 3 with c(i) = i mod 2 except
// c = 2 on the last cell of an odd periodic axis; c differs by 1 or 2 between
// face neighbours on every axis (the wrap included), so the sum mod 3 does.
__host__ __device__ __forceinline__ int col3_axis(int i, int n, int per)
{
    return (per && (n & 1) && n > 1 && i == n - 1) ? 2 : (i & 1);
}
__host__ __device__ __forceinline__ int color3(const int per[3], int x, int y, int z, int nx, int ny, int nz)
{
    return (col3_axis(x, nx, per[0]) + col3_axis(y, ny, per[1]) + col3_axis(z, nz, per[2])) % 3;
}
__host__ __device__ __forceinline__ int ncolors_of(const int per[3], int nx, int ny, int nz)
{
    const int n[3] = {nx, ny, nz};
    for (int a = 0; a < 3; a++)
        if (per[a] && (n[a] & 1) && n[a] > 1) return 3;
    return 2;
}

// Constants of one step in the arithmetic type T, precomputed on the host so
// FP32 kernels never touch GB300's slow FP64 pipe.
template <typename T>
struct Cst {
    T G, Gw, rho0, irho0, kap;       // Shan-Chen; eps = 1 + kap rho
    T sig_g, dsig, itw;              // sigma = sig_g + dsig theta(rho), 1/theta_width
    T itau_q;                        // 1/tau of the charge LB
    T E[3];                          // applied field
    T Qb, Qs, iKd, xib, xis;         // charge models
    T omega;                         // SOR relaxation
    T eq_tol;                        // alpha near-equilibrium threshold
    T htol;                          // H-error target per unit density of the FP32 alpha root
    T phi_lo, phi_hi, phi_solid, phi_slope;  // potential data; slope = (hi - lo)/(n_axis + 1)
    T nu0, nu_inf, lam, nexp;        // Carreau: nexp = (n - 1)/2
};

// neighbour coordinate along one axis: -1 when it leaves through a wall face
__device__ __forceinline__ int nbc(int v, int n, int per)
{
    if (v < 0) return per ? v + n : -1;
    if (v >= n) return per ? v - n : -1;
    return v;
}

// potential on the ghost node beyond face `face` seen from (x,y,z): the
// electrode value on faces normal to phi_axis, the linear profile between
// them on the other Dirichlet faces
template <typename T>
__device__ __forceinline__ T phi_ghost(const Geom &g, const Cst<T> &k, int face, int x, int y, int z)
{
    int axis = face >> 1;
    if (axis == g.phi_axis) return (face & 1) ? k.phi_hi : k.phi_lo;
    int c = g.phi_axis == 0 ? x : (g.phi_axis == 1 ? y : z);
    return k.phi_lo + T(c + 1) * k.phi_slope;
}

ELBM_VS_BEGIN
// ---------------------------------------------------------------------------
// Eq. (2): f^eq_p = w_p rho (1 + P_p(u)), P_p(u) = c.u/c_s^2 + ((c.u)^2 - c_s^2 u^2)/(2 c_s^4)
// ---------------------------------------------------------------------------
template <typename T>
__device__ __forceinline__ T Ppoly(int p, T ux, T uy, T uz, T usq)
{
    T cu = T(cx(p)) * ux + T(cy(p)) * uy + T(cz(p)) * uz;
    return T(3) * cu + T(4.5) * cu * cu - T(1.5) * usq;
}

// ---------------------------------------------------------------------------
// Delta = f^eq(rho, u) - f with deviation storage (FP32 arithmetic), from the
// deviations d_p = f_p - w_p and drho = rho - 1 as an unevaluated sum
// (drho_hi + drho_lo). At a low-density site w_p drho and d_p nearly cancel,
// so their difference is formed in one rounding (fmaf), the FP32 rounding of
// the weight dw_p = w_p - fl(w_p) is added back, and the compensated sum of
// the result is taken off Delta_0: the exact Delta conserves mass (f^eq has
// the density rho), and an O(ulp) residual would enter h'(0) of Eq.
// (entropic) through (1 + ln rho) sum Delta, which is larger than h'(0)
// itself near equilibrium.
// ---------------------------------------------------------------------------
__device__ __forceinline__ void two_sum_acc(float v, float &s, float &c)
{
    const float t = s + v;
    const float bp = t - s;
    c += (s - (t - bp)) + (v - bp);
    s = t;
}

__device__ __forceinline__ void delta_dev(const float *d, float drho_hi, float drho_lo, float r, float ux, float uy,
                                          float uz, float usq, float *D)
{
    float s = 0.f, c = 0.f;
#pragma unroll
    for (int p = 0; p < Q; p++) {
        const float w32 = float(wq(p));
        const float dw = float(wq(p) - double(w32));
        const float P = Ppoly<float>(p, ux, uy, uz, usq);
        // w32 drho - d_p exactly, as ah + al + pe (TwoProd of the product,
        // TwoSum of the difference): the two nearly cancel, and their
        // rounding would otherwise be the largest error of Delta
        const float pr = __fmul_rn(w32, drho_hi);
        const float pe = fmaf(w32, drho_hi, -pr);
        const float ah = pr - d[p];
        const float bb = ah - pr;
        const float al = (pr - (ah - bb)) + (-d[p] - bb);
        D[p] = ah + ((al + pe) + fmaf(w32, drho_lo, fmaf(dw, drho_hi, w32 * r * P)));
        two_sum_acc(D[p], s, c);
    }
    D[0] -= s + c;
}

// Moments of a site from its FP32 deviations d_p = f_p - w_p: drho = sum d as
// a compensated pair (rs, rs_lo), and the momentum j = sum_p c_p d_p formed
// from the differences of opposite populations first. Opposite links are
// consecutive (p = 2k-1, 2k); within a factor 2 of each other (a site near
// equilibrium, whatever its density) their difference is exact (Sterbenz
// 1974), so j carries rounding of the size of its own terms e_k, not of the
// deviations, which at the vapour density are about -0.84 w_p and cancel in
// j. esum = sum_k |e_k| bounds the rounding of j: each component's error is
// at most 2^-21 esum.
__device__ __forceinline__ void moments_dev(const float *d, float &rs, float &rs_lo, float &jx, float &jy, float &jz,
                                            float &esum)
{
    rs = 0.f;
    rs_lo = 0.f;
#pragma unroll
    for (int p = 0; p < Q; p++) two_sum_acc(d[p], rs, rs_lo);
    {
        const float t = rs + rs_lo;
        rs_lo = rs_lo - (t - rs);
        rs = t;
    }
    constexpr int NP = (Q - 1) / 2;
    float e[NP];
    esum = 0.f;
#pragma unroll
    for (int k = 0; k < NP; k++) {
        e[k] = d[2 * k + 1] - d[2 * k + 2];
        esum += fabsf(e[k]);
    }
#ifdef ELBM_D2Q9
    // e_0..e_3: +-x, +-y, (1,1), (1,-1)
    jx = (e[0] + e[2]) + e[3];
    jy = (e[1] + e[2]) - e[3];
    jz = 0.f;
#else
    // e_0..e_8: +-x, +-y, +-z, (1,1,0), (1,-1,0), (1,0,1), (1,0,-1), (0,1,1), (0,1,-1)
    jx = ((e[0] + e[3]) + (e[4] + e[5])) + e[6];
    jy = ((e[1] + e[3]) - (e[4] - e[7])) + e[8];
    jz = ((e[2] + e[5]) - (e[6] - e[7])) - e[8];
#endif
}

// Bound on the absolute FP32 error of each component of u = j (1/rho): the
// rounding of j (2^-21 esum) over rho, plus the roundings of 1/rho, of the
// product and of rho = 1 + drho itself (four units of 2^-24, taken as eight)
__device__ __forceinline__ float u_err_bound(float esum, float r, float umax)
{
    return __fdividef(0x1p-21f * esum, r) + 0x1p-21f * umax;
}

// FP32 moments and Delta of a site from its deviations d (populations
// f = w + d), as the FP32 collision forms them; returns rho. du: the bound
// of u_err_bound, umax = max |u_a|.
__device__ __forceinline__ float site_delta(const float *d, float *f, float *D, float *drho_out, float *du_out,
                                            float *umax_out)
{
    float rs, rs_lo, jx, jy, jz, esum;
    moments_dev(d, rs, rs_lo, jx, jy, jz, esum);
    const float r = 1.f + rs;
    const float ir = 1.f / r;
    const float ux = jx * ir, uy = jy * ir, uz = jz * ir;
    const float usq = ux * ux + uy * uy + uz * uz;
    delta_dev(d, rs, rs_lo, r, ux, uy, uz, usq, D);
#pragma unroll
    for (int p = 0; p < Q; p++) f[p] = float(wq(p)) + d[p];
    *drho_out = rs;
    const float umax = fmaxf(fabsf(ux), fmaxf(fabsf(uy), fabsf(uz)));
    *du_out = u_err_bound(esum, r, umax);
    *umax_out = umax;
    return r;
}

// ---------------------------------------------------------------------------
// Matrix 2-norm of the symmetric stress (Sec. II B): max |eigenvalue|, by
// the closed-form trigonometric solution of the characteristic cubic
// (Smith 1961).
// ---------------------------------------------------------------------------
// FP32 quotient and cosine in the fast forms (a few ulp; the quotient is 0
// for |b| > 2^126), FP64 exact: used where that error stays below the FP32
// result's own tolerance
__device__ __forceinline__ float qdiv(float a, float b) { return __fdividef(a, b); }
__device__ __forceinline__ double qdiv(double a, double b) { return a / b; }
__device__ __forceinline__ float qcos(float a) { return __cosf(a); }
__device__ __forceinline__ double qcos(double a) { return cos(a); }

template <typename T>
__device__ __forceinline__ T sym3_norm2(T a00, T a11, T a22, T a01, T a02, T a12)
{
    T p1 = a01 * a01 + a02 * a02 + a12 * a12;
    T q = (a00 + a11 + a22) * T(1.0 / 3.0);
    T b00 = a00 - q, b11 = a11 - q, b22 = a22 - q;
    T p2 = b00 * b00 + b11 * b11 + b22 * b22 + T(2) * p1;
    if (p2 <= T(0)) return fabs(q);
    if (p1 == T(0)) return fmax(fabs(a00), fmax(fabs(a11), fabs(a22)));
    T pp = sqrt(p2 * T(1.0 / 6.0));
    T ip = T(1) / pp;
    b00 *= ip; b11 *= ip; b22 *= ip;
    T c01 = a01 * ip, c02 = a02 * ip, c12 = a12 * ip;
    T det = b00 * (b11 * b22 - c12 * c12) - c01 * (c01 * b22 - c12 * c02) + c02 * (c01 * c12 - b11 * c02);
    T r = det * T(0.5);
    r = fmin(T(1), fmax(T(-1), r));
    T phi = acos(r) * T(1.0 / 3.0);
    T e1 = q + T(2) * pp * qcos(phi);
    T e3 = q + T(2) * pp * qcos(phi + T(2.0943951023931954923));
    return fmax(fabs(e1), fabs(e3));
}

// ---------------------------------------------------------------------------
// Carreau law Eq. (carreau) inside Eq. (strain2): gdot = A beta(nu(gdot)),
// A = Pi alpha / (rho c_s^2), beta(nu) = c_s^2/(2 nu + c_s^2) (Eq. beta).
// The root lies in [A beta(nu0), A beta(nu_inf)]; safeguarded Newton from the
// left end of that bracket. Returns nu.
// ---------------------------------------------------------------------------
__device__ __forceinline__ float powT(float b, float e) { return __powf(b, e); }
__device__ __forceinline__ double powT(double b, double e) { return pow(b, e); }

template <typename T>
__device__ __forceinline__ T carreau_nu(const Cst<T> &k, bool newtonian, T Pn, T alpha, T rho)
{
    const T cs2 = T(1.0 / 3.0);
    if (newtonian) return k.nu0;
    T A = Pn * alpha / (rho * cs2);
    if (A == T(0)) return k.nu0;
    T lo = A * cs2 / (T(2) * k.nu0 + cs2), hi = A * cs2 / (T(2) * k.nu_inf + cs2);
    T x = lo;
    // FP32: stop at a relative step of 2e-6 or when g is at the noise floor
    // of its two terms; FP64: to the last bits
    const T eps = sizeof(T) == 8 ? T(4e-16) : T(2e-6);
    const int itmax = sizeof(T) == 8 ? 100 : 16;
    for (int it = 0; it < itmax; it++) {
        T lg = k.lam * x;
        T base = T(1) + lg * lg;
        T pw = powT(base, k.nexp);
        T nux = k.nu_inf + (k.nu0 - k.nu_inf) * pw;
        T den = T(2) * nux + cs2;
        T gx = x - qdiv(A * cs2, den);
        bool done = (gx == T(0));
        if (!done) {
            if (gx < T(0)) lo = x; else hi = x;
            T dnu = qdiv((k.nu0 - k.nu_inf) * T(2) * k.nexp * k.lam * k.lam * x * pw, base);
            T gp = T(1) + qdiv(T(2) * cs2 * A * dnu, den * den);
            T xn = x - qdiv(gx, gp);
            if (xn == x) {
                done = true;  // step below the resolution of x (x is a bracket bound now)
            } else {
                if (!(xn > lo && xn < hi)) xn = T(0.5) * (lo + hi);
                done = fabs(xn - x) <= eps * fabs(x) || hi - lo <= eps * hi ||
                       (sizeof(T) == 4 && fabs(gx) <= T(5e-7) * (x + qdiv(A * cs2, den)));
                x = xn;
            }
        }
        if (sizeof(T) == 8) {
            if (done) break;
        } else if (__all_sync(__activemask(), done)) {
            break;  // FP32: leave together, no divergent tail
        }
    }
    T lg = k.lam * x;
    return k.nu_inf + (k.nu0 - k.nu_inf) * powT(T(1) + lg * lg, k.nexp);
}

// The lagged reading: Eq. (strain2) with tau from the previous step's
// viscosity nu_prev, gdot = A beta(nu_prev), no root; then Eq. (carreau).
template <typename T>
__device__ __forceinline__ T carreau_nu_lagged(const Cst<T> &k, T Pn, T alpha, T rho, T nu_prev)
{
    const T cs2 = T(1.0 / 3.0);
    const T gdot = qdiv(Pn * alpha, rho * cs2) * qdiv(cs2, T(2) * nu_prev + cs2);
    const T lg = k.lam * gdot;
    return k.nu_inf + (k.nu0 - k.nu_inf) * powT(T(1) + lg * lg, k.nexp);
}

// permittivity of a face of the Poisson operator: arithmetic or harmonic
// mean of the two sites
template <typename T>
__device__ __forceinline__ T face_eps(T ea, T eb, int harmonic)
{
    return harmonic ? qdiv(T(2) * ea * eb, ea + eb) : T(0.5) * (ea + eb);
}

// ---------------------------------------------------------------------------
// Entropic alpha, Eq. (entropic) with Eq. (H): the nontrivial root of
//   h(a) = H(f + a D) - H(f) = sum_p [ f_p phi(a x_p) ] + a h'(0),
//   x_p = D_p/f_p, phi(y) = (1+y) ln(1+y) - y,  h'(0) = sum_p D_p (1 + ln(f_p/w_p)).
// h is convex with h(0) = 0, so h'(0) < 0 gives one root in (0, a_max], a_max
// the positivity bound min_{D_p<0} -f_p/D_p. Status codes as in the
// diagnostics: 0 root, 1 near-equilibrium shortcut, 2 no root (h'(0) >= 0),
// 3 clipped at the positivity bound. The fallback in 1 and 2 is a = 2 (BGK).
// ---------------------------------------------------------------------------
struct AlphaOut { double alpha, herr; int status; };

// FP64: same root as the plain definition, Newton in the sign bracket from 2.
__device__ __forceinline__ AlphaOut alpha_fp64(const double *f, const double *d, double rho,
                                               double eq_tol)
{
    AlphaOut o; o.alpha = 2.0; o.herr = 0.0; o.status = 0;
    double x[Q], lnw[Q];
    double maxabs = 0.0, amax = 1e300, a0 = 0.0;
#pragma unroll
    for (int p = 0; p < Q; p++) {
        x[p] = d[p] / f[p];
        maxabs = fmax(maxabs, fabs(x[p]));
        if (d[p] < 0.0) amax = fmin(amax, -f[p] / d[p]);
        lnw[p] = log(f[p] / wq(p));
        a0 += d[p] * (1.0 + lnw[p]);
    }
    if (!(maxabs >= eq_tol)) { o.status = 1; return o; }
    if (a0 >= 0.0) { o.status = 2; return o; }
    auto hval = [&](double a, double *hp) {
        double h = 0.0, g = 0.0;
#pragma unroll
        for (int p = 0; p < Q; p++) {
            double y = a * x[p];
            double l = log1p(y);
            double t = (1.0 + y <= 0.0) ? 0.0 : (f[p] + a * d[p]) * l;
            h += t + a * d[p] * lnw[p];
            g += d[p] * (1.0 + lnw[p] + l);
        }
        *hp = g;
        return h;
    };
    double lo = 0.0, hi, hp;
    if (amax < 1e299) {
        hi = amax * (1.0 - 1e-15);
        if (hval(hi, &hp) < 0.0) { o.alpha = hi; o.status = 3; return o; }
    } else {
        hi = 4.0;
        int k = 0;
        while (hval(hi, &hp) < 0.0 && k++ < 100) hi *= 2.0;
    }
    double a = 2.0;
    if (!(a > lo && a < hi)) a = 0.5 * (lo + hi);
    double h = 0.0;
    for (int it = 0; it < 100; it++) {
        h = hval(a, &hp);
        if (h == 0.0) break;
        if (h < 0.0) lo = a; else hi = a;
        double an = a - h / hp;
        if (an == a) break;  // step below the FP64 resolution of alpha
        if (!(an > lo && an < hi)) an = 0.5 * (lo + hi);
        if (fabs(an - a) <= 4e-16 * fabs(a) || hi - lo <= 4e-16 * hi) { a = an; break; }
        a = an;
    }
    o.alpha = a;
    o.herr = fabs(h) / rho;
    return o;
}

ELBM_VS_END
}  // namespace elbm

#include "elbm_alpha.cuh"
