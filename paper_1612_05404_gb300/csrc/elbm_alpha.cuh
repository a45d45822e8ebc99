// elbm_alpha.cuh -- the entropic alpha of Eq. (entropic) in FP32 arithmetic,
// with a float-float guard that certifies |h(alpha)| <= 1e-10 rho.
//
// h(a) = H(f + a D) - H(f), H = sum_p f_p ln(f_p / w_p) (Eq. H), has the
// trivial root a = 0 and, when h'(0) < 0, one positive root (h is convex).
// Written without cancellation, with x_p = D_p / f_p and y = a x_p:
//   h(a) = sum_p f_p phi(a x_p) + a h'(0),  phi(y) = (1 + y) ln(1 + y) - y,
//   h'(0) = sum_p D_p (1 + ln(f_p / w_p)).
// The FP32 Newton root leaves |h| at the FP32 rounding level of its terms
// (about 1e-9 at interface sites). Where that level is above the target, the
// guard re-evaluates h'(0) and h in float-float arithmetic (an unevaluated sum
// of two FP32 values, about 44 significant bits; Dekker 1971, Knuth TAOCP
// vol. 2 4.2.2) and takes Newton steps on a float-float alpha until |h| <= 1e-10
// rho. GB300 issues FP64 at 1/64 of its FP32 rate, so the pairs of FP32
// operations are the cheaper way to the extra precision.
#pragma once

namespace elbm {
ELBM_VS_BEGIN

struct AlphaOutF {
    float alpha;    // the root (high part)
    float alpha_lo; // low part of the float-float root (0 unless the guard ran)
    float herr;     // |h(alpha)| / rho: evaluated, or the FP32 rounding bound
    int status;     // 0 root, 1 near-equilibrium shortcut, 2 no root, 3 clipped, 4 guard failed
    int guarded;    // the float-float guard ran for this site
    int iters;      // FP32 evaluations of h this lane used before it converged
};

// ---------------------------------------------------------------------------
// ln(1+y) and phi(y) in FP32 without cancellation, from the atanh series in
// s = y/(2+y): ln(1+y) = 2s (1 + t A1(t)), t = s^2, A1(t) = sum_k t^k/(2k+3),
// and, with y = 2s/(1-s), phi(y) = s y + 2 (1+y) s t A1(t) (no division).
// For |s| <= 1/3 (y in [-1/2, 1]) eight terms of A1 leave a truncation error
// below 1e-8 relative; beyond, the library log1pf (strong non-equilibrium).
// The far branch is a call, not inlined: 19 inlined copies of log1pf in the
// Newton loop would crowd the instruction cache for a branch rarely taken.
// ---------------------------------------------------------------------------
static __device__ __noinline__ float2 lphi_far(float y)
{
    const float lg = log1pf(y);
    return make_float2(lg, (1.f + y) * lg - y);
}

__device__ __forceinline__ float atanh_A1(float t)
{
    return 1.f / 3 + t * (1.f / 5 + t * (1.f / 7 + t * (1.f / 9 + t * (1.f / 11 + t * (1.f / 13 + t * (1.f / 15 + t * (1.f / 17)))))));
}

__device__ __forceinline__ void lphi_f32(float y, float *l, float *ph)
{
    const float s = __fdividef(y, 2.f + y);
    if (fabsf(s) <= 0.3334f) {
        const float t = s * s;
        const float A1 = atanh_A1(t);
        const float c = 2.f * s * t;
        *l = fmaf(c, A1, 2.f * s);
        *ph = fmaf(c * (1.f + y), A1, s * y);
    } else {
        const float2 r = lphi_far(y);
        *l = r.x;
        *ph = r.y;
    }
}

// ln(1+z) alone (the h'(0) terms)
__device__ __forceinline__ float l_f32(float z)
{
    const float s = __fdividef(z, 2.f + z);
    if (fabsf(s) <= 0.3334f) {
        const float t = s * s;
        return fmaf(2.f * s * t, atanh_A1(t), 2.f * s);
    }
    return lphi_far(z).x;
}

// ---------------------------------------------------------------------------
// float-float arithmetic. The rounded products that an error term is taken
// against are formed with __fmul_rn, which the compiler never fuses with a
// later addition: a fused p + e would count the product's rounding error
// twice, and whether the compiler fuses can change with register pressure.
// ---------------------------------------------------------------------------
struct ffl { float h, l; };

__device__ __forceinline__ ffl ff_two_sum(float a, float b)
{
    const float s = a + b;
    const float bb = s - a;
    return {s, (a - (s - bb)) + (b - bb)};
}
__device__ __forceinline__ ffl ff_norm(float a, float b)  // |a| >= |b| or a == 0
{
    const float s = a + b;
    return {s, b - (s - a)};
}
__device__ __forceinline__ ffl ff_add(ffl a, ffl b)
{
    ffl s = ff_two_sum(a.h, b.h);
    return ff_norm(s.h, s.l + (a.l + b.l));
}
__device__ __forceinline__ ffl ff_add_f(ffl a, float b)
{
    ffl s = ff_two_sum(a.h, b);
    return ff_norm(s.h, s.l + a.l);
}
__device__ __forceinline__ ffl ff_neg(ffl a) { return {-a.h, -a.l}; }
__device__ __forceinline__ ffl ff_prod(float a, float b)
{
    const float p = __fmul_rn(a, b);
    return {p, fmaf(a, b, -p)};
}
__device__ __forceinline__ ffl ff_mul(ffl a, ffl b)
{
    const float p = __fmul_rn(a.h, b.h);
    float e = fmaf(a.h, b.h, -p);
    e = fmaf(a.h, b.l, fmaf(a.l, b.h, e));
    return ff_norm(p, e);
}
__device__ __forceinline__ ffl ff_mul_f(ffl a, float b)
{
    const float p = __fmul_rn(a.h, b);
    const float e = fmaf(a.l, b, fmaf(a.h, b, -p));
    return ff_norm(p, e);
}
// a / b: FP32 quotient, its remainder in float-float, one corrective quotient
__device__ __forceinline__ ffl ff_div(ffl a, ffl b)
{
    const float q1 = __fdividef(a.h, b.h);
    const ffl r = ff_add(a, ff_neg(ff_mul_f(b, q1)));
    return ff_norm(q1, __fdividef(r.h, b.h));
}
__device__ __forceinline__ ffl ff_div_f(float a, float b)
{
    const float q1 = __fdividef(a, b);
    const float r = fmaf(-q1, b, a);  // exact remainder
    return ff_norm(q1, __fdividef(r, b));
}

__device__ __forceinline__ float atanh_A2(float t)
{
    return 1.f / 5 + t * (1.f / 7 + t * (1.f / 9 + t * (1.f / 11 + t * (1.f / 13 + t * (1.f / 15 + t * (1.f / 17))))));
}

// ln(1+y) in float-float for 1 + y > 0: reduce 1 + y by 2^k into [3/4, 3/2)
// (k = 0, no reduction, for the usual |y| < 1/4 .. 1/2), then ln = k ln 2 +
// 2 atanh(t) = k ln 2 + 2t (1 + q), t = u/(2+u), u = (1+y) 2^-k - 1, |t| <= 1/5,
// q = t^2/3 + t^4 A2(t^2): t, t^2/3 and the products in float-float, the
// tail t^4 A2 (at most 1/3 % of q) in FP32.
__device__ __forceinline__ ffl ff_log1p(ffl y)
{
    const float vh = 1.f + y.h;
    ffl u = y;
    int k = 0;
    if (vh < 0.75f || vh >= 1.5f) {
        k = ilogbf(vh * (4.f / 3.f));
        const ffl v = ff_add_f(y, 1.f);
        u = ff_add_f(ffl{ldexpf(v.h, -k), ldexpf(v.l, -k)}, -1.f);
    }
    const ffl t = ff_div(u, ff_add_f(u, 2.f));
    const ffl t2 = ff_mul(t, t);
    const float tt = t2.h;
    // 1/3 = 0x1.555556p-2 - 0x1.555556p-27 (+ below 2^-50)
    const ffl q = ff_add_f(ff_mul(t2, ffl{0x1.555556p-2f, -0x1.555556p-27f}), tt * tt * atanh_A2(tt));
    ffl l = ff_mul(ffl{2.f * t.h, 2.f * t.l}, ff_add_f(q, 1.f));
    if (k != 0) {
        // ln 2 = 0x1.62e43p-1 - 0x1.05c61p-29 (+ below 2^-52)
        const float kf = float(k);
        l = ff_add(l, ff_add_f(ff_prod(kf, 0x1.62e43p-1f), kf * -0x1.05c61p-29f));
    }
    return l;
}

// ln(1+z) for |z| <= 1/8: z - z^2/2 in float-float, the tail z^3 R3(z),
// R3 = 1/3 - z/4 + z^2/5 - ... (8 terms; below 3 % of ln), in FP32
__device__ __forceinline__ ffl ff_log1p_small(ffl z)
{
    const ffl z2 = ff_mul(z, z);
    const float zh = z.h;
    const float R3 = 1.f / 3 + zh * (-1.f / 4 + zh * (1.f / 5 + zh * (-1.f / 6 + zh * (1.f / 7 + zh * (-1.f / 8 + zh * (1.f / 9 + zh * (-1.f / 10)))))));
    return ff_add_f(ff_add(z, ffl{-0.5f * z2.h, -0.5f * z2.l}), z2.h * zh * R3);
}

// A guard runs on a group of L (1, 2, 4 or 8) consecutive lanes of a warp:
// member j takes the populations p = j, j + L, ... and the group's sums are
// combined by an XOR butterfly. Float and float-float addition are
// commutative bit for bit (TwoSum is exact in either order), so every member
// ends with the same totals and the group takes one path.
struct Grp {
    int j, L;
    unsigned mask;  // the group's lanes
};

__device__ __forceinline__ Grp grp_make(int j, int L)
{
    unsigned lane;
    asm("mov.u32 %0, %%laneid;" : "=r"(lane));
    const unsigned ones = L >= 32 ? 0xffffffffu : ((1u << L) - 1u);
    return Grp{j, L, ones << (lane & ~unsigned(L - 1))};
}
__device__ __forceinline__ float grp_sum(const Grp &g, float v)
{
    for (int o = 1; o < g.L; o <<= 1) v += __shfl_xor_sync(g.mask, v, o);
    return v;
}
__device__ __forceinline__ float grp_max(const Grp &g, float v)
{
    for (int o = 1; o < g.L; o <<= 1) v = fmaxf(v, __shfl_xor_sync(g.mask, v, o));
    return v;
}
__device__ __forceinline__ ffl grp_sum(const Grp &g, ffl v)
{
    for (int o = 1; o < g.L; o <<= 1)
        v = ff_add(v, ffl{__shfl_xor_sync(g.mask, v.h, o), __shfl_xor_sync(g.mask, v.l, o)});
    return v;
}

// ---------------------------------------------------------------------------
// The exact inputs of the guard. The populations are f_p = w_p + d_p with d_p
// the FP32 deviations and w_p the weights of the set in FP64; the
// guard forms, as float-float pairs, the site's moments drho = sum d and
// j = sum c d, u = j / rho, and Delta_p = f^eq_p - f_p of Eq. (2) written as
// w_p drho - d_p + w_p rho P_p(u), so that the root it certifies is the root
// of the exact equation for those populations (not for the FP32 Delta the
// collision applies, which carries rounding of the size of f^eq's terms).
// ---------------------------------------------------------------------------
__device__ __forceinline__ ffl w_ff(int p)
{
    constexpr double W0 = wq(0), W1 = wq(1), W2 = wq(Q - 1);  // rest, axis, diagonal
    constexpr float h0 = float(W0), h1 = float(W1), h2 = float(W2);
    constexpr float l0 = float(W0 - double(h0)), l1 = float(W1 - double(h1)), l2 = float(W2 - double(h2));
    return p == 0 ? ffl{h0, l0} : (p <= NAX ? ffl{h1, l1} : ffl{h2, l2});
}

struct SiteFF {
    ffl drho, rho, u[3], usq;
};

__device__ __forceinline__ void site_ff(const float *dev, SiteFF &m, const Grp &gp)
{
    ffl s = {0.f, 0.f}, j[3] = {{0.f, 0.f}, {0.f, 0.f}, {0.f, 0.f}};
#pragma unroll 1
    for (int p = gp.j; p < Q; p += gp.L) {
        const float v = dev[p];
        s = ff_add_f(s, v);
        const int c[3] = {cx(p), cy(p), cz(p)};
#pragma unroll
        for (int a = 0; a < 3; a++)
            if (c[a]) j[a] = ff_add_f(j[a], c[a] > 0 ? v : -v);
    }
    m.drho = grp_sum(gp, s);
    m.rho = ff_add_f(m.drho, 1.f);
#pragma unroll
    for (int a = 0; a < 3; a++) m.u[a] = ff_div(grp_sum(gp, j[a]), m.rho);
    m.usq = ff_add(ff_add(ff_mul(m.u[0], m.u[0]), ff_mul(m.u[1], m.u[1])), ff_mul(m.u[2], m.u[2]));
}

// Delta_p with P_p(u) = c.u (3 + 4.5 c.u) - 1.5 u^2 (Eq. 2, c_s^2 = 1/3)
__device__ __forceinline__ ffl delta_ff(int p, float devp, const SiteFF &m)
{
    ffl cu = {0.f, 0.f};
    const int c[3] = {cx(p), cy(p), cz(p)};
#pragma unroll
    for (int a = 0; a < 3; a++)
        if (c[a]) cu = ff_add(cu, c[a] > 0 ? m.u[a] : ff_neg(m.u[a]));
    const ffl P = ff_add(ff_mul(cu, ff_add_f(ff_mul_f(cu, 4.5f), 3.f)), ff_mul_f(m.usq, -1.5f));
    const ffl w = w_ff(p);
    return ff_add(ff_add_f(ff_mul(w, m.drho), -devp), ff_mul(ff_mul(w, m.rho), P));
}

// f_p = w_p + d_p and Delta_p of population p as pairs (Delta from the arrays
// the guard filled)
__device__ __forceinline__ ffl pop_ff(int p, const float *dev) { return ff_add_f(w_ff(p), dev[p]); }

// h'(0) in float-float: (1 + ln rho) sum Delta + sum Delta_p ln(1 + z_p), with
// z_p = f_p / (w_p rho) - 1 = (d_p - w_p drho) / (w_p rho) formed from small
// terms. The guard's loops are not unrolled: compact code for a path few
// warps take.
__device__ __forceinline__ ffl h0_ff(const float *dev, const float *Dh, const float *Dl, const SiteFF &m,
                                     const Grp &gp)
{
    ffl S = {0.f, 0.f}, T = {0.f, 0.f};
#pragma unroll 1
    for (int p = gp.j; p < Q; p += gp.L) {
        const ffl D = {Dh[p], Dl[p]};
        S = ff_add(S, D);
        const ffl w = w_ff(p);
        const ffl z = ff_div(ff_add_f(ff_neg(ff_mul(w, m.drho)), dev[p]), ff_mul(w, m.rho));
        // warp-uniform choice: a warp whose lanes disagree would run both paths
        const ffl l = __all_sync(__activemask(), fabsf(z.h) <= 0.125f) ? ff_log1p_small(z) : ff_log1p(z);
        T = ff_add(T, ff_mul(l, D));
    }
    S = grp_sum(gp, S);
    T = grp_sum(gp, T);
    // ln rho to FP32 accuracy suffices: sum Delta is at the rounding level of the pairs
    return ff_add(ff_mul_f(S, 1.f + logf(m.rho.h)), T);
}

// h(a) in float-float, h'(a) and h''(a) = sum f x^2 / (1 + a x) in FP32, at a
// float-float alpha
__device__ __forceinline__ void h_ff(const float *dev, const float *Dh, const float *Dl, ffl a, ffl a0, ffl *h,
                                     float *hp, float *hpp, const Grp &gp)
{
    ffl acc = {0.f, 0.f};
    float g = 0.f, g2 = 0.f;
#pragma unroll 1
    for (int p = gp.j; p < Q; p += gp.L) {
        const ffl F = pop_ff(p, dev), D = {Dh[p], Dl[p]};
        const ffl x = ff_div(D, F);
        const ffl y = ff_mul(a, x);
        const ffl l = ff_log1p(y);
        // phi = (1 + y) l - y: its cancellation for small y costs relative
        // accuracy 2^-44 |y| / phi, far below the target in absolute terms
        const ffl ph = ff_add(ff_mul(ff_add_f(y, 1.f), l), ff_neg(y));
        acc = ff_add(acc, ff_mul(ph, F));
        g = fmaf(D.h, l.h, g);
        g2 = fmaf(F.h * x.h, __fdividef(x.h, 1.f + y.h), g2);
    }
    *h = ff_add(grp_sum(gp, acc), ff_mul(a, a0));
    *hp = grp_sum(gp, g) + a0.h;
    *hpp = grp_sum(gp, g2);
}

// h(a) from the site's moments when |a x_p| <= 1/16 for every p: the series
// phi(y) = y^2/2 - y^3/6 + sum_{n>=4} (-1)^n y^n / (n (n-1)) summed over p gives
//   h(a) = a h'(0) + a^2 M2/2 - a^3 M3/6 + sum_{n=4}^{8} (-1)^n a^n M_n/(n(n-1)),
// M_n = sum_p f_p x_p^n. M2 and M3 in float-float, M4..M8 in FP32 (their terms
// are below 1/1000 of the M2 term); truncation after n = 8 leaves below
// 1e-10 of the M2 term. The moments do not depend on a, so each Newton step
// of the guard costs a few dozen operations instead of 19 float-float logs.
struct MomFF {
    ffl M2, M3;
    float Mh[9];  // Mh[n], n = 4..8
    float xmax;
};

__device__ __forceinline__ void mom_ff(const float *dev, const float *Dh, const float *Dl, MomFF &m, const Grp &gp)
{
    m.M2 = ffl{0.f, 0.f};
    m.M3 = ffl{0.f, 0.f};
#pragma unroll
    for (int n = 0; n < 9; n++) m.Mh[n] = 0.f;
    m.xmax = 0.f;
#pragma unroll 1
    for (int p = gp.j; p < Q; p += gp.L) {
        const ffl F = pop_ff(p, dev), D = {Dh[p], Dl[p]};
        const ffl x = ff_div(D, F);
        const ffl fx2 = ff_mul(ff_mul(x, x), F);
        const ffl fx3 = ff_mul_f(fx2, x.h);
        m.M2 = ff_add(m.M2, fx2);
        m.M3 = ff_add(m.M3, fx3);
        float t = fx3.h;
#pragma unroll
        for (int n = 4; n <= 8; n++) {
            t *= x.h;
            m.Mh[n] += t;
        }
        m.xmax = fmaxf(m.xmax, fabsf(x.h));
    }
    m.M2 = grp_sum(gp, m.M2);
    m.M3 = grp_sum(gp, m.M3);
#pragma unroll
    for (int n = 4; n <= 8; n++) m.Mh[n] = grp_sum(gp, m.Mh[n]);
    m.xmax = grp_max(gp, m.xmax);
}

__device__ __forceinline__ ffl h_mom(ffl a, ffl a0, const MomFF &m, float *hp, float *hpp)
{
    const ffl a2 = ff_mul(a, a);
    const ffl a3 = ff_mul(a2, a);
    ffl h = ff_mul(a, a0);
    const ffl t2 = ff_mul(a2, m.M2);
    h = ff_add(h, ffl{0.5f * t2.h, 0.5f * t2.l});
    // 1/6 = 0x1.555556p-3 - 0x1.555556p-28 (+ below 2^-51)
    const ffl t3 = ff_mul(ff_mul(a3, m.M3), ffl{0x1.555556p-3f, -0x1.555556p-28f});
    h = ff_add(h, ff_neg(t3));
    const float ah = a.h;
    float tail = 0.f, d1 = 0.f, d2 = 0.f;
#pragma unroll
    for (int n = 8; n >= 4; n--) {
        const float cn = ((n & 1) ? -1.f : 1.f) / float(n * (n - 1));
        tail = fmaf(tail, ah, cn * m.Mh[n]);
        d1 = fmaf(d1, ah, float(n) * cn * m.Mh[n]);
        d2 = fmaf(d2, ah, float(n * (n - 1)) * cn * m.Mh[n]);
    }
    const float a_2 = ah * ah;
    h = ff_add_f(h, tail * a_2 * a_2);
    *hp = a0.h + ah * m.M2.h - 0.5f * a_2 * m.M3.h + d1 * a_2 * ah;
    *hpp = m.M2.h - ah * m.M3.h + d2 * a_2;
    return h;
}

// The float-float guard from an FP32 root a, for the site whose FP32
// deviations are dev: the exact moments and Delta (Dh, Dl: the caller's
// scratch of Q floats each, filled here), h'(0) and h as pairs. Where h'(0)
// is small against the rounding of the FP32 Delta the exact root can lie far
// from the FP32 one, so the iteration starts from the root of the exact
// moment series (as the FP32 start, now from the pairs) when that differs
// from a by more than 1e-3 a. Newton steps a' = a - h/h' inside the sign
// bracket (0, amax) (h is convex: h < 0 left of the root), bisection when a
// step leaves it; accept when |h| <= tol/2, or after a step when the
// quadratic-convergence bound 3/4 h'' (a' - a)^2 plus 1e-11 rho (the pairs'
// evaluation error) is within tol/2; at most 12 evaluations. Returns (alpha
// high, alpha low, H-error, w) on every lane of the group (j its member
// index, L its size), w = 1 accepted, 0 not certified, 2 no root (exact
// h'(0) >= 0: alpha = 2), 3 clipped at the positivity bound. Not inlined: one copy of the code, entered only by
// warps that hold a site needing it.
static __device__ __noinline__ float4 alpha_guard(const float *dev, float *Dh, float *Dl, float a, float S,
                                                  float amax, float htol, int j, int L)
{
    const Grp gp = grp_make(j, L);
    SiteFF m;
    site_ff(dev, m, gp);
#pragma unroll 1
    for (int p = gp.j; p < Q; p += gp.L) {
        const ffl D = delta_ff(p, dev[p], m);
        Dh[p] = D.h;
        Dl[p] = D.l;
    }
    const float rho = m.rho.h;
    const float tol = htol * rho;
    const ffl A0 = h0_ff(dev, Dh, Dl, m, gp);
    // the exact h'(0) can be >= 0 where the FP32 one was < 0 (both at the
    // rounding level): no positive root, alpha = 2 as for status 2
    if (A0.h >= 0.f) return make_float4(2.f, 0.f, 0.f, 2.f);
    // the exact moments: the series start below, and the series form of h
    // wherever |a x_p| <= 1/16 (decided per evaluation for the whole warp)
    MomFF mom;
    mom_ff(dev, Dh, Dl, mom, gp);
    const float hi0 = amax * (1.f - 1e-6f);
    float lo = 0.f, hi = hi0;
    ffl al = {a, 0.f};
    if (a * S <= 0.06f) {
        // root of h'(0) + a M2/2 - a^2 M3/6 + a^3 M4/12 (Newton from -2 h'(0)/M2)
        const float a0 = A0.h, M2 = mom.M2.h, M3 = mom.M3.h, M4 = mom.Mh[4];
        float c = -2.f * a0 / M2;
#pragma unroll 1
        for (int it = 0; it < 4; it++) {
            const float gg = a0 + c * (0.5f * M2 + c * (-M3 / 6.f + c * (M4 / 12.f)));
            const float gd = 0.5f * M2 + c * (-M3 / 3.f + c * (M4 / 4.f));
            const float cn = c - gg / gd;
            if (cn > 0.f && cn < hi) c = cn;
        }
        if (c > lo && c < hi && fabsf(c - a) > 1e-3f * a) al = ffl{c, 0.f};
    }
#pragma unroll 1
    for (int it = 0; it < 12; it++) {
        ffl hf;
        float hp, hpp;
        if (__all_sync(__activemask(), al.h * mom.xmax <= 0.0625f)) hf = h_mom(al, A0, mom, &hp, &hpp);
        else h_ff(dev, Dh, Dl, al, A0, &hf, &hp, &hpp, gp);
        if (fabsf(hf.h) <= 0.5f * tol) return make_float4(al.h, al.l, fabsf(hf.h) / rho, 1.f);
        if (hf.h < 0.f) lo = fmaxf(lo, al.h); else hi = fminf(hi, al.h);
        const float delta = hf.h / hp;
        const ffl an = ff_add_f(al, -delta);
        if (!(an.h >= lo && an.h <= hi)) {  // a step within one FP32 ulp moves only the low part
            al = ffl{0.5f * (lo + hi), 0.f};  // bisection; no convergence bound from this step
            continue;
        }
        al = an;
        const float pred = 0.75f * fabsf(hpp) * delta * delta + 1e-11f * rho;
        if (pred <= 0.5f * tol) return make_float4(al.h, al.l, pred / rho, 1.f);
    }
    // the root lies beyond the positivity bound: clipped there, as status 3
    if (lo >= hi0 * (1.f - 1e-5f)) return make_float4(hi0, 0.f, 0.f, 3.f);
    return make_float4(al.h, al.l, 1e30f, 0.f);
}

// ---------------------------------------------------------------------------
// FP32 root. h'(0) = sum D_p ln(1 + z_p), z_p = f_p/(w_p rho) - 1 for the
// populations f_p = w_p + d_p (the exact Delta sums to zero, so the
// (1 + ln rho) sum D part of h'(0) vanishes). Start from the root of the moment expansion
// h(a)/a ~ h'(0) + a M2/2 - a^2 M3/6 + a^3 M4/12 (M_k = sum f x^k), then
// safeguarded Newton on the exact h (at most 12 steps; one or two near
// equilibrium). A start a_start > 0 inside the bracket (a learned proposal)
// replaces the series start. A lane has converged when h is exactly 0, or |h| is at the
// FP32 noise floor of its terms after a step below 1e-3 alpha, or the Newton
// step is below 1e-6 alpha; converged lanes keep their alpha while the rest of
// the warp iterates, and the warp leaves together.
//
// guard: the target is |h| <= 1e-10 rho (H-error) for the exact equation of
// the site's populations f_p = w_p + d_p (FP64 weights), whose Delta differs
// from the FP32 Delta the root is computed with. The bound on |h_exact - h|
// at the FP32 root a has four parts:
//  - the FP32 evaluation of h: 2^-21 (sum f phi + a (|h'(0)| + sum |D ln(1+z)|));
//  - alpha itself rounded to FP32: 2^-23 a |h'(a)|;
//  - the rounding of Delta (w drho - d_p is formed exactly): its final
//    rounding, 2^-24 |Delta_p| (taken as 2^-23; Delta_0 also carries the sum
//    of the others' through the mass correction), the rounding of w_p rho P_p
//    (2^-24 w_p rho (36 umax + 144 umax^2)) and the error du of u (through
//    dP_p/du), each entering h
//    through dh/dDelta_p = a ln(f'_p / w_p) (the ln rho part cancels: both
//    Deltas conserve mass) with |ln(f'_p/(w_p rho))| <= |ln(1+z_p)| + a |x_p| F,
//    F = 1/(1 + a min(x, 0)) (|ln(1+y)| <= |y|/(1 + min(y, 0)));
//  - the FP32 rounding of f_p = fl(w32_p + d_p) (at most 2^-25 w_p + 2^-24 f_p,
//    w_p / f_p <= 1.2 / rho) in sum f phi(a x), which moves h by
//    sum df_p (ln(1+y_p) - y_p), |ln(1+y) - y| <= y^2 F / 2:
//    2^-24 (1 + 0.6/rho) a^2 F M2.
// Lanes whose |h| + bound stays within half the target are certified as they
// are; the others take the float-float guard (alpha_guard), which forms the
// exact moments and Delta from the deviations, from the FP32 root, and report
// its H-error: the float-float |h|, or the quadratic-convergence bound after
// its Newton step. Without the guard the H-error reported is |h| + bound.
// ---------------------------------------------------------------------------
struct AlphaSetupF {
    float x[Q];      // Delta_p / f_p
    float a0;        // h'(0)
    float tla;       // sum |Delta_p ln(1 + z_p)| (rounding bound of h'(0))
    float amax;      // positivity bound min over Delta_p < 0 of -f_p/Delta_p
    float ac;        // the moment-series start
    float S;         // max |x_p|
    float M2;        // sum f x^2
    float Bz, Bx;    // sum E_p |ln(1+z_p)|, sum E_p |x_p|, E_p = |Delta_p| (+ the sum for p = 0)
    float Wz, Wx;    // sum w_p |ln(1+z_p)|, sum w_p |x_p|
    float Bu;        // rho du: the error of u scaled by the density
    float Uz, Ux;    // 3 |sum w c ln(1+z)|_1 + 46 umax Wz; (6.1 + 46 umax) Wx
    float Pr;        // 2^-22 rho (10 umax + 40 umax^2): rounding of w_p rho P_p over w_p
    float xneg;      // min(0, min_p x_p)
    int status;      // 0: solve; 1 near-equilibrium shortcut; 2 no root (h'(0) >= 0)
};

__device__ __forceinline__ void alpha_fp32_setup(const float *f, const float *d, const float *fdev, float rho,
                                                 float drho, float eq_tol, float du, float umax, AlphaSetupF &st)
{
    float maxabs = 0.f, xneg = 0.f;
    float tl0 = 0.f, tl1 = 0.f, tla = 0.f;
    float M2 = 0.f, M3 = 0.f, M4 = 0.f;
    float Bz = 0.f, Bx = 0.f, Wz = 0.f, Wx = 0.f, Esum = 0.f, lz0 = 0.f, x0 = 0.f;
    float Gx = 0.f, Gy = 0.f, Gz = 0.f;  // sum_p w_p c_p ln(1 + z_p)
    const float irho = 1.f / rho;
#pragma unroll
    for (int p = 0; p < Q; p++) {
        const float xp = __fdividef(d[p], f[p]);
        st.x[p] = xp;
        maxabs = fmaxf(maxabs, fabsf(xp));
        xneg = fminf(xneg, xp);
        // z_p = f_p / (w_p rho) - 1 for the site's population f_p = w_p + fdev_p
        // (w_p the exact weight, not its FP32 rounding w32_p = w_p + dw_p, and
        // not the rounded sum fl(w32_p + fdev_p): at the vapour density that
        // rounding is a few units of 2^-24 of f_p and would move h'(0) by
        // sum Delta_p dln_p): f_p - w_p rho = (fdev_p - w32_p drho) + dw_p drho,
        // formed from small terms; the product w32_p drho is split exactly
        // (TwoProd) because fdev_p and w32_p drho nearly cancel near equilibrium
        const float w32 = float(wq(p));
        const float dw = float(double(w32) - wq(p));
        const float iw = float(1.0 / wq(p));
        const float wd = __fmul_rn(w32, drho);   // not fused into the difference below
        const float wde = fmaf(w32, drho, -wd);  // exact error of the product (TwoProd)
        const float z = (__fsub_rn(fdev[p], wd) + fmaf(dw, drho, -wde)) * iw * irho;
        const float lz = l_f32(z);
        const float dl = d[p] * lz;
        if (p & 1) tl1 += dl; else tl0 += dl;
        tla += fabsf(dl);
        const float Ep = fabsf(d[p]);
        Bz = fmaf(Ep, fabsf(lz), Bz);
        Bx = fmaf(Ep, fabsf(xp), Bx);
        Esum += Ep;
        if (p == 0) { lz0 = fabsf(lz); x0 = fabsf(xp); }
        Wz = fmaf(w32, fabsf(lz), Wz);
        Wx = fmaf(w32, fabsf(xp), Wx);
        if (cx(p)) Gx = fmaf(float(cx(p)) * w32, lz, Gx);
        if (cy(p)) Gy = fmaf(float(cy(p)) * w32, lz, Gy);
        if (cz(p)) Gz = fmaf(float(cz(p)) * w32, lz, Gz);
        const float fx2 = f[p] * xp * xp;
        M2 += fx2;
        M3 += fx2 * xp;
        M4 += fx2 * xp * xp;
    }
    // h'(0) of the exact equation: its Delta sums to zero (f^eq has the
    // density rho), so (1 + ln rho) sum Delta is left out (for the FP32 Delta
    // that sum is a rounding residual)
    const float a0 = tl0 + tl1;
    st.a0 = a0;
    st.tla = tla;
    st.S = maxabs;
    st.status = !(maxabs >= eq_tol) ? 1 : (a0 >= 0.f ? 2 : 0);
    st.amax = xneg < 0.f ? -1.f / xneg : 1e30f;
    st.M2 = M2;
    st.xneg = xneg;
    // Delta_0 also takes the compensated sum of the others (mass), hence the
    // rounding of all of them
    st.Bz = fmaf(Esum, lz0, Bz);
    st.Bx = fmaf(Esum, x0, Bx);
    st.Wz = Wz;
    st.Wx = Wx;
    // u enters Delta through w_p rho P_p(u), dP_p/du_a = 3 c_a + 9 (c.u) c_a
    // - 3 u_a: an error du of each component moves h'(0) = sum Delta_p
    // ln(1+z_p) by at most rho du (3 |G|_1 + 45 umax Wz), G = sum w c ln(1+z)
    // (sum w dP = 0: f^eq keeps the density), and sum f phi through x_p by
    // rho du (6 + 45 umax) sum w |x| a F. The FP32 evaluation of w_p rho P_p
    // itself rounds by at most 2^-24 w_p rho (36 umax + 144 umax^2).
    const float usq = umax * umax;
    st.Bu = rho * du;
    st.Uz = fmaf(46.f * umax, Wz, 3.f * (fabsf(Gx) + fabsf(Gy) + fabsf(Gz)));
    st.Ux = fmaf(46.f, umax, 6.1f) * Wx;
    st.Pr = 0x1p-22f * rho * fmaf(40.f, usq, 10.f * umax);
    // start: root of a0 + a M2/2 - a^2 M3/6 + a^3 M4/12, Newton from -2 a0/M2
    float a = -2.f * a0 / M2;
    for (int it = 0; it < 3; it++) {
        float gg = a0 + a * (0.5f * M2 + a * (-M3 / 6.f + a * (M4 / 12.f)));
        float gp = 0.5f * M2 + a * (-M3 / 3.f + a * (M4 / 4.f));
        float an = a - gg / gp;
        if (an > 0.f && an < 8.f) a = an;
    }
    st.ac = a;
}

// Newton from a_start (a proposal) if it lies inside (0, amax), else from the
// series start. A lane has converged when h is exactly 0; or |h| is at the
// FP32 noise floor of its terms after a step below 1e-3 alpha; or the Newton
// step d predicts an error after it, h''/(2|h'|) d^2 (quadratic convergence,
// h'' = sum f x^2/(1 + a x)), below 2^-25 alpha; or the step is below 1e-6
// alpha. Converged lanes keep their alpha while the rest of the warp iterates;
// the warp leaves together. The residual carried to the guard test is the
// evaluated |h| or, after an accepted step, the predicted h''/2 d^2.
__device__ __forceinline__ AlphaOutF alpha_fp32_solve(const float *f, const float *d, const float *dev, float rho,
                                                      const AlphaSetupF &st, bool guard, float a_start,
                                                      bool defer_guard = false, float htol = 1e-10f)
{
    AlphaOutF o;
    o.alpha = 2.f; o.alpha_lo = 0.f; o.herr = 0.f; o.status = st.status; o.guarded = 0; o.iters = 0;
    if (st.status != 0) return o;
    const float a0 = st.a0, amax = st.amax, irho = 1.f / rho;
    float lo = 0.f, hi = amax * (1.f - 1e-6f);
    float a = st.ac;
    if (a_start > lo && a_start < hi) a = a_start;
    if (!(a > lo && a < hi)) a = fminf(2.f, 0.5f * hi);
    float hres = 0.f, hhl = 0.f, hpl = 0.f;
    float step_prev = 1e30f;
    bool conv = false;
    for (int it = 0; it < 12; it++) {
        // four partial sums: shorter dependency chains than one running sum
        float hq[4] = {0.f, 0.f, 0.f, 0.f}, gq[4] = {0.f, 0.f, 0.f, 0.f}, kq[2] = {0.f, 0.f};
#pragma unroll
        for (int p = 0; p < Q; p++) {
            float l, ph;
            const float y = a * st.x[p];
            if (1.f + y <= 0.f) { ph = -y; l = -88.f; }
            else lphi_f32(y, &l, &ph);
            hq[p & 3] = fmaf(f[p], ph, hq[p & 3]);
            gq[p & 3] = fmaf(d[p], l, gq[p & 3]);
            kq[p & 1] = fmaf(d[p] * st.x[p], __fdividef(1.f, 1.f + y), kq[p & 1]);
        }
        const float hh = (hq[0] + hq[1]) + (hq[2] + hq[3]);
        const float g = (gq[0] + gq[1]) + (gq[2] + gq[3]);
        const float hpp = kq[0] + kq[1];
        if (!conv) {
            o.iters++;
            const float h = hh + a * a0;
            hres = fabsf(h);
            hhl = hh;
            hpl = g + a0;
            if (h == 0.f || (step_prev <= 1e-3f * a && fabsf(h) <= 5e-7f * (hh + fabsf(a * a0)))) {
                conv = true;
            } else {
                if (h < 0.f) lo = a; else hi = a;
                float an = a - h / hpl;
                if (an == a) {
                    // the Newton step is below the FP32 resolution of alpha: a
                    // is the root at this precision (a bracket bound now, so
                    // the strict test below would send it to a bisection)
                    conv = true;
                } else {
                    const bool newton = an > lo && an < hi;
                    if (!newton) an = 0.5f * (lo + hi);
                    const float step = fabsf(an - a);
                    step_prev = step;
                    a = an;
                    const float pred = 0.5f * hpp * step * step;  // |h| after the step, to leading order
                    if (newton && (pred <= 0x1p-25f * a * fabsf(hpl) || step <= 1e-6f * a)) {
                        conv = true;
                        hres = pred;
                    }
                }
            }
        }
        if (__all_sync(__activemask(), conv)) break;
    }
    o.alpha = a;
    o.status = a >= amax * (1.f - 2e-6f) ? 3 : 0;
    const float aF = __fdividef(a, fmaxf(fmaf(a, st.xneg, 1.f), 0x1p-10f));
    const float bound = 0x1p-21f * (hhl + a * (fabsf(a0) + st.tla)) + 0x1p-23f * a * fabsf(hpl) +
                        a * (0x1p-23f * fmaf(aF, st.Bx, st.Bz) + st.Bu * fmaf(aF, st.Ux, st.Uz) +
                             st.Pr * fmaf(aF, st.Wx, st.Wz)) +
                        0x1p-24f * fmaf(0.6f, irho, 1.f) * a * aF * st.M2;
    o.herr = (hres + bound) * irho;
    if (!guard || o.status == 3) return o;
    const float tol = htol * rho;
    const bool need = !(hres + bound <= 0.5f * tol);
    if (need && defer_guard) {  // the caller runs alpha_guard (compacted) and fills in the result
        o.guarded = 2;
        return o;
    }
    if (need) {
        o.guarded = 1;
        float Dh[Q], Dl[Q];
        const float4 gr = alpha_guard(dev, Dh, Dl, a, st.S, st.amax, htol, 0, 1);
        o.alpha = gr.x;
        o.alpha_lo = gr.y;
        o.herr = gr.z;
        if (gr.w == 0.f) { o.status = 4; o.herr = hres * irho; }
        else if (gr.w >= 2.f) o.status = int(gr.w);  // 2 no root, 3 clipped
    }
    return o;
}

__device__ __forceinline__ AlphaOutF alpha_fp32(const float *f, const float *d, const float *fdev,
                                                float rho, float drho, float eq_tol, float du, float umax,
                                                bool guard, float a_start = -1.f)
{
    AlphaSetupF st;
    alpha_fp32_setup(f, d, fdev, rho, drho, eq_tol, du, umax, st);
    return alpha_fp32_solve(f, d, fdev, rho, st, guard, a_start);
}

ELBM_VS_END
}  // namespace elbm
