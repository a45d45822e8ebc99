// elbm_kernels.cuh -- the kernels of one time step of the charged entropic
// lattice Boltzmann method (arXiv:1612.05404, Sec. II C), templated on the
// population precision. Each k_*.cu translation unit instantiates them for
// one precision and one velocity set (D3Q19, or D2Q9 where it defines
// ELBM_D2Q9; see elbm_device.cuh).
//
// Data layout: populations are planes [p][site] (site = x + nx (y + ny z)) in
// two buffers A (read) and B (write); streaming is done by "pull": the step
// reads f_p(r, t) = f*_p(r - c_p, t-1) from A and writes the post-collision
// f*_p(r, t) to B at its own site, so every plane access is coalesced along x.
// Halfway bounce-back turns a pull across a wall face or from a solid node
// into a read of the opposite population of the site itself. Inlet and outlet
// nodes hold their equilibria in both buffers, so a pull from them reads
// f^eq(rho_in, u_in) or f^eq(rho_out, 0).
#pragma once

#include "elbm_internal.h"
#include "elbm_mlp.cuh"

namespace elbm {

typedef long long ll;

ELBM_VS_BEGIN

// ---------------------------------------------------------------------------
// Block reductions. FP64 precision reduces in FP64. The FP32 modes reduce
// within a warp in FP32 with an error-free transformation (TwoSum, Knuth) so
// the sums keep FP64-like accuracy without using GB300's slow FP64 pipe, then
// combine the warps in FP64. Every thread of the block must call.
// ---------------------------------------------------------------------------
__device__ __forceinline__ void two_sum(float a, float b, float &s, float &e)
{
    s = a + b;
    float bb = s - a;
    e = (a - (s - bb)) + (b - bb);
}

__device__ __forceinline__ double warp_sum(double v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    return v;
}
// float <-> int with the same order (two's complement: negative floats
// have their magnitude bits flipped); a NaN maps to the stand-in value
__device__ __forceinline__ int float_ord(float v, float nan_as)
{
    const int i = __float_as_int(v == v ? v : nan_as);
    return i >= 0 ? i : i ^ 0x7fffffff;
}
__device__ __forceinline__ float ord_float(int i) { return __int_as_float(i >= 0 ? i : i ^ 0x7fffffff); }

__device__ __forceinline__ int num_blocks() { return gridDim.x * gridDim.y * gridDim.z; }

// Per-block partial sums are stored column-major, part[k * nblocks + block],
// so the finalize kernel reads each column with coalesced loads.
// FP64 values: FP64 warp sums, thread 0 adds the warps.
template <int K>
__device__ __forceinline__ void block_sums(const double (&v)[K], double *out, int stride = 1)
{
    __shared__ double sh[K][8];
    const int tid = threadIdx.x + blockDim.x * threadIdx.y;
    const int lane = tid & 31, wid = tid >> 5;
    const int nw = (blockDim.x * blockDim.y + 31) >> 5;
#pragma unroll
    for (int k = 0; k < K; k++) {
        double w = warp_sum(v[k]);
        if (lane == 0) sh[k][wid] = w;
    }
    __syncthreads();
    if (tid == 0) {
#pragma unroll
        for (int k = 0; k < K; k++) {
            double t = 0.0;
            for (int i = 0; i < nw; i++) t += sh[k][i];
            out[(long long)k * stride] = t;
        }
    }
}

// FP32 values: compensated (hi, lo) FP32 sums across the warp and across the
// block's warps, so that no FP64 instruction runs per thread (the FP64 pipe
// of this part issues 1/64 of the FP32 rate); lane k of warp 0 turns sum k
// into FP64 once per block.
template <int K>
__device__ __forceinline__ void block_sums(const float (&v)[K], double *out, int stride = 1)
{
    __shared__ float sh[2][K][8];
    const int tid = threadIdx.x + blockDim.x * threadIdx.y;
    const int lane = tid & 31, wid = tid >> 5;
    const int nw = (blockDim.x * blockDim.y + 31) >> 5;
    // Within the warp, K values (padded to P = 1, 2, 4 or 8) are summed by a
    // transposed butterfly: at offsets 16, 8, ... each lane keeps half of its
    // values and adds its partner's copy of them, until one value per lane
    // remains, summed over the lanes that share the top lg P lane bits; the
    // last offsets sum that value over the rest. Lane L ends with value
    // L >> (5 - lg P): about 2 (P - 1) + 2 (5 - lg P) shuffles instead of 10 K.
    constexpr int P = K <= 1 ? 1 : (K <= 2 ? 2 : (K <= 4 ? 4 : 8));
    constexpr int LG = P == 1 ? 0 : (P == 2 ? 1 : (P == 4 ? 2 : 3));
    static_assert(K <= 8, "at most 8 sums per call");
    float hi[P], lo[P];
#pragma unroll
    for (int k = 0; k < P; k++) {
        hi[k] = k < K ? v[k] : 0.f;
        lo[k] = 0.f;
    }
#pragma unroll
    for (int st = 0; st < LG; st++) {
        const int o = 16 >> st, half = (P >> st) / 2;
        const bool up = (lane & o) != 0;
#pragma unroll
        for (int k = 0; k < half; k++) {
            const float kh = up ? hi[k + half] : hi[k], kl = up ? lo[k + half] : lo[k];
            const float sh_ = up ? hi[k] : hi[k + half], sl = up ? lo[k] : lo[k + half];
            const float rh = __shfl_xor_sync(0xffffffffu, sh_, o), rl = __shfl_xor_sync(0xffffffffu, sl, o);
            float sm, e;
            two_sum(kh, rh, sm, e);
            hi[k] = sm;
            lo[k] = kl + rl + e;
        }
    }
#pragma unroll
    for (int o = 16 >> LG; o > 0; o >>= 1) {
        const float rh = __shfl_xor_sync(0xffffffffu, hi[0], o), rl = __shfl_xor_sync(0xffffffffu, lo[0], o);
        float sm, e;
        two_sum(hi[0], rh, sm, e);
        hi[0] = sm;
        lo[0] += rl + e;
    }
    {
        const int k = lane >> (5 - LG);
        if ((lane & ((32 >> LG) - 1)) == 0 && k < K) { sh[0][k][wid] = hi[0]; sh[1][k][wid] = lo[0]; }
    }
    __syncthreads();
    if (tid < K) {
        float hi = sh[0][tid][0], lo = sh[1][tid][0];
        for (int i = 1; i < nw; i++) {
            float sm, e;
            two_sum(hi, sh[0][tid][i], sm, e);
            hi = sm;
            lo += sh[1][tid][i] + e;
        }
        out[(long long)tid * stride] = (double)hi + (double)lo;
    }
}

// ---------------------------------------------------------------------------
// Neighbourhood of a site: the index offsets of the -1, 0, +1 neighbours per
// axis with the periodic wrap folded in, and whether each exists (not beyond
// a wall face). Site indices are 32-bit (elbm_init refuses lattices of 2^31
// sites or more); plane offsets p * N are formed in 64 bits, once per plane.
// ---------------------------------------------------------------------------
struct Nbr {
    int s;
    int ox[3], oy[3], oz[3];
    bool vx[3], vy[3], vz[3];
};

__device__ __forceinline__ void nbr_init(Nbr &n, const Geom &g, int x, int y, int z, ll s)
{
    const int nx = g.nx, nxy = g.nx * g.ny;
    n.s = (int)s;
    n.ox[0] = x > 0 ? -1 : nx - 1;
    n.ox[1] = 0;
    n.ox[2] = x < nx - 1 ? 1 : 1 - nx;
    n.oy[0] = y > 0 ? -nx : (g.ny - 1) * nx;
    n.oy[1] = 0;
    n.oy[2] = y < g.ny - 1 ? nx : -(g.ny - 1) * nx;
    n.oz[0] = z > 0 ? -nxy : (g.nz - 1) * nxy;
    n.oz[1] = 0;
    n.oz[2] = z < g.nz - 1 ? nxy : -(g.nz - 1) * nxy;
    n.vx[0] = x > 0 || g.per[0]; n.vx[1] = true; n.vx[2] = x < nx - 1 || g.per[0];
    n.vy[0] = y > 0 || g.per[1]; n.vy[1] = true; n.vy[2] = y < g.ny - 1 || g.per[1];
    n.vz[0] = z > 0 || g.per[2]; n.vz[1] = true; n.vz[2] = z < g.nz - 1 || g.per[2];
}

// index of the site at offset (ox, oy, oz) in {-1,0,1}^3, or -1 beyond a wall
__device__ __forceinline__ int nbr_idx(const Nbr &n, const Geom &, int ox, int oy, int oz)
{
    if (!(n.vx[ox + 1] && n.vy[oy + 1] && n.vz[oz + 1])) return -1;
    return n.s + n.ox[ox + 1] + n.oy[oy + 1] + n.oz[oz + 1];
}

// plane p of a population array
template <typename S>
__device__ __forceinline__ const S *plane(const void *A, int p, ll N)
{
    return (const S *)A + (ll)p * N;
}
template <typename S>
__device__ __forceinline__ S *plane(void *A, int p, ll N)
{
    return (S *)A + (ll)p * N;
}

// stored value of population p at site idx as it enters the arithmetic: f_p
// (FP64) or d_p = f_p - w_p (deviation modes; BF16 adds back w_p (rho_ref - 1))
template <int PR>
__device__ __forceinline__ typename Tr<PR>::ct ldp(const void *A, int p, int idx, ll N, const float *rref)
{
    typedef typename Tr<PR>::ct ct;
    const ct v = to_ct(plane<typename Tr<PR>::st>(A, p, N)[idx]);
    if constexpr (Tr<PR>::rel) return v + ct(wq(p)) * (ct(rref[idx]) - ct(1));
    else return v;
}

// the value to store for population p of a site whose density is rho, from
// its FP32 deviation d = f - w (BF16: f - w rho)
template <int PR>
__device__ __forceinline__ typename Tr<PR>::st stp(typename Tr<PR>::ct d, int p, typename Tr<PR>::ct drho)
{
    typedef typename Tr<PR>::ct ct;
    if constexpr (Tr<PR>::rel) return from_ct<typename Tr<PR>::st>(d - ct(wq(p)) * drho);
    else return from_ct<typename Tr<PR>::st>(d);
}

// f_p(r, t): pull from r - c_p, bounce-back across walls and from solids.
// FP64 returns f_p; the deviation modes return d_p = f_p - w_p. rref: the
// reference-density plane of A (BF16 storage), else unused.
template <int PR>
__device__ __forceinline__ typename Tr<PR>::ct gather_pop(const Geom &g, const unsigned char *mask,
                                                          const void *A, const Nbr &n, int p,
                                                          const float *rref = nullptr)
{
    const int src = nbr_idx(n, g, -cx(p), -cy(p), -cz(p));
    bool bb = src < 0;
    if (!bb && mask) bb = mask[src] == ELBM_NODE_SOLID;
    return bb ? ldp<PR>(A, opp(p), n.s, g.N, rref) : ldp<PR>(A, p, src, g.N, rref);
}

// The same pulls from a site's precomputed bounce bits (Bufs::bbits): the
// plane and index follow from one word loaded per site, so the 19 (or 7)
// loads do not wait for the node kinds of their sources (the moments pass,
// latency-bound; the collision reads the node kinds for its wall terms
// anyway and keeps the plain pulls).
template <int PR>
__device__ __forceinline__ typename Tr<PR>::ct gather_pop_b(const Geom &g, const void *A, const Nbr &n, int p,
                                                            unsigned bits, const float *rref = nullptr)
{
    const bool bb = (bits >> p) & 1u;
    const int src = bb ? n.s : nbr_idx(n, g, -cx(p), -cy(p), -cz(p));
    return ldp<PR>(A, bb ? opp(p) : p, src, g.N, rref);
}
template <int PR>
__device__ __forceinline__ typename Tr<PR>::gt gather_g_b(const Geom &g, const void *A, const Nbr &n, int i,
                                                          unsigned bits)
{
    typedef typename Tr<PR>::gt gt;
    const bool bb = (bits >> i) & 1u;
    const int src = bb ? n.s : nbr_idx(n, g, -c7x(i), -c7y(i), -c7z(i));
    const int io = i == 0 ? 0 : ((i & 1) ? i + 1 : i - 1);
    return plane<gt>(A, bb ? io : i, g.N)[src];
}
template <int PR>
__device__ __forceinline__ typename Tr<PR>::gt gather_g(const Geom &g, const unsigned char *mask,
                                                        const void *A, const Nbr &n, int i)
{
    typedef typename Tr<PR>::gt gt;
    const int src = nbr_idx(n, g, -c7x(i), -c7y(i), -c7z(i));
    bool bb = src < 0;
    if (!bb && mask) bb = mask[src] == ELBM_NODE_SOLID;
    const int io = i == 0 ? 0 : ((i & 1) ? i + 1 : i - 1);
    return bb ? plane<gt>(A, io, g.N)[n.s] : plane<gt>(A, i, g.N)[src];
}

template <typename T>
__device__ __forceinline__ T psi_of(T rho, T rho0) { return rho0 * (T(1) - exp(-rho / rho0)); }
// the same in the collision's arithmetic: FP32 as rho0 - rho0 2^(rho c),
// c = -log2(e)/rho0 (no division per neighbour); FP64 as psi_of
__device__ __forceinline__ float psi_nb(float rho, float rho0, float c) { return fmaf(-rho0, exp2f(rho * c), rho0); }
__device__ __forceinline__ double psi_nb(double rho, double rho0, double) { return psi_of<double>(rho, rho0); }
// conductivity sigma = sig_g + dsig (1 + tanh((rho - rho0)/w))/2; FP32 through
// (1 + tanh x)/2 = 1/(1 + e^(-2x)) with the fast exponential and quotient
// (the quotient tends to 0 as the exponential overflows)
__device__ __forceinline__ float sigma_of(const Cst<float> &k, float rho)
{
    return k.sig_g + __fdividef(k.dsig, 1.f + __expf(-2.f * (rho - k.rho0) * k.itw));
}
__device__ __forceinline__ double sigma_of(const Cst<double> &k, double rho)
{
    return k.sig_g + k.dsig * 0.5 * (1.0 + tanh((rho - k.rho0) * k.itw));
}

__device__ __forceinline__ void site_xyz(const Geom &g, int &x, int &y, int &z, bool &inb, ll &s)
{
    x = blockIdx.x * blockDim.x + threadIdx.x;
    y = blockIdx.y * blockDim.y + threadIdx.y;
    z = blockIdx.z;
    inb = x < g.nx && y < g.ny;
    s = inb ? x + (ll)g.nx * (y + (ll)g.ny * z) : 0;
}
__device__ __forceinline__ int block_id() { return blockIdx.x + gridDim.x * (blockIdx.y + gridDim.y * blockIdx.z); }

// the bounce bits of every site (once, at initialisation)
static __global__ void __launch_bounds__(128) k_bounce_bits(Geom g, const unsigned char *mask, unsigned *bits)
{
    int x, y, z;
    bool inb;
    ll s;
    site_xyz(g, x, y, z, inb, s);
    if (!inb) return;
    Nbr n;
    nbr_init(n, g, x, y, z, s);
    unsigned w = 0;
#pragma unroll
    for (int p = 0; p < Q; p++) {
        const int src = nbr_idx(n, g, -cx(p), -cy(p), -cz(p));
        if (src < 0 || (mask && mask[src] == ELBM_NODE_SOLID)) w |= 1u << p;
    }
    bits[s] = w;
}


// Potential of the face neighbour along +-axis (Sec. II Poisson problem):
// kind 0 = unknown (index in *nb), 1 = Dirichlet value in *v, 2 = no term.
// With the deviation form (g.phi_lin) the plane holds psi = phi - phi_lin,
// phi_lin the linear electrode profile along phi_axis: a Dirichlet value is
// returned as psi (0 on every electrode or lateral Dirichlet face, which
// carry phi_lin; phi_solid - phi_lin at a conductor) and *dl is
// phi_lin(neighbour) - phi_lin(site) (+-slope along phi_axis, else 0), which
// the caller adds to the neighbour's psi: every face term c (phi_nb - phi_s)
// is then c (psi_nb + dl - psi_s), the same difference formed from small
// numbers. Without it *dl = 0 and the plane holds phi.
template <typename T>
__device__ __forceinline__ int pois_nb(const Geom &g, const Cst<T> &k, const unsigned char *mask,
                                       const Nbr &n, int x, int y, int z, int axis, int sign, int *nb, T *v, T *dl)
{
    int o[3] = {0, 0, 0};
    o[axis] = sign;
    const int i = nbr_idx(n, g, o[0], o[1], o[2]);
    const bool lin = g.phi_lin != 0;
    *dl = (lin && axis == g.phi_axis) ? T(sign) * k.phi_slope : T(0);
    if (i < 0) {
        int face = 2 * axis + (sign > 0 ? 1 : 0);
        if (g.phi_kind[face] == ELBM_PHI_DIRICHLET) { *v = lin ? T(0) : phi_ghost<T>(g, k, face, x, y, z); return 1; }
        *dl = T(0);
        return 2;
    }
    if (mask && mask[i] == ELBM_NODE_SOLID) {
        if (lin) {
            const int c = (g.phi_axis == 0 ? x : (g.phi_axis == 1 ? y : z)) + (axis == g.phi_axis ? sign : 0);
            *v = k.phi_solid - (k.phi_lo + T(c + 1) * k.phi_slope);
        } else {
            *v = k.phi_solid;
        }
        return 1;
    }
    *nb = i;
    return 0;
}
// The quotient of a Gauss-Seidel / SOR update: in FP32 the fast reciprocal
// quotient (2 ulp; the sweep is an iteration towards the discrete solution,
// whose accuracy the residual test decides), in FP64 the exact one (the FP64
// path follows the oracle's sweeps)
__device__ __forceinline__ float pois_div(float a, float b) { return __fdividef(a, b); }
__device__ __forceinline__ double pois_div(double a, double b) { return a / b; }

// The fast path of the Poisson stencil: a site inside the lattice along y
// and z, none of its face neighbours solid. Its y and z neighbours are at
// s +- nx and s +- nx ny; its x neighbours xn[0] (x - 1) and xn[1] (x + 1),
// wrapped on a periodic axis, or -1 beyond a boundary face of the lattice
// (then the face's own term, as pois_nb gives it). The profile difference dl
// is +-slope along phi_axis in the deviation form. A row's first and last
// sites then cost their warp a few instructions instead of the general path
// (pois_nb), with the same operations in the same order.
__device__ __forceinline__ bool pois_fast(const Geom &g, const unsigned char *mask, int x, int y, int z, int si,
                                          int xn[2])
{
    if (y <= 0 || y >= g.ny - 1 || z <= 0 || z >= g.nz - 1) return false;
    xn[0] = x > 0 ? si - 1 : (g.per[0] ? si + g.nx - 1 : -1);
    xn[1] = x < g.nx - 1 ? si + 1 : (g.per[0] ? si - (g.nx - 1) : -1);
    if (!mask) return true;
    // six independent loads of one byte each (the site itself stands in for
    // a missing x neighbour: the callers have returned at solid sites); the
    // 4-byte bounce word would answer the same question with more traffic
    const int nx = g.nx, nxy = g.nx * g.ny;
    const unsigned char m0 = mask[xn[0] >= 0 ? xn[0] : si], m1 = mask[xn[1] >= 0 ? xn[1] : si];
    const unsigned char m2 = mask[si - nx], m3 = mask[si + nx], m4 = mask[si - nxy], m5 = mask[si + nxy];
    return (m0 != ELBM_NODE_SOLID) & (m1 != ELBM_NODE_SOLID) & (m2 != ELBM_NODE_SOLID) & (m3 != ELBM_NODE_SOLID) &
           (m4 != ELBM_NODE_SOLID) & (m5 != ELBM_NODE_SOLID);
}
template <typename T>
__device__ __forceinline__ T interior_dl(const Geom &g, const Cst<T> &k, int a, int sg)
{
    return (g.phi_lin && a == g.phi_axis) ? T(sg) * k.phi_slope : T(0);
}
// a boundary x face of the fast path: 1 with its Dirichlet value in *v (as
// pois_nb), 0 for a face with no term
template <typename T>
__device__ __forceinline__ int pois_xface(const Geom &g, const Cst<T> &k, int x, int y, int z, int sg, T *v)
{
    const int face = sg > 0 ? 1 : 0;
    if (g.phi_kind[face] != ELBM_PHI_DIRICHLET) return 0;
    *v = g.phi_lin ? T(0) : phi_ghost<T>(g, k, face, x, y, z);
    return 1;
}

// phi_lin at the site (0 without the deviation form)
template <typename T>
__device__ __forceinline__ T phi_lin_at(const Geom &g, const Cst<T> &k, int x, int y, int z)
{
    if (!g.phi_lin) return T(0);
    const int c = g.phi_axis == 0 ? x : (g.phi_axis == 1 ? y : z);
    return k.phi_lo + T(c + 1) * k.phi_slope;
}

template <typename T> __device__ __forceinline__ T scal_of(const Bufs &b, int i);
template <> __device__ __forceinline__ double scal_of<double>(const Bufs &b, int i) { return b.scal[i]; }
template <> __device__ __forceinline__ float scal_of<float>(const Bufs &b, int i) { return b.scalf[i]; }

// ===========================================================================
// Initial state: f(r,0) = f^eq(rho0, u0) (Eq. 2) or the given f0, placed so
// that the first pull returns it (inverse of the streaming map). Inlet /
// outlet nodes hold their equilibria in A and B.
// ===========================================================================
template <int PR>
__global__ void k_init_pop(Geom g, Phys ph, Bufs b, const double *rho0, const double *u0,
                           const double *f0, const double *u_in, const double *q0)
{
    typedef Tr<PR> T;
    typedef typename T::st st;
    typedef typename T::sc sc;
    typedef typename T::gt gt;
    int x, y, z;
    bool inb;
    ll s;
    site_xyz(g, x, y, z, inb, s);
    if (!inb) return;
    unsigned char kind = b.mask ? b.mask[s] : 0;
    st *A = (st *)b.fA, *B = (st *)b.fB;
    sc *rho = (sc *)b.rho;
    // BF16 storage: the reference density of the values stored at a site is
    // its initial density (1 where none is given); inlet and outlet nodes
    // keep theirs
    auto rref_of = [&](ll i) -> double {
        if (b.mask && b.mask[i] == ELBM_NODE_INLET) return ph.rho_in;
        if (b.mask && b.mask[i] == ELBM_NODE_OUTLET) return ph.rho_out;
        return rho0 ? rho0[i] : 1.0;
    };
    auto stored = [&](double f, int p, ll at) -> st {
        if constexpr (T::rel) return from_ct<st>((typename T::ct)(f - wq(p) * rref_of(at)));
        else if constexpr (T::dev) return from_ct<st>((typename T::ct)(f - wq(p)));
        else return from_ct<st>((typename T::ct)f);
    };
    if constexpr (T::rel) {
        const float r0 = kind == ELBM_NODE_SOLID ? 1.f : float(rref_of(s));
        b.rA[s] = r0;
        b.rB[s] = r0;
    }
    if (kind == ELBM_NODE_SOLID) { rho[s] = sc(0); return; }
    if (kind == ELBM_NODE_INLET || kind == ELBM_NODE_OUTLET) {
        double r = kind == ELBM_NODE_INLET ? ph.rho_in : ph.rho_out;
        double ux = 0, uy = 0, uz = 0;
        if (kind == ELBM_NODE_INLET && u_in) { ux = u_in[3 * s]; uy = u_in[3 * s + 1]; uz = u_in[3 * s + 2]; }
        double usq = ux * ux + uy * uy + uz * uz;
#pragma unroll
        for (int p = 0; p < Q; p++) {
            double fe = wq(p) * r * (1.0 + Ppoly<double>(p, ux, uy, uz, usq));
            st v = stored(fe, p, s);
            A[(ll)p * g.N + s] = v;
            B[(ll)p * g.N + s] = v;
        }
        rho[s] = sc(r);
        return;
    }
    Nbr n;
    nbr_init(n, g, x, y, z, s);
    double ux = 0, uy = 0, uz = 0;
    if (u0) { ux = u0[3 * s]; uy = u0[3 * s + 1]; uz = u0[3 * s + 2]; }
    double usq = ux * ux + uy * uy + uz * uz;
#pragma unroll
    for (int p = 0; p < Q; p++) {
        double fp = f0 ? f0[(ll)p * g.N + s] : wq(p) * rho0[s] * (1.0 + Ppoly<double>(p, ux, uy, uz, usq));
        ll src = nbr_idx(n, g, -cx(p), -cy(p), -cz(p));
        unsigned char k2 = (src >= 0 && b.mask) ? b.mask[src] : 0;
        if (src < 0 || k2 == ELBM_NODE_SOLID) A[(ll)opp(p) * g.N + s] = stored(fp, p, s);
        else if (k2 == ELBM_NODE_FLUID) A[(ll)p * g.N + src] = stored(fp, p, src);
    }
    if (b.gA) {
        gt *GA = (gt *)b.gA;
        double qv = q0 ? q0[s] : 0.0;
#pragma unroll
        for (int i = 0; i < Q7; i++) {
            double cu = c7x(i) * ux + c7y(i) * uy + c7z(i) * uz;
            gt v = (gt)(w7(i) * qv * (1.0 + cu / CS2Q));
            ll src = nbr_idx(n, g, -c7x(i), -c7y(i), -c7z(i));
            unsigned char k2 = (src >= 0 && b.mask) ? b.mask[src] : 0;
            int io = i == 0 ? 0 : ((i & 1) ? i + 1 : i - 1);
            if (src < 0 || k2 == ELBM_NODE_SOLID) GA[(ll)io * g.N + s] = v;
            else if (k2 == ELBM_NODE_FLUID) GA[(ll)i * g.N + src] = v;
        }
    }
}

// ===========================================================================
// Moments: rho = sum_p f_p (Sec. II), and in transport mode q = sum_i g_i with
// the per-block sums of q and q^2 (neutralisation, Poisson reference norm).
// ===========================================================================
template <int PR>
__global__ void __launch_bounds__(128) k_moments(Geom g, Phys ph, Bufs b)
{
    typedef Tr<PR> T;
    typedef typename T::ct ct;
    typedef typename T::sc sc;
    typedef typename T::gt gt;
    int x, y, z;
    bool inb;
    ll s;
    site_xyz(g, x, y, z, inb, s);
    bool active = inb && (!b.mask || b.mask[s] == ELBM_NODE_FLUID);
    gt qv = 0, q2 = 0;
    if (active) {
        Nbr n;
        nbr_init(n, g, x, y, z, s);
        const unsigned bits = b.bbits ? b.bbits[s] : 0u;
        ct rs = 0, rs_lo = 0;
#pragma unroll
        for (int p = 0; p < Q; p++) {
            const ct v = gather_pop_b<PR>(g, b.fA, n, p, bits, b.rA);
            // deviations: a compensated sum (at the vapour density sum d ~ -0.84
            // and its rounding would be ~6x larger relative to rho ~ 0.16)
            if constexpr (T::dev) two_sum_acc(v, rs, rs_lo);
            else rs += v;
        }
        ((sc *)b.rho)[s] = sc(T::dev ? (ct(1) + rs) + rs_lo : rs);
        if (ph.charge_model == ELBM_CHARGE_TRANSPORT) {
            gt qs = 0;
#pragma unroll
            for (int i = 0; i < Q7; i++) qs += gather_g_b<PR>(g, b.gA, n, i, bits);
            ((sc *)b.q)[s] = sc(qs);
            qv = qs;
            q2 = qs * qs;
        }
    }
    if (inb) {
        // the per-site functions of rho that the collision takes at its
        // neighbours, at every node (inlet and outlet nodes keep their
        // prescribed density): psi of the Shan-Chen force, sigma of the
        // Ohmic current
        const Cst<ct> &k = cst<ct>(ph);
        const ct rv = ct(((const sc *)b.rho)[s]);
        ((sc *)b.psi)[s] = sc(psi_nb(rv, k.rho0, ct(-1.4426950408889634) * k.irho0));
        if (ph.charge_model == ELBM_CHARGE_TRANSPORT) ((sc *)b.sig)[s] = sc(sigma_of(k, rv));
    }
    if (ph.charge_model == ELBM_CHARGE_TRANSPORT) {
        gt v[2] = {qv, q2};
        block_sums<2>(v, b.part + block_id(), num_blocks());
    }
}

// ===========================================================================
// Free charge, Eqs. (surface-q2) / (surface-q3): lattice gradient of rho,
// interface normal, mean curvature K = -div n (positive on convex drops).
// A solid or out-of-domain neighbour takes the site's own value.
// ===========================================================================
template <int PR>
__global__ void __launch_bounds__(128) k_charge_grad(Geom g, Phys ph, Bufs b)
{
    typedef typename Tr<PR>::sc sc;
    int x, y, z;
    bool inb;
    ll s;
    site_xyz(g, x, y, z, inb, s);
    if (!inb) return;
    if (b.mask && b.mask[s] == ELBM_NODE_SOLID) return;
    Nbr n;
    nbr_init(n, g, x, y, z, s);
    const sc *rho = (const sc *)b.rho;
    // the neighbour r + c_p is beyond a wall face or solid exactly when the
    // pull of the opposite population bounces (bit opp(p) of the bounce bits)
    const unsigned bits = b.bbits ? b.bbits[s] : 0u;
    sc gx = 0, gy = 0, gz = 0;
#pragma unroll
    for (int p = 1; p < Q; p++) {
        const int nb = nbr_idx(n, g, cx(p), cy(p), cz(p));
        sc v = rho[((bits >> opp(p)) & 1u) ? n.s : nb];
        sc wv = sc(wq(p)) * v / sc(CS2);
        gx += wv * sc(cx(p));
        gy += wv * sc(cy(p));
        gz += wv * sc(cz(p));
    }
    sc g2 = gx * gx + gy * gy + gz * gz;
    sc gn = sqrt(g2);
    if (gn < sc(1e-12)) gn = sc(1e-12);
    sc *nh = (sc *)b.nh;
    nh[s] = gx / gn;
    nh[g.N + s] = gy / gn;
    nh[2 * g.N + s] = gz / gn;
    nh[3 * g.N + s] = g2;
}

template <int PR>
__global__ void __launch_bounds__(128) k_charge_ab(Geom g, Phys ph, Bufs b)
{
    // the xi form, Eq. (surface-q3), needs no global sum: the free charge
    // q = xi_b a + xi_s b is written here with its block sums (q, q^2), the
    // same values k_charge_q would form from the stored a and b
    const bool xi = ph.charge_model == ELBM_CHARGE_XI;
    typedef typename Tr<PR>::sc sc;
    int x, y, z;
    bool inb;
    ll s;
    site_xyz(g, x, y, z, inb, s);
    bool active = inb && (!b.mask || b.mask[s] == ELBM_NODE_FLUID);
    sc av = 0, bv = 0;
    if (active) {
        Nbr n;
        nbr_init(n, g, x, y, z, s);
        const sc *nh = (const sc *)b.nh;
        const unsigned bits = b.bbits ? b.bbits[s] : 0u;  // as in k_charge_grad
        sc div = 0;
#pragma unroll
        for (int p = 1; p < Q; p++) {
            const int nb = nbr_idx(n, g, cx(p), cy(p), cz(p));
            const int src = ((bits >> opp(p)) & 1u) ? n.s : nb;
            sc wv = sc(wq(p)) / sc(CS2);
            div += wv * (nh[src] * sc(cx(p)) + nh[g.N + src] * sc(cy(p)) + nh[2 * g.N + src] * sc(cz(p)));
        }
        sc K = -div;
        sc kp = K > sc(0) ? K : sc(0);
        sc r = ((const sc *)b.rho)[s];
        const Cst<sc> &k = cst<sc>(ph);
        av = r * sc(0.5) * (sc(1) + tanh((r - k.rho0) * k.itw));
        bv = nh[3 * g.N + s] * (sc(1) + sqrt(sqrt(kp * k.iKd)));
        if (!xi) {  // the conserved form scales a and b by global sums first (k_charge_q)
            sc *ab = (sc *)b.ab;
            ab[s] = av;
            ab[g.N + s] = bv;
        } else {
            const sc qv = k.xib * av + k.xis * bv;
            ((sc *)b.q)[s] = qv;
            av = qv;
            bv = qv * qv;
        }
    } else if (xi && inb) {
        ((sc *)b.q)[s] = sc(0);
    }
    sc v[2] = {av, bv};
    block_sums<2>(v, b.part + block_id(), num_blocks());
}

template <int PR>
__global__ void __launch_bounds__(128) k_charge_q(Geom g, Phys ph, Bufs b)
{
    typedef typename Tr<PR>::sc sc;
    int x, y, z;
    bool inb;
    ll s;
    site_xyz(g, x, y, z, inb, s);
    bool active = inb && (!b.mask || b.mask[s] == ELBM_NODE_FLUID);
    sc qv = 0;
    if (active) {
        const sc *ab = (const sc *)b.ab;
        const Cst<sc> &k = cst<sc>(ph);
        if (ph.charge_model == ELBM_CHARGE_CONSERVED) {
            // S_SA / S_SB slots hold Q_b / sum(a) and Q_s / sum(b) (0 for an empty sum)
            qv = scal_of<sc>(b, S_SA) * ab[s] + scal_of<sc>(b, S_SB) * ab[g.N + s];
        } else {
            qv = k.xib * ab[s] + k.xis * ab[g.N + s];
        }
        ((sc *)b.q)[s] = qv;
    } else if (inb) {
        ((sc *)b.q)[s] = sc(0);
    }
    sc v[2] = {qv, qv * qv};
    block_sums<2>(v, b.part + block_id(), num_blocks());
}

// ===========================================================================
// Poisson equation div(eps grad phi) = -(q - qmean) (Sec. II), eps = 1 +
// kappa rho/rho0, face permittivity the mean of the two sites: red-black SOR
// half-sweep over the sites of one colour, (x+y+z) mod 2 = color.
// ===========================================================================
template <int PR, int NC>
__global__ void __launch_bounds__(128) k_sor(Geom g, Phys ph, Bufs b, int color, int gauss_seidel)
{
    typedef typename Tr<PR>::sc sc;
    // red-black (NC = 2): one thread per site of the colour, x = 2 i + ((y +
    // z + color) & 1); three colours: one thread per site, those of the colour work
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    const int y = blockIdx.y * blockDim.y + threadIdx.y;
    const int z = blockIdx.z;
    const int x = NC == 3 ? i : 2 * i + ((y + z + color) & 1);
    if (x >= g.nx || y >= g.ny) return;
    if (NC == 3 && color3(g.per, x, y, z, g.nx, g.ny, g.nz) != color) return;
    const ll s = x + (ll)g.nx * (y + (ll)g.ny * z);
    unsigned char kind = b.mask ? b.mask[s] : 0;
    if (kind == ELBM_NODE_SOLID) return;
    const Cst<sc> &k = cst<sc>(ph);
    sc *phi = (sc *)b.phi;
    const sc *rho = (const sc *)b.rho;
    sc es = sc(1) + k.kap * rho[s];
    sc num = kind == ELBM_NODE_FLUID ? ((const sc *)b.q)[s] - scal_of<sc>(b, S_QMEAN) : sc(0);
    sc den = 0;
    int xn[2];
    if (pois_fast(g, b.mask, x, y, z, (int)s, xn)) {
        const int off[3] = {1, g.nx, g.nx * g.ny};
#pragma unroll
        for (int a = 0; a < 3; a++)
#pragma unroll
            for (int sg = -1; sg <= 1; sg += 2) {
                const int nb = a == 0 ? xn[sg > 0] : (int)s + sg * off[a];  // 32-bit site index (N < 2^31)
                // loads from a valid index whatever the face (the site itself
                // beyond a boundary x face), so none waits on the face test
                const int li = nb >= 0 ? nb : (int)s;
                const sc rn = rho[li], pn = phi[li];
                const sc dl = interior_dl<sc>(g, k, a, sg);
                if (nb >= 0) {
                    const sc ef = face_eps<sc>(es, sc(1) + k.kap * rn, ph.eps_face);
                    num += ef * (pn + dl);
                    den += ef;
                } else {
                    sc v = 0;
                    if (pois_xface<sc>(g, k, x, y, z, sg, &v)) {
                        num += es * (v + dl);
                        den += es;
                    }
                }
            }
    } else {
        Nbr n;
        nbr_init(n, g, x, y, z, s);
#pragma unroll
        for (int a = 0; a < 3; a++)
#pragma unroll
            for (int sg = -1; sg <= 1; sg += 2) {
                int nb = 0;
                sc v = 0, dl = 0;
                int kk = pois_nb<sc>(g, k, b.mask, n, x, y, z, a, sg, &nb, &v, &dl);
                if (kk == 0) {
                    sc ef = face_eps<sc>(es, sc(1) + k.kap * rho[nb], ph.eps_face);
                    num += ef * (phi[nb] + dl);
                    den += ef;
                } else if (kk == 1) {
                    num += es * (v + dl);
                    den += es;
                }
            }
    }
    if (!(den > sc(0))) return;
    if (gauss_seidel) phi[s] = pois_div(num, den);
    else phi[s] = (sc(1) - k.omega) * phi[s] + pois_div(k.omega * num, den);
}

// residual r = div(eps grad phi) + q - qmean with the reference norms:
// per-block sums of r^2, q^2 (fluid) and b^2 (Dirichlet data)
// The stop rule's sums at site (x, y, z), added to acc: r^2, q^2, b^2 and
// t^2, t = the magnitude of the terms of r (source and every face term with
// |phi| in place of its difference): the residual of a potential stored in
// FP32 cannot fall much below 2^-24 |t|
template <int PR>
__device__ __forceinline__ void resid_site(const Geom &g, const Phys &ph, const Bufs &b, int zc, int x, int y, int z,
                                           typename Tr<PR>::sc (&acc)[4])
{
    typedef typename Tr<PR>::sc sc;
    const ll s = x + (ll)g.nx * (y + (ll)g.ny * z);
    unsigned char kind = b.mask ? b.mask[s] : 0;
    if (kind != ELBM_NODE_SOLID) {
        const sc *phi = (const sc *)b.phi;
        const sc *rho = (const sc *)b.rho;
        const Cst<sc> &k = cst<sc>(ph);
        sc es = sc(1) + k.kap * rho[s];
        sc qs = kind == ELBM_NODE_FLUID ? ((const sc *)b.q)[s] : sc(0);
        sc r = kind == ELBM_NODE_FLUID ? qs - scal_of<sc>(b, S_QMEAN) : sc(0);
        sc bs = 0;
        sc ps = phi[s];
        sc t = fabs(r);
        int xn[2];
        sc tw = 1;  // weight of t^2 (see below)
        if (zc >= 0 && ((x + y + z) & 1) == zc && pois_fast(g, b.mask, x, y, z, (int)s, xn)) {
            // a site of the colour a Gauss-Seidel sweep has just updated: its
            // residual is the rounding of that update (the level the FP32
            // floor stop tolerates), taken as 0; only the Dirichlet data of a
            // row's end faces enter (the reference norm), and its |t| is
            // counted by the sites of the other colour (tw = 2 there)
            r = 0;
            t = 0;
#pragma unroll
            for (int sg = -1; sg <= 1; sg += 2) {
                sc v = 0;
                if (xn[sg > 0] < 0 && pois_xface<sc>(g, k, x, y, z, sg, &v))
                    bs += es * (v + interior_dl<sc>(g, k, 0, sg) + phi_lin_at<sc>(g, k, x, y, z));
            }
        } else if (pois_fast(g, b.mask, x, y, z, (int)s, xn)) {
            if (zc >= 0) tw = 2;
            const int off[3] = {1, g.nx, g.nx * g.ny};
#pragma unroll
            for (int a = 0; a < 3; a++)
#pragma unroll
                for (int sg = -1; sg <= 1; sg += 2) {
                    const int nb = a == 0 ? xn[sg > 0] : (int)s + sg * off[a];
                    const int li = nb >= 0 ? nb : (int)s;  // loads independent of the face test
                    const sc rn = rho[li], pn = phi[li];
                    const sc dl = interior_dl<sc>(g, k, a, sg);
                    if (nb >= 0) {
                        const sc cf = face_eps<sc>(es, sc(1) + k.kap * rn, ph.eps_face);
                        r += cf * ((pn + dl) - ps);
                        t += cf * (fabs(pn) + fabs(dl) + fabs(ps));
                    } else {
                        sc v = 0;
                        if (pois_xface<sc>(g, k, x, y, z, sg, &v)) {
                            r += es * ((v + dl) - ps);
                            bs += es * (v + dl + phi_lin_at<sc>(g, k, x, y, z));  // the Dirichlet datum itself
                            t += es * (fabs(v) + fabs(dl) + fabs(ps));
                        }
                    }
                }
        } else {
            Nbr n;
            nbr_init(n, g, x, y, z, s);
            const sc pl = phi_lin_at<sc>(g, k, x, y, z);
#pragma unroll
            for (int a = 0; a < 3; a++)
#pragma unroll
                for (int sg = -1; sg <= 1; sg += 2) {
                    int nb = 0;
                    sc v = 0, dl = 0;
                    int kk = pois_nb<sc>(g, k, b.mask, n, x, y, z, a, sg, &nb, &v, &dl);
                    if (kk == 0) {
                        const sc cf = face_eps<sc>(es, sc(1) + k.kap * rho[nb], ph.eps_face);
                        r += cf * ((phi[nb] + dl) - ps);
                        t += cf * (fabs(phi[nb]) + fabs(dl) + fabs(ps));
                    } else if (kk == 1) {
                        r += es * ((v + dl) - ps);
                        bs += es * (v + dl + pl);  // the Dirichlet datum itself (reference norm)
                        t += es * (fabs(v) + fabs(dl) + fabs(ps));
                    }
                }
        }
        acc[0] += r * r;
        acc[1] += qs * qs;
        acc[2] += bs * bs;
        acc[3] += tw * t * t;
    }
}

// per-block sums of r^2, q^2 (fluid), b^2 (Dirichlet data) and t^2, one
// thread per site
template <int PR>
__global__ void __launch_bounds__(128) k_resid(Geom g, Phys ph, Bufs b, int zc)
{
    typedef typename Tr<PR>::sc sc;
    int x, y, z;
    bool inb;
    ll s;
    site_xyz(g, x, y, z, inb, s);
    sc acc[4] = {0, 0, 0, 0};
    if (inb) resid_site<PR>(g, ph, b, zc, x, y, z, acc);
    block_sums<4>(acc, b.part + block_id(), num_blocks());
}

// The same sums with the colour zc settled (red-black, reduced precision):
// one thread per site of the other colour, x = 2 i + ((y + z + 1 - zc) & 1),
// which also takes its partner of colour zc in the same pair of x (the
// settled site costs its own q and the Dirichlet data of a row's end), so
// that no warp splits between the full and the settled sites.
template <int PR>
__global__ void __launch_bounds__(128) k_resid_pairs(Geom g, Phys ph, Bufs b, int zc)
{
    typedef typename Tr<PR>::sc sc;
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    const int y = blockIdx.y * blockDim.y + threadIdx.y;
    const int z = blockIdx.z;
    sc acc[4] = {0, 0, 0, 0};
    if (y < g.ny) {
        const int xa = 2 * i + ((y + z + 1 - zc) & 1), xb = 2 * i + ((y + z + zc) & 1);
        if (xa < g.nx) resid_site<PR>(g, ph, b, zc, xa, y, z, acc);
        if (xb < g.nx) resid_site<PR>(g, ph, b, zc, xb, y, z, acc);
    }
    block_sums<4>(acc, b.part + block_id(), num_blocks());
}

template <int PR>
__global__ void __launch_bounds__(128) k_phi_sum(Geom g, Phys ph, Bufs b)
{
    typedef typename Tr<PR>::sc sc;
    int x, y, z;
    bool inb;
    ll s;
    site_xyz(g, x, y, z, inb, s);
    bool active = inb && (!b.mask || b.mask[s] != ELBM_NODE_SOLID);
    sc v[1] = {active ? ((const sc *)b.phi)[s] : sc(0)};
    block_sums<1>(v, b.part + block_id(), num_blocks());
}

template <int PR>
__global__ void k_phi_shift(Geom g, Bufs b)
{
    typedef typename Tr<PR>::sc sc;
    int x, y, z;
    bool inb;
    ll s;
    site_xyz(g, x, y, z, inb, s);
    if (!inb || (b.mask && b.mask[s] == ELBM_NODE_SOLID)) return;
    ((sc *)b.phi)[s] -= scal_of<sc>(b, S_PHIMEAN);
}

// ===========================================================================
// The fused site update, Eq. (lattice-b): pull f; Shan-Chen force Eq. (sc);
// E = -grad phi + E_ext, F_el = q E; f^eq Eq. (2); alpha Eq. (entropic);
// stress Eq. (stress) and its 2-norm; Carreau viscosity Eqs. (strain2),
// (carreau), (beta); exact-difference source Eq. (add); write f*; in
// transport mode the D3Q7 charge update. Optional diagnostics per block.
// ===========================================================================
// Guarded FP32 alpha: lanes whose root needs the float-float guard queue their
// inputs in shared memory; after a barrier the block's threads run the
// queued guards together, L lanes per site (L = 8, 4, 2 or 1 for up to 16,
// 32, 64 or 128 sites: full warps instead of a few lanes in many warps), and
// the results return through the queue. The queue holds one entry per
// thread of the block (the kernel is launched with 128 threads).
constexpr int kGuardQ = 128;
struct GuardEntry {
    float dev[Q];     // the site's FP32 deviations d_p = f_p - w_p (the exact inputs)
    float Dh[Q], Dl[Q];  // scratch: the exact Delta as pairs (filled by the guard)
    float a, S, amax;
    float4 res;
};

// Learned mode (LRN): the proposal's network runs inside the collision, only
// in the warps that hold a site whose Newton iteration starts from it (S >=
// 2^-5), with the weights loaded only by blocks that have one; its tiles use
// the shared memory that the guard queue takes afterwards.
struct MlpTiles {
    MlpSmem sm;
    __nv_bfloat16 xs[4][32 * MLP_XS];
    float os[4][32];
};
// a call, not inlined: the network's fragments stay out of the collision's
// register allocation, and warps without such a site never enter it
static __device__ __noinline__ void mlp_warp_call(const MlpSmem *sm, const __nv_bfloat16 *xs, float *o)
{
    mlp_warp_bf16(*sm, xs, o);
}

template <int PR, int AP, bool LRN>
__global__ void __launch_bounds__(128, (PR == ELBM_PREC_FP64 || AP == ELBM_APREC_FP64) ? 1 : 5) k_collide(Geom g, Phys ph, Bufs b, int diag)
{
    typedef Tr<PR> T;
    typedef typename T::ct ct;
    typedef typename T::sc sc;
    typedef typename T::st st;
    typedef typename T::gt gt;
    constexpr bool kQueue = AP == ELBM_APREC_FP32 && sizeof(ct) == 4;
    static_assert(!LRN || (sizeof(ct) == 4 && AP != ELBM_APREC_FP64), "the learned start needs FP32 arithmetic");
    constexpr size_t kQBytes = sizeof(GuardEntry) * (kQueue ? kGuardQ : 1);
    constexpr size_t kSmem = (LRN && sizeof(MlpTiles) > kQBytes) ? sizeof(MlpTiles) : kQBytes;
    __shared__ __align__(16) unsigned char smem[kSmem];
    GuardEntry *gq = reinterpret_cast<GuardEntry *>(smem);
    __shared__ int gq_n;
    const int tid = threadIdx.x + blockDim.x * threadIdx.y;
    if (kQueue) {
        if (tid == 0) gq_n = 0;
        __syncthreads();
    }
    int x, y, z;
    bool inb;
    ll s;
    site_xyz(g, x, y, z, inb, s);
    const bool active = inb && (!b.mask || b.mask[s] == ELBM_NODE_FLUID);
    ct dm = 0, dmx = 0, dmy = 0, dmz = 0, dq = 0, dasum = 0;
    unsigned dnfl = 0, dsh = 0, dnr = 0, dcl = 0, dbad = 0, dgd = 0, dgf = 0, dlf = 0;
    float damin = 1e30f, damax = -1e30f, dherr = 0.f, dumax = 0.f;
    float sherr = 0.f;   // a step without diagnostics: the site's H-error and
    unsigned sflag = 0;  // flags (1 non-finite or non-positive density, 2 guard failure)
    // the first part's results, carried across the block-level guard section
    Nbr n;
    ct f[Q], D[Q];
    ct r = 0, drho = 0, jx = 0, jy = 0, jz = 0, Fx = 0, Fy = 0, Fz = 0, qs = 0;
    ct ir = 0, ux = 0, uy = 0, uz = 0, usq = 0, Rq = 0;
    float esum = 0.f;  // rounding scale of the FP32 momentum (deviation modes)
    ct uin_v = 0;      // adaptive inlet: u . d at a region site
    ct alpha = ct(2);
    float alpha_lo = 0.f;  // low part of a guarded root
    // FP32 alpha: its setup (carried across the network's barrier in learned mode)
    AlphaSetupF ast;
    bool need_mlp = false;
    float a_herr = 0.f;
    int a_status = 0, a_guard = 0, a_lfall = 0;
    int gslot = -1;
    // the FP32 Newton root from a_start (< 0: the moment-series start); a
    // lane whose root needs the float-float guard queues its inputs
    // (deviation modes: f holds d_p, D the FP32 Delta)
    auto solve_alpha = [&](float a_start) {
        if constexpr (sizeof(ct) == 4) {
            float ff[Q];  // the FP32 populations w + d
#pragma unroll
            for (int p = 0; p < Q; p++) ff[p] = float(wq(p)) + f[p];
            if constexpr (LRN) {  // x_p = Delta_p / f_p again, rather than kept across the barrier
#pragma unroll
                for (int p = 0; p < Q; p++) ast.x[p] = __fdividef(D[p], ff[p]);
            }
            AlphaOutF ao = alpha_fp32_solve(ff, D, f, float(r), ast, AP == ELBM_APREC_FP32, a_start, kQueue, ph.cf.htol);
            alpha = ct(ao.alpha);
            alpha_lo = ao.alpha_lo;
            a_herr = ao.herr;
            a_status = ao.status;
            a_guard = ao.guarded;
            a_lfall = LRN && ao.status == 0 && ao.iters > 1;
            if (kQueue && ao.guarded == 2) {
                a_guard = 1;
                gslot = atomicAdd(&gq_n, 1);  // < kGuardQ: one entry per thread
                GuardEntry &e = gq[gslot];
#pragma unroll
                for (int p = 0; p < Q; p++) e.dev[p] = f[p];
                e.a = ao.alpha;
                e.amax = ast.amax;
                e.S = ast.S;
            }
        }
    };
    if (active) {
        nbr_init(n, g, x, y, z, s);
        const sc *phi = (const sc *)b.phi;
#pragma unroll
        for (int p = 0; p < Q; p++) f[p] = gather_pop<PR>(g, b.mask, b.fA, n, p, b.rA);
        ct rs = 0, rs_lo = 0;  // deviations: sum d_p compensated (Delta below)
        if constexpr (T::dev) {
            // compensated density, momentum from opposite-link differences
            moments_dev(f, rs, rs_lo, jx, jy, jz, esum);
        } else {
#pragma unroll
            for (int p = 0; p < Q; p++) {
                rs += f[p];
                jx += ct(cx(p)) * f[p];
                jy += ct(cy(p)) * f[p];
                jz += ct(cz(p)) * f[p];
            }
        }
        r = T::dev ? ct(1) + rs : rs;
        drho = T::dev ? rs : rs - ct(1);

        const Cst<ct> &k = cst<ct>(ph);
        // Eq. (sc): F_int = -G psi(r) sum_fluid w psi(r+c) c - G_w psi(r) sum_wall w psi(r) c
        const ct rho0 = k.rho0;
        const ct ps = psi_of<ct>(r, rho0);
        const sc *psi = (const sc *)b.psi;
        ct sfx = 0, sfy = 0, sfz = 0, swx = 0, swy = 0, swz = 0;
#pragma unroll
        for (int p = 1; p < Q; p++) {
            const int nb = nbr_idx(n, g, cx(p), cy(p), cz(p));
            bool wall = nb < 0 || (b.mask && b.mask[nb] == ELBM_NODE_SOLID);
            ct wv = ct(wq(p)) * (wall ? ps : ct(psi[nb]));
            if (wall) { swx += wv * ct(cx(p)); swy += wv * ct(cy(p)); swz += wv * ct(cz(p)); }
            else { sfx += wv * ct(cx(p)); sfy += wv * ct(cy(p)); sfz += wv * ct(cz(p)); }
        }
        Fx = -k.G * ps * sfx - k.Gw * ps * swx;
        Fy = -k.G * ps * sfy - k.Gw * ps * swy;
        Fz = -k.G * ps * sfz - k.Gw * ps * swz;

        // electric force q E, E = -grad phi (central differences) + E_ext; in
        // transport mode the same face neighbours give the Ohmic source
        // R = div(sigma grad phi) of the charge update
        if (ph.charge_model != ELBM_CHARGE_NONE) {
            qs = ct(((const sc *)b.q)[s]);
            ct E[3];
            const ct phs = ct(phi[s]);
            const bool tr = ph.charge_model == ELBM_CHARGE_TRANSPORT;
            const sc *sig = (const sc *)b.sig;
            const ct ss = tr ? ct(sig[s]) : ct(0);
#pragma unroll
            for (int a = 0; a < 3; a++) {
                ct pv[2];
#pragma unroll
                for (int kk = 0; kk < 2; kk++) {
                    int nb = 0;
                    ct v = 0, dl = 0;
                    int kind = pois_nb<ct>(g, k, b.mask, n, x, y, z, a, kk ? 1 : -1, &nb, &v, &dl);
                    pv[kk] = kind == 0 ? ct(phi[nb]) + dl : (kind == 1 ? v + dl : phs);
                    if (tr) {
                        if (kind == 0) Rq += ct(0.5) * (ss + ct(sig[nb])) * (pv[kk] - phs);
                        else if (kind == 1) Rq += ss * (pv[kk] - phs);
                    }
                }
                E[a] = -(pv[1] - pv[0]) * ct(0.5) + k.E[a];
            }
            Fx += qs * E[0];
            Fy += qs * E[1];
            Fz += qs * E[2];
        }
        if (ph.force_el == ELBM_FEL_FULL) {
            // Eq. (force_el2): + (eps - 1)/2 grad|E|^2, central differences of
            // the E2 plane; a neighbour that is not fluid (or beyond a wall)
            // takes the site's own |E|^2
            const sc *E2 = (const sc *)b.E2;
            const ct e2s = ct(E2[s]);
            ct gE[3];
#pragma unroll
            for (int a = 0; a < 3; a++) {
                ct ev[2];
#pragma unroll
                for (int kk = 0; kk < 2; kk++) {
                    const int nb = nbr_idx(n, g, a == 0 ? (kk ? 1 : -1) : 0, a == 1 ? (kk ? 1 : -1) : 0,
                                           a == 2 ? (kk ? 1 : -1) : 0);
                    const bool own = nb < 0 || (b.mask && b.mask[nb] != ELBM_NODE_FLUID);
                    ev[kk] = own ? e2s : ct(E2[nb]);
                }
                gE[a] = (ev[1] - ev[0]) * ct(0.5);
            }
            const ct h = ct(0.5) * (k.kap * r);  // (eps - 1)/2, eps = 1 + kappa rho
            Fx += h * gE[0];
            Fy += h * gE[1];
            Fz += h * gE[2];
        }

        // Eq. (2) at the bare velocity, Delta = f^eq - f
        ir = ct(1) / r;
        ux = jx * ir; uy = jy * ir; uz = jz * ir;
        usq = ux * ux + uy * uy + uz * uz;
        if constexpr (T::dev) {
            delta_dev(f, drho, rs_lo, r, ux, uy, uz, usq, D);
        } else {
#pragma unroll
            for (int p = 0; p < Q; p++) D[p] = ct(wq(p)) * r * (ct(1) + Ppoly<ct>(p, ux, uy, uz, usq)) - f[p];
        }

        // Eq. (entropic)
        if (ph.alpha_mode != ELBM_ALPHA_BGK) {
            if constexpr (sizeof(ct) == 8 || AP == ELBM_APREC_FP64) {
                double fd[Q], dd[Q];
#pragma unroll
                for (int p = 0; p < Q; p++) {
                    fd[p] = T::dev ? wq(p) + double(f[p]) : double(f[p]);
                    dd[p] = double(D[p]);
                }
                AlphaOut ao = alpha_fp64(fd, dd, double(r), ph.cd.eq_tol);
                alpha = ct(ao.alpha);
                a_herr = float(ao.herr);
                a_status = ao.status;
            } else {
                float ff[Q];  // the FP32 populations w + d
#pragma unroll
                for (int p = 0; p < Q; p++) ff[p] = float(wq(p)) + f[p];
                const float umax = fmaxf(fabsf(float(ux)), fmaxf(fabsf(float(uy)), fabsf(float(uz))));
                alpha_fp32_setup(ff, D, f, float(r), float(drho), ph.cf.eq_tol,
                                 u_err_bound(esum, float(r), umax), umax, ast);
                if constexpr (LRN) {
                    // the proposal alpha_c + S^3 o is the start where S >= 2^-5
                    need_mlp = ast.status == 0 && ast.S >= 0x1p-5f;
                    if (need_mlp)
                        mlp_site_features(ast.x, ast.S, reinterpret_cast<MlpTiles *>(smem)->xs[tid >> 5] +
                                                            (tid & 31) * MLP_XS);
                } else {
                    solve_alpha(-1.f);
                }
            }
        }
    }
    if constexpr (LRN) {
        // the block's sites that start from the proposal: the network for
        // the warps that hold one
        MlpTiles &mt = *reinterpret_cast<MlpTiles *>(smem);
        float o = 0.f;
        if (__syncthreads_or(need_mlp ? 1 : 0)) {
            const uint4 *src = (const uint4 *)b.mlpimg;
            uint4 *dst = (uint4 *)&mt.sm;
            for (int i = tid; i < (int)(sizeof(MlpSmem) / 16); i += blockDim.x * blockDim.y) dst[i] = src[i];
            __syncthreads();
            if (__any_sync(0xffffffffu, need_mlp)) {
                __nv_bfloat16 *row = mt.xs[tid >> 5] + (tid & 31) * MLP_XS;
                if (!need_mlp)
#pragma unroll
                    for (int c = 0; c < 32; c += 2) *reinterpret_cast<unsigned *>(row + c) = 0u;
                __syncwarp();
                mlp_warp_call(&mt.sm, mt.xs[tid >> 5], mt.os[tid >> 5]);
                o = mt.os[tid >> 5][tid & 31];
            }
        }
        __syncthreads();  // the tiles' memory becomes the guard queue
        if (active && ph.alpha_mode != ELBM_ALPHA_BGK)
            solve_alpha(need_mlp ? ast.ac + ast.S * ast.S * ast.S * o : -1.f);
    }
    if (kQueue) {
        static_assert(!kQueue || kGuardQ >= 128, "one guard-queue entry per thread of a 128-thread block");
        __syncthreads();
        const int nq = gq_n;
        // L lanes per queued site (the fewer the sites, the more lanes each),
        // as many as the block's threads cover (blocks of 96 threads when a
        // row of 65..96 sites is one block row)
        const int nthr = blockDim.x * blockDim.y;
        const int lg = 8 * nq <= nthr ? 3 : (4 * nq <= nthr ? 2 : (2 * nq <= nthr ? 1 : 0));
        const int site = tid >> lg, j = tid & ((1 << lg) - 1);
        if (site < nq) {
            GuardEntry &e = gq[site];
            const float4 gr = alpha_guard(e.dev, e.Dh, e.Dl, e.a, e.S, e.amax, ph.cf.htol, j, 1 << lg);
            if (j == 0) gq[site].res = gr;
        }
        __syncthreads();
        if (gslot >= 0) {
            const float4 gr = gq[gslot].res;
            alpha = ct(gr.x);
            alpha_lo = gr.y;
            if (gr.w == 0.f) a_status = 4;  // not certified: the FP32 report stays
            else a_herr = gr.z;
            if (gr.w >= 2.f) a_status = int(gr.w);  // no root (alpha = 2) / clipped
        }
    }
    if (active) {
        const Cst<ct> &k = cst<ct>(ph);
        // Eq. (stress): Pi = sum (f - f^eq) c c = -sum D c c; 2-norm; Carreau; Eq. (beta)
        ct nu = k.nu0;
        if (!ph.newtonian) {
            ct pxx = 0, pyy = 0, pzz = 0, pxy = 0, pxz = 0, pyz = 0;
#pragma unroll
            for (int p = 1; p < Q; p++) {
                pxx -= D[p] * ct(cx(p) * cx(p));
                pyy -= D[p] * ct(cy(p) * cy(p));
                pzz -= D[p] * ct(cz(p) * cz(p));
                pxy -= D[p] * ct(cx(p) * cy(p));
                pxz -= D[p] * ct(cx(p) * cz(p));
                pyz -= D[p] * ct(cy(p) * cz(p));
            }
#ifdef ELBM_D2Q9
            // a set without z links leaves the stress 2x2: max |eigenvalue| = |mean| + radius
            (void)pzz; (void)pxz; (void)pyz;
            const ct hm = ct(0.5) * (pxx + pyy), hd = ct(0.5) * (pxx - pyy);
            ct Pn = fabs(hm) + sqrt(hd * hd + pxy * pxy);
#else
            ct Pn = sym3_norm2<ct>(pxx, pyy, pzz, pxy, pxz, pyz);
#endif
            if (ph.carreau_lagged) {
                const ct np = ct(((const sc *)b.nu)[s]);  // 0 before the first step: nu0
                nu = carreau_nu_lagged<ct>(k, Pn, alpha, r, np > ct(0) ? np : k.nu0);
            } else {
                nu = carreau_nu<ct>(k, false, Pn, alpha, r);
            }
        }
        if (ph.carreau_lagged && !ph.store_macro) ((sc *)b.nu)[s] = sc(nu);  // for the next step
        const ct beta = ct(CS2) / (ct(2) * nu + ct(CS2));
        const ct ab = alpha * beta;

        // Eq. (add): S = f^eq(rho, u + F/rho) - f^eq(rho, u); Eq. (lattice-b)
        const ct vx = ux + Fx * ir, vy = uy + Fy * ir, vz = uz + Fz * ir;
        const ct vsq = vx * vx + vy * vy + vz * vz;
#pragma unroll
        for (int p = 0; p < Q; p++) {
            ct Sp = ct(wq(p)) * r * (Ppoly<ct>(p, vx, vy, vz, vsq) - Ppoly<ct>(p, ux, uy, uz, usq));
            ct fo = f[p] + ab * D[p] + Sp;
            // (BF16: relative to r - 1 as the reader forms it from the stored r)
            plane<st>(b.fB, p, g.N)[n.s] = stp<PR>(fo, p, r - ct(1));
        }
        if constexpr (T::rel) b.rB[n.s] = float(r);

        // half-step velocity (Sec. II): rho u = sum f c + F/2
        const ct upx = (jx + ct(0.5) * Fx) * ir, upy = (jy + ct(0.5) * Fy) * ir, upz = (jz + ct(0.5) * Fz) * ir;
        if (b.region && b.region[s])  // adaptive inlet: this site's velocity along the inlet direction
            uin_v = upx * ct(ph.in_d[0]) + upy * ct(ph.in_d[1]) + upz * ct(ph.in_d[2]);

        if (ph.charge_model == ELBM_CHARGE_TRANSPORT) {
            // D3Q7 advection-diffusion of q with the Ohmic source R (above)
            const ct R = Rq;
            const ct itq = k.itau_q;
#pragma unroll
            for (int i = 0; i < Q7; i++) {
                ct gi = ct(gather_g<PR>(g, b.mask, b.gA, n, i));
                ct cu = ct(c7x(i)) * upx + ct(c7y(i)) * upy + ct(c7z(i)) * upz;
                ct geq = ct(w7(i)) * qs * (ct(1) + cu / ct(CS2Q));
                plane<gt>(b.gB, i, g.N)[n.s] = gt(gi - (gi - geq) * itq + ct(w7(i)) * R);
            }
        }

        if (ph.store_macro) {
            ((sc *)b.ux)[s] = sc(upx);
            ((sc *)b.uy)[s] = sc(upy);
            ((sc *)b.uz)[s] = sc(upz);
            ((sc *)b.alpha)[s] = sc(alpha);
            if (b.alpha_lo) b.alpha_lo[s] = alpha_lo;  // the guarded root as a pair
            ((sc *)b.nu)[s] = sc(nu);
        }
        if (diag) {
            dm = r;
            dmx = jx + ct(0.5) * Fx;
            dmy = jy + ct(0.5) * Fy;
            dmz = jz + ct(0.5) * Fz;
            dq = qs;
            dasum = alpha;
            dnfl = 1;
            damin = damax = float(alpha);
            if (a_status == 1) dsh = 1;
            else if (a_status == 2) dnr = 1;
            else if (a_status == 3) dcl = 1;
            else if (a_status == 4) dgf = 1;
            dgd = a_guard;
            dlf = a_lfall;
            dherr = a_herr;
            const float um2 = float(upx * upx + upy * upy + upz * upz);  // |u|^2; the root once per block
            dumax = um2;
            if (!(r > ct(0)) || !isfinite(float(r)) || !isfinite(um2) || !isfinite(float(alpha))) dbad = 1;
        } else {
            sherr = a_herr;
            const float um2 = float(upx * upx + upy * upy + upz * upz);
            if (!(r > ct(0)) || !isfinite(float(r)) || !isfinite(um2) || !isfinite(float(alpha))) sflag = 1u;
            if (a_status == 4) sflag |= 2u;
        }
    }
    if (!diag) {
        // a step without diagnostics still keeps the sticky record that the
        // next diagnostics fold in: one warp-wide maximum of the H-error (as
        // its order-preserving integer) and one OR of the flags, each a
        // single reduction into the record per warp
        const int hw = __reduce_max_sync(0xffffffffu, float_ord(sherr, 0.f));
        const unsigned fw = __reduce_or_sync(0xffffffffu, sflag);
        if ((tid & 31) == 0) {
            if (hw > 0) atomicMax(reinterpret_cast<int *>(b.sticky), hw);
            if (fw) atomicOr(b.sticky + 1, fw);
        }
    }
    if (b.region) {  // adaptive inlet, every step: block sums of u . d over the region
        ct v[1] = {uin_v};
        block_sums<1>(v, b.part + (ll)D_UIN * num_blocks() + block_id());
    }
    if (diag) {
        // sums: compensated FP32 (or FP64) block sums; the five 0/1 counts
        // packed 6 bits each (a warp count is at most 32) into one integer
        // warp reduction; extrema by shuffles
        ct v[6] = {dm, dmx, dmy, dmz, dq, dasum};
        __shared__ double res[6];
        __shared__ float mm[4][8];
        __shared__ unsigned cn[2][8];
        const int tid = threadIdx.x + blockDim.x * threadIdx.y;
        const int lane = tid & 31, wid = tid >> 5;
        unsigned packed = dsh | (dnr << 6) | (dcl << 12) | (dbad << 18) | (dnfl << 24);
        packed = __reduce_add_sync(0xffffffffu, packed);
        unsigned packed2 = __reduce_add_sync(0xffffffffu, dgd | (dgf << 6) | (dlf << 12));
        // extrema as order-preserving integers (NaN lanes left out), one
        // warp-wide integer min/max each
        damin = ord_float(__reduce_min_sync(0xffffffffu, float_ord(damin, 1e30f)));
        damax = ord_float(__reduce_max_sync(0xffffffffu, float_ord(damax, -1e30f)));
        dherr = ord_float(__reduce_max_sync(0xffffffffu, float_ord(dherr, 0.f)));
        dumax = ord_float(__reduce_max_sync(0xffffffffu, float_ord(dumax, 0.f)));
        if (lane == 0) {
            mm[0][wid] = damin; mm[1][wid] = damax; mm[2][wid] = dherr; mm[3][wid] = dumax;
            cn[0][wid] = packed;
            cn[1][wid] = packed2;
        }
        block_sums<6>(v, res);
        __syncthreads();
        // thread j writes column j of the block's partials (one lane each,
        // so the block does not wait on one thread's serial loop)
        if (tid < D_NPART) {
            const int j = tid;
            const int nw = (blockDim.x * blockDim.y + 31) >> 5;
            double val;
            if (j <= D_Q || j == D_ASUM) {
                val = res[j == D_ASUM ? 5 : j];
            } else if (j == D_AMIN || j == D_AMAX || j == D_HERR || j == D_UMAX) {
                const int m = j == D_AMIN ? 0 : (j == D_AMAX ? 1 : (j == D_HERR ? 2 : 3));
                float e = mm[m][0];
                for (int i = 1; i < nw; i++) e = m == 0 ? fminf(e, mm[m][i]) : fmaxf(e, mm[m][i]);
                val = m == 3 ? sqrt(double(e)) : double(e);
            } else {
                const int word = j >= D_NGUARD ? 1 : 0;
                const int field = word ? j - D_NGUARD
                                       : (j == D_NBAD ? 3 : (j == D_NFLUID ? 4 : j - D_NSHORT));
                unsigned c = 0;
                for (int i = 0; i < nw; i++) c += (cn[word][i] >> (6 * field)) & 63u;
                val = double(c);
            }
            b.part[(ll)j * num_blocks() + block_id()] = val;
        }
    }
}

// Adaptive inlet: f^eq(rho_in, r u0) of every inlet node, r the scale that
// the finalize derived from the nozzle mean, stored as k_init_pop stores it,
// into B (the buffer the next step pulls from)
template <int PR>
__global__ void k_inlet_update(Geom g, Phys ph, Bufs b, const double *scal)
{
    typedef Tr<PR> T;
    typedef typename T::st st;
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= ph.n_inlet) return;
    const ll i = b.inlet_idx[t];
    const double r = scal[S_INRATIO];
    const double ux = r * b.inlet_u0[3 * t], uy = r * b.inlet_u0[3 * t + 1], uz = r * b.inlet_u0[3 * t + 2];
    const double usq = ux * ux + uy * uy + uz * uz;
    st *B = (st *)b.fB;
#pragma unroll
    for (int p = 0; p < Q; p++) {
        const double fe = wq(p) * ph.rho_in * (1.0 + Ppoly<double>(p, ux, uy, uz, usq));
        st v;
        if constexpr (T::rel) v = from_ct<st>((typename T::ct)(fe - wq(p) * ph.rho_in));
        else if constexpr (T::dev) v = from_ct<st>((typename T::ct)(fe - wq(p)));
        else v = from_ct<st>((typename T::ct)fe);
        B[(ll)p * g.N + i] = v;
    }
}

// |E|^2 of every site for the FULL electric force, E = -grad phi (central
// differences, the collision's stencil) + E_ext; 0 at nodes that are not fluid
template <int PR>
__global__ void __launch_bounds__(128) k_efield2(Geom g, Phys ph, Bufs b)
{
    typedef Tr<PR> T;
    typedef typename T::ct ct;
    typedef typename T::sc sc;
    int x, y, z;
    bool inb;
    ll s;
    site_xyz(g, x, y, z, inb, s);
    if (!inb) return;
    ct e2 = 0;
    if (!b.mask || b.mask[s] == ELBM_NODE_FLUID) {
        const Cst<ct> &k = cst<ct>(ph);
        Nbr n;
        nbr_init(n, g, x, y, z, s);
        const sc *phi = (const sc *)b.phi;
        const ct phs = ct(phi[s]);
#pragma unroll
        for (int a = 0; a < 3; a++) {
            ct pv[2];
#pragma unroll
            for (int kk = 0; kk < 2; kk++) {
                int nb = 0;
                ct v = 0, dl = 0;
                const int kind = pois_nb<ct>(g, k, b.mask, n, x, y, z, a, kk ? 1 : -1, &nb, &v, &dl);
                pv[kk] = kind == 0 ? ct(phi[nb]) + dl : (kind == 1 ? v + dl : phs);
            }
            const ct E = -(pv[1] - pv[0]) * ct(0.5) + k.E[a];
            e2 += E * E;
        }
    }
    ((sc *)b.E2)[s] = sc(e2);
}

// Warm start of the Poisson solve by linear extrapolation in time,
// phi <- 2 phi(t-1) - phi(t-2); the first call (no phi(t-2) yet, flag set by
// the following pre-solve test) only records phi(t-1). Solid (conductor)
// nodes hold a constant, which the extrapolation keeps.
// It also opens the step's Poisson loop, which then runs as do-while (no
// test before the first unit): unit counter 0, no previous residual.
template <typename T>
__global__ void k_phi_extrap(T *__restrict__ phi, T *__restrict__ phi_old, double *__restrict__ scal, ll N)
{
    const ll i = (ll)blockIdx.x * blockDim.x + threadIdx.x;
    if (i == 0) {
        scal[S_ITER] = 0.0;
        scal[S_PREV] = 1e300;
    }
    if (i >= N) return;
    const T p = phi[i];
    if (scal[S_HAVE_OLD] != 0.0) phi[i] = T(2) * p - phi_old[i];
    phi_old[i] = p;
}

// f(r, t) for the caller: the pull of every fluid site, 0 elsewhere
template <int PR>
__global__ void k_export_pop(Geom g, Bufs b, double *out)
{
    typedef Tr<PR> T;
    int x, y, z;
    bool inb;
    ll s;
    site_xyz(g, x, y, z, inb, s);
    if (!inb) return;
    bool fluid = !b.mask || b.mask[s] == ELBM_NODE_FLUID;
    Nbr n;
    nbr_init(n, g, x, y, z, s);
#pragma unroll
    for (int p = 0; p < Q; p++) {
        double v = 0.0;
        if (fluid) {
            double fv = double(gather_pop<PR>(g, b.mask, b.fA, n, p, b.rA));
            v = T::dev ? wq(p) + fv : fv;
        }
        out[(ll)p * g.N + s] = v;
    }
}

template <int PR>
__global__ void k_export_gpop(Geom g, Bufs b, double *out)
{
    int x, y, z;
    bool inb;
    ll s;
    site_xyz(g, x, y, z, inb, s);
    if (!inb) return;
    bool fluid = !b.mask || b.mask[s] == ELBM_NODE_FLUID;
    Nbr n;
    nbr_init(n, g, x, y, z, s);
#pragma unroll
    for (int i = 0; i < Q7; i++)
        out[(ll)i * g.N + s] = fluid ? double(gather_g<PR>(g, b.mask, b.gA, n, i)) : 0.0;
}

template <typename S>
__global__ void k_to_double(const S *in, double *out, ll n)
{
    ll i = blockIdx.x * (ll)blockDim.x + threadIdx.x;
    if (i < n) out[i] = double(in[i]);
}

template <typename S>
__global__ void k_add_lo(const S *lo, double *out, ll n)
{
    ll i = blockIdx.x * (ll)blockDim.x + threadIdx.x;
    if (i < n) out[i] += double(lo[i]);
}

// ---------------------------------------------------------------------------
// Host launchers for one precision.
// ---------------------------------------------------------------------------
template <int PR>
struct Launchers {
    typedef typename Tr<PR>::sc sc;
    static void init_pop(const Geom &g, const Phys &ph, const Bufs &b, const double *rho0,
                         const double *u0, const double *f0, const double *u_in, const double *q0,
                         const Launch &L, cudaStream_t s)
    {
        k_init_pop<PR><<<L.grid, L.block, 0, s>>>(g, ph, b, rho0, u0, f0, u_in, q0);
    }
    static void moments(const Geom &g, const Phys &ph, const Bufs &b, const Launch &L, cudaStream_t s)
    {
        k_moments<PR><<<L.grid, L.block, 0, s>>>(g, ph, b);
    }
    static void charge(const Geom &g, const Phys &ph, const Bufs &b, int stage, const Launch &L, cudaStream_t s)
    {
        if (stage == 0) {
            k_charge_grad<PR><<<L.grid, L.block, 0, s>>>(g, ph, b);
            k_charge_ab<PR><<<L.grid, L.block, 0, s>>>(g, ph, b);
        } else {
            k_charge_q<PR><<<L.grid, L.block, 0, s>>>(g, ph, b);
        }
    }
    static void sor(const Geom &g, const Phys &ph, const Bufs &b, int color, const Launch &L, cudaStream_t s)
    {
        if (g.ncol == 3) k_sor<PR, 3><<<L.grid, L.block, 0, s>>>(g, ph, b, color, 0);
        else k_sor<PR, 2><<<L.grid, L.block, 0, s>>>(g, ph, b, color, 0);
    }
    static void resid(const Geom &g, const Phys &ph, const Bufs &b, int zc, const Launch &L, cudaStream_t s)
    {
        if (zc >= 0) k_resid_pairs<PR><<<L.grid, L.block, 0, s>>>(g, ph, b, zc);  // L: the half-row shape
        else k_resid<PR><<<L.grid, L.block, 0, s>>>(g, ph, b, zc);
    }
    static void phi_mean(const Geom &g, const Phys &ph, const Bufs &b, int stage, const Launch &L, cudaStream_t s)
    {
        if (stage == 0) k_phi_sum<PR><<<L.grid, L.block, 0, s>>>(g, ph, b);
        else k_phi_shift<PR><<<L.grid, L.block, 0, s>>>(g, b);
    }
    static void collide(const Geom &g, const Phys &ph, const Bufs &b, int diag, const Launch &L, cudaStream_t s)
    {
        const bool lrn = ph.alpha_mode == ELBM_ALPHA_LEARNED;
        if constexpr (PR == ELBM_PREC_FP64) {
            k_collide<PR, ELBM_APREC_FP64, false><<<L.grid, L.block, 0, s>>>(g, ph, b, diag);
        } else if constexpr (Q != 19) {
            // other sets: the FP64 root or the guarded FP32 one (elbm_init
            // refuses the learned proposal, whose features are D3Q19's, and
            // the unguarded root)
            (void)lrn;
            if (ph.aprec == ELBM_APREC_FP64)
                k_collide<PR, ELBM_APREC_FP64, false><<<L.grid, L.block, 0, s>>>(g, ph, b, diag);
            else
                k_collide<PR, ELBM_APREC_FP32, false><<<L.grid, L.block, 0, s>>>(g, ph, b, diag);
        } else {
            if (ph.aprec == ELBM_APREC_FP64)
                k_collide<PR, ELBM_APREC_FP64, false><<<L.grid, L.block, 0, s>>>(g, ph, b, diag);
            else if (ph.aprec == ELBM_APREC_FP32_FAST && lrn)
                k_collide<PR, ELBM_APREC_FP32_FAST, true><<<L.grid, L.block, 0, s>>>(g, ph, b, diag);
            else if (ph.aprec == ELBM_APREC_FP32_FAST)
                k_collide<PR, ELBM_APREC_FP32_FAST, false><<<L.grid, L.block, 0, s>>>(g, ph, b, diag);
            else if (lrn)
                k_collide<PR, ELBM_APREC_FP32, true><<<L.grid, L.block, 0, s>>>(g, ph, b, diag);
            else
                k_collide<PR, ELBM_APREC_FP32, false><<<L.grid, L.block, 0, s>>>(g, ph, b, diag);
        }
    }
    static void bounce_bits(const Geom &g, const Bufs &b, const Launch &L, cudaStream_t s)
    {
        k_bounce_bits<<<L.grid, L.block, 0, s>>>(g, b.mask, const_cast<unsigned *>(b.bbits));
    }
    static void efield2(const Geom &g, const Phys &ph, const Bufs &b, const Launch &L, cudaStream_t s)
    {
        k_efield2<PR><<<L.grid, L.block, 0, s>>>(g, ph, b);
    }
    static void inlet(const Geom &g, const Phys &ph, const Bufs &b, cudaStream_t s)
    {
        k_inlet_update<PR><<<(unsigned)((ph.n_inlet + 127) / 128), 128, 0, s>>>(g, ph, b, b.scal);
    }
    static void phi_extrap(const Geom &g, const Bufs &b, cudaStream_t s)
    {
        k_phi_extrap<sc><<<(unsigned)((g.N + 255) / 256), 256, 0, s>>>((sc *)b.phi, (sc *)b.phi_old, b.scal, g.N);
    }
    static void export_pop(const Geom &g, const Bufs &b, double *out, const Launch &L, cudaStream_t s)
    {
        k_export_pop<PR><<<L.grid, L.block, 0, s>>>(g, b, out);
    }
    static void export_gpop(const Geom &g, const Bufs &b, double *out, const Launch &L, cudaStream_t s)
    {
        k_export_gpop<PR><<<L.grid, L.block, 0, s>>>(g, b, out);
    }
    static void export_plane(const void *plane, double *out, ll n, cudaStream_t s)
    {
        k_to_double<sc><<<(unsigned)((n + 255) / 256), 256, 0, s>>>((const sc *)plane, out, n);
    }
    static void add_plane(const float *lo, double *out, ll n, cudaStream_t s)
    {
        k_add_lo<float><<<(unsigned)((n + 255) / 256), 256, 0, s>>>(lo, out, n);
    }
    static Ops table()
    {
        Ops o;
        o.add_plane = add_plane;
        o.init_pop = init_pop;
        o.moments = moments;
        o.charge = charge;
        o.sor = sor;
        o.resid = resid;
        o.phi_mean = phi_mean;
        o.collide = collide;
        o.efield2 = efield2;
        o.inlet = inlet;
        o.phi_extrap = phi_extrap;
        o.export_pop = export_pop;
        o.export_gpop = export_gpop;
        o.export_plane = export_plane;
        o.bounce_bits = bounce_bits;
        o.heavy[0] = (const void *)k_collide<PR, ELBM_APREC_FP64, false>;
        if constexpr (PR == ELBM_PREC_FP64) {
            o.heavy[1] = o.heavy[2] = o.heavy[3] = o.heavy[4] = nullptr;
        } else if constexpr (Q != 19) {
            o.heavy[1] = (const void *)k_collide<PR, ELBM_APREC_FP32, false>;
            o.heavy[2] = o.heavy[3] = o.heavy[4] = nullptr;
        } else {
            o.heavy[1] = (const void *)k_collide<PR, ELBM_APREC_FP32, false>;
            o.heavy[2] = (const void *)k_collide<PR, ELBM_APREC_FP32_FAST, false>;
            o.heavy[3] = (const void *)k_collide<PR, ELBM_APREC_FP32, true>;
            o.heavy[4] = (const void *)k_collide<PR, ELBM_APREC_FP32_FAST, true>;
        }
        return o;
    }
};


ELBM_VS_END  // the multigrid below is the same for every velocity set

// ===========================================================================
// Geometric multigrid for the same fine-level Poisson operator (an
// accelerator for the SOR / Gauss-Seidel solve of Sec. II; the stopping rule
// is the same). Cell-centred coarsening by 2 per axis; coarse cell
// permittivity = mean of its 8 children; coarse face coupling 2^l (eps_I +
// eps_J)/2 (flux through a face of area 4^l over a distance 2^l); a coarse
// Dirichlet face couples with 2 4^l/(2^l + 1) eps_I, which places the
// boundary where the fine problem has it; restriction sums the 8 child
// residuals; trilinear (cell-centred) prolongation; red-black Gauss-Seidel
// smoothing (three colours on a level with an odd periodic extent). An odd
// extent coarsens to (n + 1)/2 cells, the last of one child: such a level
// re-discretises the operator on its cell sizes (mg_face) and interpolates
// by the cell centres (mg_pweights). Level 0 works on phi, q and rho
// directly; level l >= 1 on the correction e_l, right side b_l and
// permittivity eps_l.
// ===========================================================================
struct MGLevel {
    int nx, ny, nz;
    long long N;
    void *e, *b, *eps;       // level >= 1
    const unsigned char *m;  // level >= 1: 1 = conductor cell (correction held at 0), or NULL
    int last[3];             // fine (level-0) cells spanned by the last cell along each axis
    int irr;                 // 1 when a last[a] differs from 2^level (coarsened from an odd extent)
    int ncol;                // colours of its sweep ordering: 2 (red-black) or 3 (an odd periodic extent)
};

// Coarse-level geometry. The cells of level l span S = 2^l fine (level-0)
// cells along each axis, except where an axis was coarsened from an odd
// extent: its last cell, a single child, spans last[a] < S. The coarse
// operator is the fine one re-discretised on these cells: a face couples its
// two cells with eps_face A / d (A the face area, d the distance of the two
// centres, in fine cells), a Dirichlet face couples the cell with eps_s A /
// d_D, d_D = (s_a + 1)/2 the distance to the fine ghost plane. On a regular
// level A / d = 2^l and A / d_D = 2 4^l / (2^l + 1) (kap, kb below).
template <typename T>
__device__ __forceinline__ T mg_span(int i, int n, int last, int S) { return T(i == n - 1 ? last : S); }
template <typename T>
__device__ __forceinline__ T mg_face(const int n[3], const int last[3], int S, const int c[3], int a, int v)
{
    const int b = a == 0 ? 1 : 0, e = a == 2 ? 1 : 2;
    const T A = mg_span<T>(c[b], n[b], last[b], S) * mg_span<T>(c[e], n[e], last[e], S);
    return A / (T(0.5) * (mg_span<T>(c[a], n[a], last[a], S) + mg_span<T>(v, n[a], last[a], S)));
}
template <typename T>
__device__ __forceinline__ T mg_dface(const int n[3], const int last[3], int S, const int c[3], int a)
{
    const int b = a == 0 ? 1 : 0, e = a == 2 ? 1 : 2;
    const T A = mg_span<T>(c[b], n[b], last[b], S) * mg_span<T>(c[e], n[e], last[e], S);
    return A / (T(0.5) * (mg_span<T>(c[a], n[a], last[a], S) + T(1)));
}

// Gauss-Seidel update of coarse cell (x, y, z) of level `level` (the
// correction equation: homogeneous Dirichlet data)
template <typename T, bool IRR>
__device__ __forceinline__ void mg_gs_cell(const Geom &g, T *e, const T *b, const T *ep, const int n[3],
                                           const int last[3], int level, int x, int y, int z)
{
    const ll s = x + (ll)n[0] * (y + (ll)n[1] * z);
    const int S = 1 << level;
    const T kap = T(S), kb = T(2 * (1 << (2 * level))) / T(S + 1);
    const T es = ep[s];
    T num = b[s], den = 0;
    const int cc[3] = {x, y, z};
#pragma unroll
    for (int a = 0; a < 3; a++)
#pragma unroll
        for (int sg = -1; sg <= 1; sg += 2) {
            int c[3] = {cc[0], cc[1], cc[2]};
            const int v = nbc(c[a] + sg, n[a], g.per[a]);
            if (v < 0) {
                if (g.phi_kind[2 * a + (sg > 0)] == ELBM_PHI_DIRICHLET)
                    den += (IRR ? mg_dface<T>(n, last, S, cc, a) : kb) * es;
                continue;
            }
            c[a] = v;
            const ll nb = c[0] + (ll)n[0] * (c[1] + (ll)n[1] * c[2]);
            const T cf = (IRR ? mg_face<T>(n, last, S, cc, a, v) : kap) * T(0.5) * (es + ep[nb]);
            num += cf * e[nb];
            den += cf;
        }
    if (den > T(0)) e[s] = num / den;
}

// residual of the correction equation at coarse cell (x, y, z)
template <typename T, bool IRR>
__device__ __forceinline__ T mg_res_cell(const Geom &g, const T *e, const T *b, const T *ep, const int n[3],
                                         const int last[3], int level, int x, int y, int z)
{
    const ll s = x + (ll)n[0] * (y + (ll)n[1] * z);
    const int S = 1 << level;
    const T kap = T(S), kb = T(2 * (1 << (2 * level))) / T(S + 1);
    const T es = ep[s], xs = e[s];
    T r = b[s];
    const int cc[3] = {x, y, z};
#pragma unroll
    for (int a = 0; a < 3; a++)
#pragma unroll
        for (int sg = -1; sg <= 1; sg += 2) {
            int c[3] = {cc[0], cc[1], cc[2]};
            const int v = nbc(c[a] + sg, n[a], g.per[a]);
            if (v < 0) {
                if (g.phi_kind[2 * a + (sg > 0)] == ELBM_PHI_DIRICHLET)
                    r -= (IRR ? mg_dface<T>(n, last, S, cc, a) : kb) * es * xs;
                continue;
            }
            c[a] = v;
            const ll nb = c[0] + (ll)n[0] * (c[1] + (ll)n[1] * c[2]);
            r += (IRR ? mg_face<T>(n, last, S, cc, a, v) : kap) * T(0.5) * (es + ep[nb]) * (e[nb] - xs);
        }
    return r;
}

// Prolongation along one axis: fine cell i of a level whose cells span Sf
// fine (level-0) cells (its last one lastf) from the coarse level above
// (spans 2 Sf, its last one lastc). i0 is the parent, i1 the other coarse
// cell of the pair and w1 its weight (the parent's 1 - w1), linear in the
// positions of the cell centres: 1/4 on a regular pair, 0 for a single child
// (its centre is the parent's). Beyond a Neumann face the edge value (w1 =
// 0); beyond a Dirichlet face the correction is 0 (skip: the i1 term drops,
// its weight taken as for a regular ghost cell).
template <typename T>
__device__ __forceinline__ void mg_pweights(const Geom &g, int a, int i, int nf, int lastf, int Sf, int nc,
                                            int lastc, int &i0, int &i1, T &w1, bool &skip)
{
    const int Sc = 2 * Sf;
    i0 = i >> 1;
    i1 = i0;
    w1 = T(0);
    skip = false;
    const T xf = T(i) * T(Sf) + T(0.5) * mg_span<T>(i, nf, lastf, Sf);
    const T xp = T(i0) * T(Sc) + T(0.5) * mg_span<T>(i0, nc, lastc, Sc);
    if (xf == xp) return;
    const int o = xf > xp ? 1 : -1;
    const int v = nbc(i0 + o, nc, g.per[a]);
    T dist;
    if (v < 0) {
        if (g.phi_kind[2 * a + (o > 0)] != ELBM_PHI_DIRICHLET) return;
        skip = true;
        dist = T(0.5) * (mg_span<T>(i0, nc, lastc, Sc) + T(Sc));
    } else {
        T xn = T(v) * T(Sc) + T(0.5) * mg_span<T>(v, nc, lastc, Sc);
        const T len = T(nc - 1) * T(Sc) + T(lastc);  // the axis in fine cells (periodic wrap)
        if (o > 0 && v < i0) xn += len;
        if (o < 0 && v > i0) xn -= len;
        dist = xn > xp ? xn - xp : xp - xn;
        i1 = v;
    }
    w1 = (xf > xp ? xf - xp : xp - xf) / dist;
}

// Gauss-Seidel sweep of one colour on a coarse level
template <typename T, bool IRR, int NC>
__global__ void __launch_bounds__(128) k_mg_smooth(Geom g, MGLevel L, int level, int color)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    const int y = blockIdx.y * blockDim.y + threadIdx.y;
    const int z = blockIdx.z;
    const int x = NC == 3 ? i : 2 * i + ((y + z + color) & 1);
    if (x >= L.nx || y >= L.ny) return;
    if (NC == 3 && color3(g.per, x, y, z, L.nx, L.ny, L.nz) != color) return;
    const ll s = x + (ll)L.nx * (y + (ll)L.ny * z);
    if (L.m && L.m[s]) return;  // conductor cell: correction stays 0
    const int n[3] = {L.nx, L.ny, L.nz};
    mg_gs_cell<T, IRR>(g, (T *)L.e, (const T *)L.b, (const T *)L.eps, n, L.last, level, x, y, z);
}

// residual of level l at one cell (level 0: phi / q / rho and the Dirichlet data)
template <int PR>
__device__ __forceinline__ typename Tr<PR>::sc mg_resid_at(const Geom &g, const Phys &ph, const Bufs &bf,
                                                          const MGLevel &L, int level, int x, int y, int z)
{
    typedef typename Tr<PR>::sc T;
    const ll s = x + (ll)L.nx * (y + (ll)L.ny * z);
    if (level == 0) {
        // the fine operator exactly as the fine smoother and residual use it
        // (pois_nb): solid (conductor) nodes are fixed, with residual 0, and a
        // solid neighbour enters as Dirichlet data at phi_solid
        const Cst<T> &k = cst<T>(ph);
        const T *phi = (const T *)bf.phi, *rho = (const T *)bf.rho;
        unsigned char kind = bf.mask ? bf.mask[s] : 0;
        if (kind == ELBM_NODE_SOLID) return T(0);
        const T es = T(1) + k.kap * rho[s];
        const T ps = phi[s];
        T r = kind == ELBM_NODE_FLUID ? ((const T *)bf.q)[s] - scal_of<T>(bf, S_QMEAN) : T(0);
        int xn[2];
        if (pois_fast(g, bf.mask, x, y, z, (int)s, xn)) {
            const int off[3] = {1, g.nx, g.nx * g.ny};
#pragma unroll
            for (int a = 0; a < 3; a++)
#pragma unroll
                for (int sg = -1; sg <= 1; sg += 2) {
                    const int nb = a == 0 ? xn[sg > 0] : (int)s + sg * off[a];
                    const int li = nb >= 0 ? nb : (int)s;  // loads independent of the face test
                    const T rn = rho[li], pn = phi[li];
                    const T dl = interior_dl<T>(g, k, a, sg);
                    if (nb >= 0) {
                        r += face_eps<T>(es, T(1) + k.kap * rn, ph.eps_face) * ((pn + dl) - ps);
                    } else {
                        T v = 0;
                        if (pois_xface<T>(g, k, x, y, z, sg, &v)) r += es * ((v + dl) - ps);
                    }
                }
            return r;
        }
        Nbr n;
        nbr_init(n, g, x, y, z, s);
#pragma unroll
        for (int a = 0; a < 3; a++)
#pragma unroll
            for (int sg = -1; sg <= 1; sg += 2) {
                int nb = 0;
                T v = 0, dl = 0;
                const int kk = pois_nb<T>(g, k, bf.mask, n, x, y, z, a, sg, &nb, &v, &dl);
                if (kk == 0) r += face_eps<T>(es, T(1) + k.kap * rho[nb], ph.eps_face) * ((phi[nb] + dl) - ps);
                else if (kk == 1) r += es * ((v + dl) - ps);
            }
        return r;
    }
    if (L.m && L.m[s]) return T(0);
    const int n[3] = {L.nx, L.ny, L.nz};
    if (L.irr) return mg_res_cell<T, true>(g, (const T *)L.e, (const T *)L.b, (const T *)L.eps, n, L.last, level, x, y, z);
    return mg_res_cell<T, false>(g, (const T *)L.e, (const T *)L.b, (const T *)L.eps, n, L.last, level, x, y, z);
}

// b_{l+1} = sum of the child residuals of level l (8, or fewer in the last
// cell of an axis coarsened from an odd extent); e_{l+1} = 0. Eight
// consecutive lanes handle the children of one coarse cell and sum them with
// a fixed shuffle tree.
template <int PR, bool ODD>
__global__ void __launch_bounds__(128) k_mg_restrict(Geom g, Phys ph, Bufs bf, MGLevel F, MGLevel C, int level,
                                                     int zc)
{
    typedef typename Tr<PR>::sc T;
    const unsigned gid = blockIdx.x * blockDim.x + threadIdx.x;
    const unsigned S = gid >> 3;
    const int c = (int)(gid & 7);
    const bool act = S < (unsigned)C.N;
    T r = 0, ep = 0;
    int X = 0, Y = 0, Z = 0;
    if (act) {
        const unsigned nxy = (unsigned)C.nx * (unsigned)C.ny;
        Z = (int)(S / nxy);
        const unsigned rem = S - (unsigned)Z * nxy;
        Y = (int)(rem / (unsigned)C.nx);
        X = (int)(rem - (unsigned)Y * (unsigned)C.nx);
        const int fx = 2 * X + (c & 1), fy = 2 * Y + ((c >> 1) & 1), fz = 2 * Z + (c >> 2);
        if (!ODD || (fx < F.nx && fy < F.ny && fz < F.nz)) {
            // zc: the colour the fine Gauss-Seidel sweep updated last, whose
            // residual is the rounding of that update, taken as 0 (-1: none)
            if (zc < 0 || ((fx + fy + fz) & 1) != zc) r = mg_resid_at<PR>(g, ph, bf, F, level, fx, fy, fz);
            // the coarse permittivity (mean of the children) comes with the
            // restriction: the coarse level's smoothing and residual read it next
            const ll fs = fx + (ll)F.nx * (fy + (ll)F.ny * fz);
            ep = level == 0 ? T(1) + cst<T>(ph).kap * ((const T *)bf.rho)[fs] : ((const T *)F.eps)[fs];
        }
    }
    r += __shfl_down_sync(0xffffffffu, r, 4, 8);
    r += __shfl_down_sync(0xffffffffu, r, 2, 8);
    r += __shfl_down_sync(0xffffffffu, r, 1, 8);
    ep += __shfl_down_sync(0xffffffffu, ep, 4, 8);
    ep += __shfl_down_sync(0xffffffffu, ep, 2, 8);
    ep += __shfl_down_sync(0xffffffffu, ep, 1, 8);
    if (act && c == 0) {
        const int nch = ODD ? (2 * X + 1 < F.nx ? 2 : 1) * (2 * Y + 1 < F.ny ? 2 : 1) * (2 * Z + 1 < F.nz ? 2 : 1) : 8;
        ((T *)C.b)[S] = (C.m && C.m[S]) ? T(0) : r;
        ((T *)C.e)[S] = T(0);
        ((T *)C.eps)[S] = ep * (T(1) / T(nch));
    }
}

// Level 0 -> 1 with the colour zc settled (red-black, reduced precision,
// even extents): four lanes per coarse cell, each taking one pair of x
// children: the residual of its unsettled child (the settled child's is the
// rounding of its update, taken as 0) and the permittivity of both; so no
// warp splits between full and settled children.
template <int PR>
__global__ void __launch_bounds__(128) k_mg_restrict_pairs(Geom g, Phys ph, Bufs bf, MGLevel F, MGLevel C, int zc)
{
    typedef typename Tr<PR>::sc T;
    const unsigned gid = blockIdx.x * blockDim.x + threadIdx.x;
    const unsigned S = gid >> 2;
    const int c = (int)(gid & 3);
    const bool act = S < (unsigned)C.N;
    T r = 0, ep = 0;
    if (act) {
        const unsigned nxy = (unsigned)C.nx * (unsigned)C.ny;
        const int Z = (int)(S / nxy);
        const unsigned rem = S - (unsigned)Z * nxy;
        const int Y = (int)(rem / (unsigned)C.nx);
        const int X = (int)(rem - (unsigned)Y * (unsigned)C.nx);
        const int fy = 2 * Y + (c & 1), fz = 2 * Z + (c >> 1);
        r = mg_resid_at<PR>(g, ph, bf, F, 0, 2 * X + ((fy + fz + 1 - zc) & 1), fy, fz);
        const ll f0 = 2 * X + (ll)F.nx * (fy + (ll)F.ny * fz);
        const T kap = cst<T>(ph).kap;
        const T *rho = (const T *)bf.rho;
        ep = (T(1) + kap * rho[f0]) + (T(1) + kap * rho[f0 + 1]);
    }
    r += __shfl_down_sync(0xffffffffu, r, 2, 4);
    r += __shfl_down_sync(0xffffffffu, r, 1, 4);
    ep += __shfl_down_sync(0xffffffffu, ep, 2, 4);
    ep += __shfl_down_sync(0xffffffffu, ep, 1, 4);
    if (act && c == 0) {
        ((T *)C.b)[S] = (C.m && C.m[S]) ? T(0) : r;
        ((T *)C.e)[S] = T(0);
        ((T *)C.eps)[S] = ep * T(0.125);
    }
}

// coarse permittivity: mean of the children (level 0 children from rho)
template <int PR>
__global__ void __launch_bounds__(128) k_mg_eps(Geom g, Phys ph, Bufs bf, MGLevel F, MGLevel C, int level)
{
    typedef typename Tr<PR>::sc T;
    const int X = blockIdx.x * blockDim.x + threadIdx.x;
    const int Y = blockIdx.y * blockDim.y + threadIdx.y;
    const int Z = blockIdx.z;
    if (X >= C.nx || Y >= C.ny) return;
    const Cst<T> &k = cst<T>(ph);
    T sum = 0;
    int nch = 0;
#pragma unroll
    for (int c = 0; c < 8; c++) {
        const int fx = 2 * X + (c & 1), fy = 2 * Y + ((c >> 1) & 1), fz = 2 * Z + (c >> 2);
        if (fx >= F.nx || fy >= F.ny || fz >= F.nz) continue;
        const ll s = fx + (ll)F.nx * (fy + (ll)F.ny * fz);
        sum += level == 0 ? T(1) + k.kap * ((const T *)bf.rho)[s] : ((const T *)F.eps)[s];
        nch++;
    }
    ((T *)C.eps)[X + (ll)C.nx * (Y + (ll)C.ny * Z)] = sum * (T(1) / T(nch));
}

// trilinear prolongation of e_{l+1} added to level l (phi at level 0).
// Beyond a Dirichlet face the coarse error is 0, beyond a Neumann face the
// edge value. A coarse level with a smaller last cell (odd extent) takes the
// weights from the positions of the cell centres (mg_pweights).
template <int PR, bool IRR>
__global__ void __launch_bounds__(128) k_mg_prolong(Geom g, Bufs bf, MGLevel F, MGLevel C, int level)
{
    typedef typename Tr<PR>::sc T;
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    const int y = blockIdx.y * blockDim.y + threadIdx.y;
    const int z = blockIdx.z;
    if (x >= F.nx || y >= F.ny) return;
    const T *ec = (const T *)C.e;
    const int fc[3] = {x, y, z}, nc[3] = {C.nx, C.ny, C.nz}, nf[3] = {F.nx, F.ny, F.nz};
    int i0[3], i1[3];
    bool z1[3];
    T acc = 0;
    if (IRR) {
        T w1[3];
#pragma unroll
        for (int a = 0; a < 3; a++)
            mg_pweights<T>(g, a, fc[a], nf[a], level == 0 ? 1 : F.last[a], 1 << level, nc[a], C.last[a], i0[a],
                           i1[a], w1[a], z1[a]);
#pragma unroll
        for (int c = 0; c < 8; c++) {
            int ax = c & 1, ay = (c >> 1) & 1, az = c >> 2;
            if ((ax && z1[0]) || (ay && z1[1]) || (az && z1[2])) continue;
            T w = (ax ? w1[0] : T(1) - w1[0]) * (ay ? w1[1] : T(1) - w1[1]) * (az ? w1[2] : T(1) - w1[2]);
            int X = ax ? i1[0] : i0[0], Y = ay ? i1[1] : i0[1], Z = az ? i1[2] : i0[2];
            acc += w * ec[X + (ll)C.nx * (Y + (ll)C.ny * Z)];
        }
    } else {
#pragma unroll
        for (int a = 0; a < 3; a++) {
            i0[a] = fc[a] >> 1;
            int o = (fc[a] & 1) ? 1 : -1;  // the other coarse cell of the 3/4 - 1/4 pair
            int v = nbc(i0[a] + o, nc[a], g.per[a]);
            z1[a] = false;
            if (v < 0) {
                int face = 2 * a + (o > 0);
                if (g.phi_kind[face] == ELBM_PHI_DIRICHLET) { z1[a] = true; v = i0[a]; }
                else v = i0[a];
            }
            i1[a] = v;
        }
#pragma unroll
        for (int c = 0; c < 8; c++) {
            int ax = c & 1, ay = (c >> 1) & 1, az = c >> 2;
            if ((ax && z1[0]) || (ay && z1[1]) || (az && z1[2])) continue;
            T w = (ax ? T(0.25) : T(0.75)) * (ay ? T(0.25) : T(0.75)) * (az ? T(0.25) : T(0.75));
            int X = ax ? i1[0] : i0[0], Y = ay ? i1[1] : i0[1], Z = az ? i1[2] : i0[2];
            acc += w * ec[X + (ll)C.nx * (Y + (ll)C.ny * Z)];
        }
    }
    const ll s = x + (ll)F.nx * (y + (ll)F.ny * z);
    if (level == 0) {
        if (bf.mask && bf.mask[s] == ELBM_NODE_SOLID) return;
        ((T *)bf.phi)[s] += acc;
    } else {
        if (F.m && F.m[s]) return;
        ((T *)F.e)[s] += acc;
    }
}

// ---------------------------------------------------------------------------
// The bottom of the V-cycle in one CTA: every level from `lt` down (at most
// kTailCells cells on level lt) lives in shared memory; smoothing,
// restriction, the coarsest sweeps and prolongation run with block barriers
// instead of kernel launches. Same operators as the launched levels.
// ---------------------------------------------------------------------------
constexpr int kTailCells = 4096;
constexpr int kTailMaxLevels = 8;

struct MGTail {
    int nt;                       // levels in the tail
    int lt;                       // global index of the first tail level
    int nx[kTailMaxLevels], ny[kTailMaxLevels], nz[kTailMaxLevels];
    long long N[kTailMaxLevels], off[kTailMaxLevels];  // cells, offset in each smem array
    int last[kTailMaxLevels][3];  // fine cells spanned by the last cell along each axis (MGLevel::last)
    int irr[kTailMaxLevels];      // MGLevel::irr
    int ncol[kTailMaxLevels];     // MGLevel::ncol
    long long total;              // cells over all tail levels
    int coarse_sweeps;
    MGLevel top;                  // global arrays of level lt
    const unsigned char *m;       // conductor masks of the tail levels (offsets off[k]), or NULL
};

// The tail runs as one CTA of (BX, BY, BZ) threads: a level is swept with
// x = tx + BX i (or, in a red-black pass, x = 2 (tx + BX i) + parity so that
// every thread owns cells of the active colour), y = ty + BY j, z = tz + BZ k;
// no integer division, no idle half in a red-black pass.
template <typename T>
__device__ void tail_smooth(const Geom &g, const MGTail &t, T *E, T *B, T *P, const unsigned char *M, int k,
                            int sweeps)
{
    const int nx = t.nx[k], ny = t.ny[k], nz = t.nz[k];
    const unsigned char *m = M ? M + t.off[k] : nullptr;
    T *e = E + t.off[k];
    const T *b = B + t.off[k], *ep = P + t.off[k];
    const int level = t.lt + k;
    const int n_[3] = {nx, ny, nz};
    const int nc = t.ncol[k];
    if (nc == 2 && !t.irr[k]) {  // red-black on a regular level
        for (int it = 0; it < 2 * sweeps; it++) {
            const int color = it & 1;
            for (int z = threadIdx.z; z < nz; z += blockDim.z)
                for (int y = threadIdx.y; y < ny; y += blockDim.y)
                    for (int xi = threadIdx.x;; xi += blockDim.x) {
                        const int x = 2 * xi + ((y + z + color) & 1);
                        if (x >= nx) break;
                        if (m && m[x + nx * (y + ny * z)]) continue;  // conductor cell: correction stays 0
                        mg_gs_cell<T, false>(g, e, b, ep, n_, t.last[k], level, x, y, z);
                    }
            __syncthreads();
        }
        return;
    }
    for (int it = 0; it < nc * sweeps; it++) {
        const int color = it % nc;
        for (int z = threadIdx.z; z < nz; z += blockDim.z)
            for (int y = threadIdx.y; y < ny; y += blockDim.y)
                for (int xi = threadIdx.x;; xi += blockDim.x) {
                    const int x = nc == 3 ? xi : 2 * xi + ((y + z + color) & 1);
                    if (x >= nx) break;
                    if (nc == 3 && color3(g.per, x, y, z, nx, ny, nz) != color) continue;
                    if (m && m[x + nx * (y + ny * z)]) continue;
                    mg_gs_cell<T, true>(g, e, b, ep, n_, t.last[k], level, x, y, z);
                }
        __syncthreads();
    }
}

// The coarsest level when it has at most 32 cells: one warp, a cell per
// lane, warp-level synchronisation between colours instead of the block's
// barriers; the same updates in the same colour order as tail_smooth.
template <typename T>
__device__ void tail_smooth_warp(const Geom &g, const MGTail &t, T *E, T *B, T *P, const unsigned char *M, int k,
                                 int sweeps)
{
    const int tid = threadIdx.x + blockDim.x * (threadIdx.y + blockDim.y * threadIdx.z);
    if (tid < 32) {
        const int nx = t.nx[k], ny = t.ny[k], nz = t.nz[k];
        const int n_[3] = {nx, ny, nz};
        const unsigned char *m = M ? M + t.off[k] : nullptr;
        T *e = E + t.off[k];
        const T *b = B + t.off[k], *ep = P + t.off[k];
        const int level = t.lt + k, nc = t.ncol[k];
        const bool live = tid < (int)t.N[k];
        const int x = tid % nx, y = (tid / nx) % ny, z = tid / (nx * ny);
        const int col = live ? (nc == 3 ? color3(g.per, x, y, z, nx, ny, nz) : ((x + y + z) & 1)) : -1;
        const bool work = live && !(m && m[tid]);  // conductor cell: correction stays 0
        for (int it = 0; it < nc * sweeps; it++) {
            if (work && col == it % nc) {
                if (t.irr[k]) mg_gs_cell<T, true>(g, e, b, ep, n_, t.last[k], level, x, y, z);
                else mg_gs_cell<T, false>(g, e, b, ep, n_, t.last[k], level, x, y, z);
            }
            __syncwarp();
        }
    }
    __syncthreads();
}

template <typename T>
__global__ void __launch_bounds__(1024) k_mg_tail(Geom g, MGTail t, int nu)
{
    extern __shared__ unsigned char smem_raw[];
    T *E = (T *)smem_raw;
    T *B = E + t.total;
    T *P = B + t.total;
    unsigned char *M = t.m ? (unsigned char *)(P + t.total) : nullptr;
    const int tid = threadIdx.x + blockDim.x * (threadIdx.y + blockDim.y * threadIdx.z);
    const int nthr = blockDim.x * blockDim.y * blockDim.z;
    for (int s = tid; s < (int)t.N[0]; s += nthr) {
        E[s] = T(0);
        B[s] = ((const T *)t.top.b)[s];
        P[s] = ((const T *)t.top.eps)[s];
    }
    if (M)
        for (int s = tid; s < (int)t.total; s += nthr) M[s] = t.m[s];
    __syncthreads();
    for (int k = 1; k < t.nt; k++) {  // coarse permittivities: mean of the children
        const int nx = t.nx[k], ny = t.ny[k], nz = t.nz[k], fx = t.nx[k - 1], fy = t.ny[k - 1], fz = t.nz[k - 1];
        const T *pf = P + t.off[k - 1];
        for (int Z = threadIdx.z; Z < nz; Z += blockDim.z)
            for (int Y = threadIdx.y; Y < ny; Y += blockDim.y)
                for (int X = threadIdx.x; X < nx; X += blockDim.x) {
                    T sum = 0;
                    int nch = 0;
                    for (int c = 0; c < 8; c++) {
                        const int cx_ = 2 * X + (c & 1), cy_ = 2 * Y + ((c >> 1) & 1), cz_ = 2 * Z + (c >> 2);
                        if (cx_ >= fx || cy_ >= fy || cz_ >= fz) continue;
                        sum += pf[cx_ + fx * (cy_ + fy * cz_)];
                        nch++;
                    }
                    P[t.off[k] + X + nx * (Y + ny * Z)] = sum * (T(1) / T(nch));
                }
        __syncthreads();
    }
    // down: smooth, restrict
    for (int k = 0; k + 1 < t.nt; k++) {
        tail_smooth<T>(g, t, E, B, P, M, k, nu);
        const int nx = t.nx[k + 1], ny = t.ny[k + 1], nz = t.nz[k + 1];
        const int fx = t.nx[k], fy = t.ny[k], fz = t.nz[k];
        const int nf[3] = {fx, fy, fz};
        const unsigned char *mf = M ? M + t.off[k] : nullptr;
        for (int Z = threadIdx.z; Z < nz; Z += blockDim.z)
            for (int Y = threadIdx.y; Y < ny; Y += blockDim.y)
                for (int X = threadIdx.x; X < nx; X += blockDim.x) {
                    T sum = 0;
                    for (int c = 0; c < 8; c++) {
                        const int cx_ = 2 * X + (c & 1), cy_ = 2 * Y + ((c >> 1) & 1), cz_ = 2 * Z + (c >> 2);
                        if (cx_ >= fx || cy_ >= fy || cz_ >= fz) continue;
                        if (mf && mf[cx_ + fx * (cy_ + fy * cz_)]) continue;  // a conductor's residual is 0
                        if (t.irr[k])
                            sum += mg_res_cell<T, true>(g, E + t.off[k], B + t.off[k], P + t.off[k], nf, t.last[k],
                                                        t.lt + k, cx_, cy_, cz_);
                        else
                            sum += mg_res_cell<T, false>(g, E + t.off[k], B + t.off[k], P + t.off[k], nf, t.last[k],
                                                         t.lt + k, cx_, cy_, cz_);
                    }
                    const int S = X + nx * (Y + ny * Z);
                    B[t.off[k + 1] + S] = (M && M[t.off[k + 1] + S]) ? T(0) : sum;
                    E[t.off[k + 1] + S] = T(0);
                }
        __syncthreads();
    }
    if (t.N[t.nt - 1] <= 32 && nthr >= 32) tail_smooth_warp<T>(g, t, E, B, P, M, t.nt - 1, t.coarse_sweeps);
    else tail_smooth<T>(g, t, E, B, P, M, t.nt - 1, t.coarse_sweeps);
    // up: prolong (trilinear), smooth
    for (int k = t.nt - 2; k >= 0; k--) {
        const int nx = t.nx[k], ny = t.ny[k], nz = t.nz[k];
        const int nc[3] = {t.nx[k + 1], t.ny[k + 1], t.nz[k + 1]}, nf[3] = {nx, ny, nz};
        const T *ec = E + t.off[k + 1];
        const bool irr = t.irr[k + 1] != 0;
        const int Sf = 1 << (t.lt + k);
        for (int fz_ = threadIdx.z; fz_ < nz; fz_ += blockDim.z)
            for (int fy_ = threadIdx.y; fy_ < ny; fy_ += blockDim.y)
                for (int fx_ = threadIdx.x; fx_ < nx; fx_ += blockDim.x) {
                    const int fc[3] = {fx_, fy_, fz_};
                    int i0[3], i1[3];
                    bool z1[3];
                    T w1[3];
                    for (int a = 0; a < 3; a++) {
                        if (irr) {
                            mg_pweights<T>(g, a, fc[a], nf[a], t.last[k][a], Sf, nc[a], t.last[k + 1][a], i0[a], i1[a],
                                           w1[a], z1[a]);
                            continue;
                        }
                        w1[a] = T(0.25);
                        i0[a] = fc[a] >> 1;
                        int o = (fc[a] & 1) ? 1 : -1;
                        int v = nbc(i0[a] + o, nc[a], g.per[a]);
                        z1[a] = false;
                        if (v < 0) {
                            if (g.phi_kind[2 * a + (o > 0)] == ELBM_PHI_DIRICHLET) z1[a] = true;
                            v = i0[a];
                        }
                        i1[a] = v;
                    }
                    T acc = 0;
                    for (int c = 0; c < 8; c++) {
                        int ax = c & 1, ay = (c >> 1) & 1, az = c >> 2;
                        if ((ax && z1[0]) || (ay && z1[1]) || (az && z1[2])) continue;
                        T w = irr ? (ax ? w1[0] : T(1) - w1[0]) * (ay ? w1[1] : T(1) - w1[1]) *
                                        (az ? w1[2] : T(1) - w1[2])
                                  : (ax ? T(0.25) : T(0.75)) * (ay ? T(0.25) : T(0.75)) * (az ? T(0.25) : T(0.75));
                        int X = ax ? i1[0] : i0[0], Y = ay ? i1[1] : i0[1], Z = az ? i1[2] : i0[2];
                        acc += w * ec[X + nc[0] * (Y + nc[1] * Z)];
                    }
                    const int fs = fx_ + nx * (fy_ + ny * fz_);
                    if (!(M && M[t.off[k] + fs])) E[t.off[k] + fs] += acc;
                }
        __syncthreads();
        tail_smooth<T>(g, t, E, B, P, M, k, nu);
    }
    for (int s = tid; s < (int)t.N[0]; s += nthr) ((T *)t.top.e)[s] = E[s];
}

// One CTA of at most 1024 threads for a tail whose top level is nx x ny x nz:
// BX covers half a row (colour-compacted passes), then BY, BZ.
inline dim3 tail_block(int nx, int ny, int nz)
{
    int bx = (nx + 1) / 2;
    if (bx > 32) bx = 32;
    int by = ny < 1024 / bx ? ny : 1024 / bx;
    int bz = nz < 1024 / (bx * by) ? nz : 1024 / (bx * by);
    return dim3(bx, by, bz < 1 ? 1 : bz);
}

// ---------------------------------------------------------------------------
// Multigrid launchers for one precision.
// ---------------------------------------------------------------------------
template <int PR>
struct MGLaunchers {
    typedef typename Tr<PR>::sc sc;
    static dim3 grid_of(int nx, int ny, int nz, dim3 blk) { return dim3((nx + blk.x - 1) / blk.x, (ny + blk.y - 1) / blk.y, nz); }
    static dim3 blk_of(int nx) { int bx = nx >= 128 ? 128 : ((nx + 31) / 32) * 32; return dim3(bx, 128 / bx, 1); }
    static void smooth(const Geom &g, const Phys &ph, const Bufs &b, const MGLevel &L, int level, int color,
                       const Launch &fine_half, cudaStream_t s)
    {
        if (level == 0) {
            if (g.ncol == 3) k_sor<PR, 3><<<fine_half.grid, fine_half.block, 0, s>>>(g, ph, b, color, 1);
            else k_sor<PR, 2><<<fine_half.grid, fine_half.block, 0, s>>>(g, ph, b, color, 1);
        } else {
            const int nh = L.ncol == 3 ? L.nx : (L.nx + 1) / 2;
            dim3 blk = blk_of(nh);
            const dim3 gr = grid_of(nh, L.ny, L.nz, blk);
            if (L.ncol == 3) k_mg_smooth<sc, true, 3><<<gr, blk, 0, s>>>(g, L, level, color);
            else if (L.irr) k_mg_smooth<sc, true, 2><<<gr, blk, 0, s>>>(g, L, level, color);
            else k_mg_smooth<sc, false, 2><<<gr, blk, 0, s>>>(g, L, level, color);
        }
    }
    static void restrict_(const Geom &g, const Phys &ph, const Bufs &b, const MGLevel &F, const MGLevel &C,
                          int level, int zc, cudaStream_t s)
    {
        long long thr = 8 * C.N;
        const unsigned nb = (unsigned)((thr + 127) / 128);
        const bool odd = ((F.nx | F.ny | F.nz) & 1) != 0;
        if (level == 0 && zc >= 0 && !odd)
            k_mg_restrict_pairs<PR><<<(unsigned)((4 * C.N + 127) / 128), 128, 0, s>>>(g, ph, b, F, C, zc);
        else if (odd) k_mg_restrict<PR, true><<<nb, 128, 0, s>>>(g, ph, b, F, C, level, zc);
        else k_mg_restrict<PR, false><<<nb, 128, 0, s>>>(g, ph, b, F, C, level, zc);
    }
    static void eps(const Geom &g, const Phys &ph, const Bufs &b, const MGLevel &F, const MGLevel &C, int level,
                    cudaStream_t s)
    {
        dim3 blk = blk_of(C.nx);
        k_mg_eps<PR><<<grid_of(C.nx, C.ny, C.nz, blk), blk, 0, s>>>(g, ph, b, F, C, level);
    }
    static void prolong(const Geom &g, const Bufs &b, const MGLevel &F, const MGLevel &C, int level, cudaStream_t s)
    {
        dim3 blk = blk_of(F.nx);
        if (C.irr) k_mg_prolong<PR, true><<<grid_of(F.nx, F.ny, F.nz, blk), blk, 0, s>>>(g, b, F, C, level);
        else k_mg_prolong<PR, false><<<grid_of(F.nx, F.ny, F.nz, blk), blk, 0, s>>>(g, b, F, C, level);
    }
    static void prepare()
    {
        cudaFuncSetAttribute(k_mg_tail<sc>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
    }
    static void tail_(const Geom &g, const MGTail &t, int nu, cudaStream_t s)
    {
        size_t sm = 3 * (size_t)t.total * sizeof(sc) + (t.m ? (size_t)t.total : 0);
        k_mg_tail<sc><<<1, tail_block(t.nx[0], t.ny[0], t.nz[0]), sm, s>>>(g, t, nu);
    }
    static MGOps table()
    {
        MGOps o;
        o.tail = tail_;
        o.prepare = prepare;
        o.smooth = smooth;
        o.restrict_ = restrict_;
        o.eps = eps;
        o.prolong = prolong;
        return o;
    }
};

}  // namespace elbm
