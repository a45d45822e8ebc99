// elbm_capi.cu -- the C ABI declared in include/elbm.h: parameter checks,
// device state, the order of the passes of one step (Sec. II C of
// arXiv:1612.05404) and field export. Every pass runs in the kernels of
// k_fp64.cu / k_fp32.cu / k_bf16.cu (D3Q19) or k_fp64_d2q9.cu /
// k_fp32_d2q9.cu (D2Q9); this file only sequences them, plus the
// small deterministic reductions that turn per-block partial sums into the
// global sums the step needs (mean charge, Poisson residual, diagnostics).
#include <cmath>
#include <cstdlib>
#include <cstring>
#include <array>
#include <vector>
#include <map>
#include <mutex>
#include <new>

#include "elbm.h"
#include "elbm_internal.h"
#include "elbm_kernels.cuh"

using namespace elbm;

namespace {
constexpr int kMaxLevels = 10;
constexpr int kNu = 2;             // pre- and post-smoothing sweeps (FP64; the tail in FP64)
constexpr int kNuPre = 2, kNuPost = 2;  // the same on the launched levels in reduced precision
constexpr int kNuTail = 1;         // the same on the levels of the one-CTA tail (reduced precision;
                                   // FP64 solves to 1e-13 keep kNu)
constexpr int kCoarseSweeps = 8;   // red-black sweeps on the coarsest level (<= 8 cells per axis pair)
constexpr int kCoarseCells = 512;  // a coarsest level above this size coarsens further, odd extents included
}

struct elbm_handle {
    elbm_params p;
    Geom g;
    Phys ph;
    Bufs b;
    Launch L;
    Launch Lh;                 // one thread per site of one red-black colour
    Ops ops;
    cudaStream_t s;            // the caller's stream: all work runs here
    int Q;                     // populations per site of the velocity set (19 or 9)
    int has_dirichlet;
    double *pin;               // pinned host scalars; [9] Poisson no-convergence counter, [16..39] diagnostics
    int diag_mirror;           // pin[16..39] holds the last step's diagnostics (graph steps)
    double *xtmp;              // elbm_fields' FP64 export scratch, kept for the next call
    size_t xtmp_n;
    void *arena;               // every device buffer of the handle, carved from one allocation
    long long step;
    size_t pop_bytes, g_bytes, sc_bytes;
    MGOps mg;
    int nlev;                  // multigrid levels (0 = SOR)
    MGLevel lev[kMaxLevels];
    int lt;                    // first level solved by the one-CTA tail kernel
    MGTail tail;
    int ce;                    // SOR sweeps per convergence test (1 for multigrid)
    int units_max;             // cap on Poisson units per step
    cudaStream_t cap, cap2;    // private streams used only to capture graphs
    cudaGraphExec_t gexec[2];  // one whole step for each A/B parity
    cudaGraphExec_t gsec[2][3];  // profiling: the step as three section graphs
    int use_graph;
    int want_graph, graph_tried;  // step graphs requested; capture attempted (on the first elbm_step)
    int n_pre, n_body, n_post; // kernels per graph section (launch accounting)
    double noconv_seen;
    cudaEvent_t ev[5];         // pass boundaries when profiling
    double pass_ms[4];
    double prof_steps, prof_collide, prof_sweeps, launches;
    // batch of instances (elbm_batch_create): n_sub > 0
    int n_sub;
    elbm_handle **sub;
    long long *sub_step0;      // each instance's step counter when the batch was made
    cudaGraphExec_t bexec[2];  // all instances' steps, one graph per A/B parity
    cudaGraphExec_t bspan[2];  // span consecutive steps per launch (span > 1), per starting parity
    int span;
    cudaEvent_t ev_fork;
    cudaEvent_t *ev_join;
    int pipe;                  // ELBM_BATCH_PIPELINE: odd positions run half a step ahead
};

namespace {

// The potential for the caller: with the deviation form the plane holds
// psi = phi - phi_lin; add the linear electrode profile back at non-solid
// nodes (solid nodes keep the plane's value, as without it)
__global__ void k_add_profile(double *out, Geom g, double phi_lo, double slope, const unsigned char *mask)
{
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= g.N) return;
    if (mask && mask[i] == ELBM_NODE_SOLID) return;
    const long long c = g.phi_axis == 0 ? i % g.nx : (g.phi_axis == 1 ? (i / g.nx) % g.ny : i / ((long long)g.nx * g.ny));
    out[i] += phi_lo + double(c + 1) * slope;
}

// BF16 image of the learned proposal's network (shared-memory layout of
// elbm_mlp.cuh) from the caller's FP32 parameters, made once at elbm_init
__global__ void k_mlp_image(const float *th, MlpSmem *img)
{
    __shared__ MlpSmem sm;
    mlp_load_smem(th, sm);
    const uint4 *src = (const uint4 *)&sm;
    uint4 *dst = (uint4 *)img;
    for (int i = threadIdx.x; i < (int)(sizeof(MlpSmem) / 16); i += blockDim.x) dst[i] = src[i];
}

enum { FIN_CHARGE_AB = 0, FIN_CHARGE_Q = 1, FIN_RESID_PRE = 2, FIN_PHI = 3, FIN_DIAG = 4, FIN_RESID_BODY = 5,
       FIN_INLET = 6 };

// Control of the Poisson loop, evaluated on the device after each
// convergence test (so the loop can run inside a CUDA graph).
struct Ctl {
    unsigned long long cond;   // cudaGraphConditionalHandle of the while node
    int use_cond;              // 1 inside a captured graph
    int fixed;                 // > 0: exactly this many units
    int units_max;
    int reduced;               // FP32 potential: stop at the rounding floor
    int ce;
    int steps;                 // FIN_DIAG: time steps these diagnostics close (the step counter's increment)
};

// Sum (or min / max) each of the K columns of the per-block partials in a
// fixed order, then derive the scalars of `mode`. One block of kFinThreads
// per column, each thread with kFinAcc independent accumulators (so that
// that many loads are in flight: a lattice of 50 M sites has 400 k partials
// per column): run-to-run reproducible.
constexpr int kFinThreads = 1024, kFinAcc = 8;
constexpr int kMaxCols = 32;  // columns a finalize reduces at most (diagnostics: D_NPART + 1)
static_assert(D_NPART + 1 <= kMaxCols, "finalize columns");
__device__ __forceinline__ double fin_op(int op, double a, double v)
{
    return op == 0 ? a + v : (op == 1 ? fmin(a, v) : fmax(a, v));
}
__global__ void __launch_bounds__(kFinThreads) k_finalize(const double *part, int nblocks, int K, int mode, Phys ph,
                                                          Ctl ctl, double *scal, float *scalf, double *diag,
                                                          double *colres, unsigned int *ticket)
{
    // block k reduces column k of the column-major partials in a fixed order
    __shared__ double wsum[kFinThreads / 32];
    __shared__ bool last;
    const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
    const int k = blockIdx.x;
    int op = 0;  // 0 sum, 1 min, 2 max
    if (mode == FIN_DIAG) {
        if (k == D_AMIN) op = 1;
        else if (k == D_AMAX || k == D_HERR || k == D_UMAX) op = 2;
    }
    const double id = op == 1 ? 1e300 : (op == 2 ? -1e300 : 0.0);
    const double *col = part + (long long)k * nblocks;
    double a[kFinAcc];
#pragma unroll
    for (int j = 0; j < kFinAcc; j++) a[j] = id;
    int i = t;
    for (; i + (kFinAcc - 1) * kFinThreads < nblocks; i += kFinAcc * kFinThreads) {
        double v[kFinAcc];
#pragma unroll
        for (int j = 0; j < kFinAcc; j++) v[j] = col[i + j * kFinThreads];
#pragma unroll
        for (int j = 0; j < kFinAcc; j++) a[j] = fin_op(op, a[j], v[j]);
    }
    for (; i < nblocks; i += kFinThreads) a[0] = fin_op(op, a[0], col[i]);
    double acc = a[0];
#pragma unroll
    for (int j = 1; j < kFinAcc; j++) acc = fin_op(op, acc, a[j]);
    for (int o = 16; o > 0; o >>= 1) acc = fin_op(op, acc, __shfl_down_sync(0xffffffffu, acc, o));
    if (lane == 0) wsum[warp] = acc;
    __syncthreads();
    if (t == 0) {
        double r = wsum[0];
        for (int w = 1; w < kFinThreads / 32; w++) r = fin_op(op, r, wsum[w]);
        colres[k] = r;
        __threadfence();
        unsigned int tk = atomicAdd(ticket, 1u);
        last = (tk == gridDim.x - 1);
    }
    __syncthreads();
    if (!last || t != 0) return;
    // the last block to finish derives the scalars of `mode`
    __threadfence();
    *ticket = 0u;
    double res[kMaxCols];
    for (int c = 0; c < K && c < kMaxCols; c++) res[c] = ((volatile double *)colres)[c];
    if (mode == FIN_CHARGE_AB) {
        // the factors of Eq. (surface-q2): Q_b / sum(rho theta), Q_s / sum(|grad rho|^2 (1 + ...))
        scal[S_SA] = res[0] > 0.0 ? ph.cd.Qb / res[0] : 0.0;
        scal[S_SB] = res[1] > 0.0 ? ph.cd.Qs / res[1] : 0.0;
    } else if (mode == FIN_CHARGE_Q) {
        scal[S_QSUM] = res[0];
        scal[S_Q2] = res[1];
        scal[S_QMEAN] = (ph.neutralize && ph.n_fluid > 0) ? res[0] / ph.n_fluid : 0.0;
    } else if (mode == FIN_RESID_PRE || mode == FIN_RESID_BODY) {
        scal[S_HAVE_OLD] = 1.0;
        double rn = sqrt(res[0]), ref = sqrt(res[1]) + sqrt(res[2]);
        scal[S_RESID] = ref > 0.0 ? rn / ref : rn;
        double iter = mode == FIN_RESID_PRE ? 0.0 : scal[S_ITER] + 1.0;
        scal[S_ITER] = iter;
        if (mode == FIN_RESID_BODY) scal[S_ITER_TOTAL] += 1.0;
        bool conv = rn <= ph.tol * ref;
        // FP32 potential: stop at its rounding floor, once the residual is
        // within 2^-23 |t| (t: magnitude of the residual's terms), or when a
        // test interval brought no progress within 2^-17 |t|
        if (!conv && ctl.reduced && rn <= 0x1p-23 * sqrt(res[3])) conv = true;
        // (the no-progress rule only near the floor: SOR's residual is not
        // monotone early in a solve)
        if (!conv && ctl.reduced && mode == FIN_RESID_BODY && rn > 0.97 * scal[S_PREV] &&
            rn <= 0x1p-17 * sqrt(res[3]))
            conv = true;
        scal[S_PREV] = rn;
        scal[S_CONV] = conv ? 1.0 : 0.0;
        bool keep;
        if (ctl.fixed > 0) {
            keep = iter < ctl.fixed;
        } else {
            keep = !conv && iter < ctl.units_max;
            if (!conv && iter >= ctl.units_max) scal[S_NOCONV] += 1.0;
        }
        scal[S_KEEP] = keep ? 1.0 : 0.0;
        if (ctl.use_cond) cudaGraphSetConditional(ctl.cond, keep ? 1u : 0u);
    } else if (mode == FIN_PHI) {
        scal[S_PHISUM] = res[0];
        scal[S_PHIMEAN] = res[0] / ph.n_unknown;
    } else if (mode == FIN_INLET) {
        // adaptive inlet: the nozzle mean along d over the initial profile's mean
        const double r = (ph.n_region > 0.0 && ph.in_m0 != 0.0) ? (res[0] / ph.n_region) / ph.in_m0 : 1.0;
        scal[S_INRATIO] = r;
        diag[22] = r;
    } else if (mode == FIN_DIAG) {
        diag[0] = res[D_MASS];
        diag[1] = res[D_MX];
        diag[2] = res[D_MY];
        diag[3] = res[D_MZ];
        diag[4] = res[D_Q];
        diag[5] = res[D_AMIN];
        diag[6] = res[D_AMAX];
        diag[7] = res[D_NFLUID] > 0 ? res[D_ASUM] / res[D_NFLUID] : 0.0;
        diag[8] = res[D_NSHORT];
        diag[9] = res[D_NNOROOT];
        diag[10] = res[D_NCLIP];
        diag[11] = scal[S_ITER] * ctl.ce;
        diag[12] = scal[S_RESID];
        // the sticky record of the steps without diagnostics since the
        // last ones (k-step graphs, diag_every > 1) folds in, then restarts
        volatile unsigned int *sk = ticket + 2;
        const unsigned int sflags = sk[1];
        diag[13] = fmax(res[D_HERR], (double)__uint_as_float(sk[0]));
        diag[14] = res[D_UMAX];
        diag[15] = res[D_NBAD] + ((sflags & 1u) ? 1.0 : 0.0);
        diag[16] = scal[S_QMEAN];
        scal[S_STEPS] += double(ctl.steps);
        diag[17] = scal[S_STEPS];
        diag[18] = scal[S_ITER_TOTAL] * ctl.ce;
        diag[19] = res[D_NGUARD];
        diag[20] = res[D_NGFAIL] + ((sflags & 2u) ? 1.0 : 0.0);
        diag[21] = res[D_NLFALL];
        diag[23] = (double)sflags;
        sk[0] = 0u;
        sk[1] = 0u;
    }
    for (int i = 0; i < S_NSCAL; i++) scalf[i] = (float)scal[i];
}

bool cuda_ok(cudaError_t e) { return e == cudaSuccess; }

int validate(const elbm_params *p, const elbm_init_fields *in, int n_instances)
{
    if (!p || !in || !in->rho0 || n_instances != 1) return 1;
    if (p->nx < 1 || p->ny < 1 || p->nz < 1) return 1;
    if ((long long)p->nx * p->ny * p->nz >= (1LL << 31)) return 1;  // 32-bit site indices
    for (int f = 0; f < 6; f++) {
        if (p->face_bc[f] != ELBM_FACE_PERIODIC && p->face_bc[f] != ELBM_FACE_WALL) return 1;
        if (p->phi_bc[f] < ELBM_PHI_PERIODIC || p->phi_bc[f] > ELBM_PHI_NEUMANN) return 1;
        if ((p->face_bc[f] == ELBM_FACE_PERIODIC) != (p->phi_bc[f] == ELBM_PHI_PERIODIC)) return 1;
    }
    for (int a = 0; a < 3; a++)
        if ((p->face_bc[2 * a] == ELBM_FACE_PERIODIC) != (p->face_bc[2 * a + 1] == ELBM_FACE_PERIODIC)) return 1;
    if (p->phi_axis < 0 || p->phi_axis > 2) return 1;
    if (p->charge_model < ELBM_CHARGE_NONE || p->charge_model > ELBM_CHARGE_TRANSPORT) return 1;
    if (p->force_el != ELBM_FEL_QE && p->force_el != ELBM_FEL_FULL) return 1;
    if (p->eps_face != ELBM_EPS_FACE_ARITH && p->eps_face != ELBM_EPS_FACE_HARMONIC) return 1;
    if (p->carreau_lagged != 0 && p->carreau_lagged != 1) return 1;
    if (p->alpha_mode < ELBM_ALPHA_ENTROPIC || p->alpha_mode > ELBM_ALPHA_LEARNED) return 1;
    // the learned proposal starts the FP32 Newton iteration of FP32/BF16 storage
    if (p->alpha_mode == ELBM_ALPHA_LEARNED &&
        (!p->mlp || p->precision == ELBM_PREC_FP64 || p->alpha_precision == ELBM_APREC_FP64))
        return 1;
    if (p->precision < ELBM_PREC_FP64 || p->precision > ELBM_PREC_BF16) return 1;
    if (p->alpha_precision < ELBM_APREC_FP64 || p->alpha_precision > ELBM_APREC_FP32_FAST) return 1;
    if (!(p->nu0 > 0.0) || !(p->nu_inf > 0.0) || !(p->rho0 > 0.0)) return 1;
    if (!(p->n_carreau > 0.0) || !(p->lambda >= 0.0)) return 1;
    // FP32 arithmetic leaves about 3e-7 of noise in Delta_p/f_p; an alpha root
    // sought below a few times that is a root of rounding noise
    if (p->precision != ELBM_PREC_FP64 && !(p->alpha_eq_tol >= 0x1p-18)) return 1;
    if (!(p->alpha_h_tol >= 0.0) || !(p->alpha_h_tol < 1.0)) return 1;
    if (p->charge_model != ELBM_CHARGE_NONE) {
        if (!(p->theta_width > 0.0) || !(p->K_d > 0.0)) return 1;
        if (!(p->sor_omega > 0.0 && p->sor_omega < 2.0)) return 1;
        if (!(p->poisson_tol >= 0.0) || p->poisson_maxit < 0 || p->poisson_fixed_sweeps < 0) return 1;
    }
    if (p->charge_model == ELBM_CHARGE_TRANSPORT && !(p->Dq >= 0.0)) return 1;
    if (p->diag_every < 0) return 1;
    if (p->poisson_solver != ELBM_POISSON_SOR && p->poisson_solver != ELBM_POISSON_MG) return 1;
    if (p->autotune != 0 && p->autotune != 1) return 1;
    if (p->velset != ELBM_VSET_D3Q19 && p->velset != ELBM_VSET_D2Q9) return 1;
    if (p->velset == ELBM_VSET_D2Q9) {
        // one site thick, potential data in the plane
        if (p->nz != 1 || p->phi_axis > 1 || p->E_ext[2] != 0.0) return 1;
        // the kernels built for D2Q9: FP64 / FP32 populations, FP64 or guarded FP32 root, SOR
        if (p->precision == ELBM_PREC_BF16 || p->alpha_mode == ELBM_ALPHA_LEARNED ||
            p->alpha_precision == ELBM_APREC_FP32_FAST)
            return 1;
        if (p->charge_model == ELBM_CHARGE_TRANSPORT || p->poisson_solver != ELBM_POISSON_SOR) return 1;
    }
    return 0;
}

void free_bufs(elbm_handle *h)
{
    if (h->arena) cudaFree(h->arena);  // every device buffer of the handle
    h->arena = nullptr;
    if (h->xtmp) cudaFree(h->xtmp);
    h->xtmp = nullptr;
    if (h->pin) cudaFreeHost(h->pin);
    for (int i = 0; i < 5; i++)
        if (h->ev[i]) cudaEventDestroy(h->ev[i]);
    for (int i = 0; i < 2; i++) {
        if (h->gexec[i]) cudaGraphExecDestroy(h->gexec[i]);
        for (int k = 0; k < 3; k++)
            if (h->gsec[i][k]) cudaGraphExecDestroy(h->gsec[i][k]);
    }
    if (h->cap) cudaStreamDestroy(h->cap);
    if (h->cap2) cudaStreamDestroy(h->cap2);
}

Ctl make_ctl(const elbm_handle *h, unsigned long long cond, int use_cond)
{
    Ctl c;
    c.cond = cond;
    c.use_cond = use_cond;
    c.fixed = h->p.poisson_fixed_sweeps;
    c.units_max = h->units_max;
    c.reduced = h->p.precision != ELBM_PREC_FP64;
    c.ce = h->ce;
    c.steps = 1;
    return c;
}

int fin(elbm_handle *h, const Bufs &b, cudaStream_t s, int K, int mode, unsigned long long cond = 0,
        int use_cond = 0, int steps = 1, int nblocks = 0)
{
    Ctl c = make_ctl(h, cond, use_cond);
    c.steps = steps;
    // nblocks: the block count of the kernel that wrote the partials (its
    // own column stride); 0 = the site kernels' shape
    k_finalize<<<K, kFinThreads, 0, s>>>(b.part, nblocks > 0 ? nblocks : h->L.nblocks, K, mode, h->ph, c, b.scal,
                                         b.scalf, b.diag, b.colres, b.ticket);
    return 1;
}

// adaptive inlet, after the collision: the profile scale from the region's
// block sums (their own column of the partials), then the inlet equilibria
// into the buffer of the next step
int enq_inlet(elbm_handle *h, const Bufs &b, cudaStream_t s)
{
    if (!h->ph.adaptive) return 0;
    Ctl c = make_ctl(h, 0, 0);
    k_finalize<<<1, kFinThreads, 0, s>>>(b.part + (long long)D_UIN * h->L.nblocks, h->L.nblocks, 1, FIN_INLET, h->ph, c,
                                 b.scal, b.scalf, b.diag, b.colres, b.ticket);
    h->ops.inlet(h->g, h->ph, b, s);
    return 2;
}

// The colour of the fine level that the multigrid's red-black Gauss-Seidel
// smoothing updates last, whose residual (the rounding of that update) the
// residual passes take as 0 in reduced precision; -1 where they take every
// site (FP64, which follows the oracle's procedure; SOR, whose over-relaxed
// update leaves (1 - omega) of the residual; three-colour orderings).
int gs_settled(const elbm_handle *h)
{
    return (h->nlev > 0 && h->p.precision != ELBM_PREC_FP64 && h->g.ncol == 2) ? 1 : -1;
}

int vcycle(elbm_handle *h, const Bufs &b, cudaStream_t s, int l)
{
    const MGOps &m = h->mg;
    if (l == h->lt) {
        m.tail(h->g, h->tail, h->p.precision == ELBM_PREC_FP64 ? kNu : kNuTail, s);
        return 1;
    }
    const int nc = h->lev[l].ncol;
    const bool fp64 = h->p.precision == ELBM_PREC_FP64;
    const int pre = fp64 ? kNu : kNuPre, post = fp64 ? kNu : kNuPost;
    for (int i = 0; i < pre; i++)
        for (int c = 0; c < nc; c++) m.smooth(h->g, h->ph, b, h->lev[l], l, c, h->Lh, s);
    m.restrict_(h->g, h->ph, b, h->lev[l], h->lev[l + 1], l, l == 0 ? gs_settled(h) : -1, s);
    int n = vcycle(h, b, s, l + 1);
    m.prolong(h->g, b, h->lev[l], h->lev[l + 1], l, s);
    for (int i = 0; i < post; i++)
        for (int c = 0; c < nc; c++) m.smooth(h->g, h->ph, b, h->lev[l], l, c, h->Lh, s);
    return n + nc * (pre + post) + 2;
}

// moments, and the free charge with its global sums (Sec. II C, item 3)
int enq_pre(elbm_handle *h, const Bufs &b, cudaStream_t s)
{
    const Ops &o = h->ops;
    int n = 1;
    o.moments(h->g, h->ph, b, h->L, s);
    const int cm = h->p.charge_model;
    if (cm == ELBM_CHARGE_TRANSPORT) {
        n += fin(h, b, s, 2, FIN_CHARGE_Q);
    } else if (cm == ELBM_CHARGE_CONSERVED) {
        o.charge(h->g, h->ph, b, 0, h->L, s);
        n += 2 + fin(h, b, s, 2, FIN_CHARGE_AB);
        o.charge(h->g, h->ph, b, 1, h->L, s);
        n += 1 + fin(h, b, s, 2, FIN_CHARGE_Q);
    } else if (cm == ELBM_CHARGE_XI) {
        // Eq. (surface-q3) needs no global sum: the second charge kernel
        // writes q with its sums (q, q^2)
        o.charge(h->g, h->ph, b, 0, h->L, s);
        n += 2 + fin(h, b, s, 2, FIN_CHARGE_Q);
    }
    return n;
}

// the extrapolated warm start (not with a fixed sweep count, which the
// caller means as an exact number of smoothing sweeps from phi(t-1))
int enq_eps(elbm_handle *h, const Bufs &b, cudaStream_t s)
{
    // (the coarse permittivities of the multigrid come with each restriction)
    if (!b.phi_old) return 0;
    h->ops.phi_extrap(h->g, b, s);
    return 1;
}

// convergence test: residual sums, then the device-side decision
int enq_check(elbm_handle *h, const Bufs &b, cudaStream_t s, int mode, unsigned long long cond, int use_cond)
{
    // with a settled colour the residual runs one thread per pair of x
    // (the half-row shape of the red-black sweeps)
    const int zc = mode == FIN_RESID_BODY ? gs_settled(h) : -1;
    const Launch &L = zc >= 0 ? h->Lh : h->L;
    h->ops.resid(h->g, h->ph, b, zc, L, s);
    return 1 + fin(h, b, s, 4, mode, cond, use_cond, 1, L.nblocks);
}

// one Poisson unit: a V-cycle, or ce red-black SOR sweeps
int enq_unit(elbm_handle *h, const Bufs &b, cudaStream_t s)
{
    if (h->nlev > 0) return vcycle(h, b, s, 0);
    for (int i = 0; i < h->ce; i++)
        for (int c = 0; c < h->g.ncol; c++) h->ops.sor(h->g, h->ph, b, c, h->Lh, s);
    return h->g.ncol * h->ce;
}

// zero-mean potential when nothing pins its constant
int enq_shift(elbm_handle *h, const Bufs &b, cudaStream_t s)
{
    if (h->has_dirichlet) return 0;
    h->ops.phi_mean(h->g, h->ph, b, 0, h->L, s);
    int n = 1 + fin(h, b, s, 1, FIN_PHI);
    h->ops.phi_mean(h->g, h->ph, b, 1, h->L, s);
    return n + 1;
}

void swap_ab(Bufs &b)
{
    void *t = b.fA; b.fA = b.fB; b.fB = t;
    t = b.gA; b.gA = b.gB; b.gB = t;
    float *r = b.rA; b.rA = b.rB; b.rB = r;
}

// One step issued from the host; the Poisson loop reads the device decision
// after each test (a host synchronisation per test).
elbm_status step_host(elbm_handle *h, bool diag)
{
    const bool prof = h->p.profile != 0;
    cudaStream_t s = h->s;
    const Bufs &b = h->b;
    const bool charged = h->p.charge_model != ELBM_CHARGE_NONE;
    if (prof) cudaEventRecord(h->ev[0], s);
    h->launches += enq_pre(h, b, s);
    if (prof) cudaEventRecord(h->ev[1], s);
    if (charged) {
        h->launches += enq_eps(h, b, s);
        const bool dowhile = b.phi_old != nullptr;
        if (!dowhile) h->launches += enq_check(h, b, s, FIN_RESID_PRE, 0, 0);
        for (bool first = true;; first = false) {
            if (!(dowhile && first)) {
                if (!cuda_ok(cudaMemcpyAsync(h->pin, b.scal + S_KEEP, sizeof(double), cudaMemcpyDeviceToHost, s)) ||
                    !cuda_ok(cudaStreamSynchronize(s)))
                    return ELBM_E_CUDA;
                if (h->pin[0] == 0.0) break;
            }
            h->launches += enq_unit(h, b, s);
            h->launches += enq_check(h, b, s, FIN_RESID_BODY, 0, 0);
        }
        h->launches += enq_shift(h, b, s);
    }
    if (prof) cudaEventRecord(h->ev[2], s);
    if (h->ph.force_el == ELBM_FEL_FULL) {
        h->ops.efield2(h->g, h->ph, b, h->L, s);
        h->launches += 1;
    }
    h->ops.collide(h->g, h->ph, b, diag ? 1 : 0, h->L, s);
    h->launches += 1;
    if (prof) cudaEventRecord(h->ev[3], s);
    if (diag) h->launches += fin(h, b, s, D_NPART, FIN_DIAG);
    h->launches += enq_inlet(h, b, s);
    if (prof) cudaEventRecord(h->ev[4], s);
    return cuda_ok(cudaGetLastError()) ? ELBM_OK : ELBM_E_CUDA;
}

// Capture sections of one step into an executable graph for buffers of the
// given A/B parity: bit 0 moments and charge, bit 1 the Poisson loop (a
// device-side while node), bit 2 collision and diagnostics.
// One step of h enqueued into stream s, which is being captured (the Poisson
// loop becomes a conditional while node whose body is captured on h->cap2).
// Kernel priorities in a captured graph: every kernel node except the
// site-wide compute kernels (Ops::heavy) gets the device's highest stream
// priority, so that when several instances share the GPU the block scheduler
// serves the short, latency-bound Poisson chain of one instance ahead of the
// pending blocks of another's collision. Takes effect in graphs instantiated
// with cudaGraphInstantiateFlagUseNodePriority.
bool prioritize(cudaGraph_t graph, const std::vector<const void *> &heavy_fns)
{
    int least = 0, greatest = 0;
    if (!cuda_ok(cudaDeviceGetStreamPriorityRange(&least, &greatest))) return false;
    size_t n = 0;
    if (!cuda_ok(cudaGraphGetNodes(graph, nullptr, &n))) return false;
    std::vector<cudaGraphNode_t> nodes(n);
    if (n && !cuda_ok(cudaGraphGetNodes(graph, nodes.data(), &n))) return false;
    for (cudaGraphNode_t node : nodes) {
        cudaGraphNodeType type;
        if (!cuda_ok(cudaGraphNodeGetType(node, &type))) return false;
        if (type != cudaGraphNodeTypeKernel) continue;
        cudaKernelNodeParams kp;
        if (!cuda_ok(cudaGraphKernelNodeGetParams(node, &kp))) return false;
        bool heavy = false;
        for (const void *f : heavy_fns) heavy = heavy || (f && kp.func == f);
        if (heavy) continue;
        cudaKernelNodeAttrValue v;
        std::memset(&v, 0, sizeof(v));
        v.priority = greatest;
        if (!cuda_ok(cudaGraphKernelNodeSetAttribute(node, cudaKernelNodeAttributePriority, &v))) return false;
    }
    return true;
}

// diag_steps: the collision's diagnostics and their finalize close this
// many steps (the step counter advances by it); 0 skips both, for a step
// inside a multi-step graph whose diagnostics the last step supersedes.
bool enqueue_step(elbm_handle *h, int parity, cudaStream_t s, int sections, int &n_pre, int &n_body, int &n_post,
                  int diag_steps = 1)
{
    Bufs b = h->b;
    if (parity) swap_ab(b);
    const bool charged = h->p.charge_model != ELBM_CHARGE_NONE && (sections & 2);
    bool ok = true;
    cudaGraphConditionalHandle cond = 0;
    if (sections & 1) n_pre += enq_pre(h, b, s);
    if (charged) {
        cudaStreamCaptureStatus st;
        cudaGraph_t cg = nullptr;
        const cudaGraphNode_t *deps = nullptr;
        size_t nd = 0;
        ok = ok && cuda_ok(cudaStreamGetCaptureInfo(s, &st, nullptr, &cg, &deps, nullptr, &nd));
        // do-while (reduced precision, extrapolated start): the loop's first
        // unit runs untested; else the test before the loop decides
        const bool dowhile = b.phi_old != nullptr;
        ok = ok && cuda_ok(cudaGraphConditionalHandleCreate(&cond, cg, dowhile ? 1u : 0u, cudaGraphCondAssignDefault));
        n_pre += enq_eps(h, b, s);
        if (!dowhile) n_pre += enq_check(h, b, s, FIN_RESID_PRE, cond, 1);
        cudaGraphNode_t node;
        cudaGraphNodeParams np = {cudaGraphNodeTypeConditional};
        np.conditional.handle = cond;
        np.conditional.type = cudaGraphCondTypeWhile;
        np.conditional.size = 1;
        ok = ok && cuda_ok(cudaStreamGetCaptureInfo(s, &st, nullptr, &cg, &deps, nullptr, &nd));
        ok = ok && cuda_ok(cudaGraphAddNode(&node, cg, deps, nullptr, nd, &np));
        if (ok) {
            cudaGraph_t body = np.conditional.phGraph_out[0];
            ok = cuda_ok(cudaStreamBeginCaptureToGraph(h->cap2, body, nullptr, nullptr, 0,
                                                       cudaStreamCaptureModeThreadLocal));
            if (ok) {
                n_body += enq_unit(h, b, h->cap2);
                n_body += enq_check(h, b, h->cap2, FIN_RESID_BODY, cond, 1);
                ok = cuda_ok(cudaStreamEndCapture(h->cap2, &body));
                ok = ok && prioritize(body, std::vector<const void *>(h->ops.heavy, h->ops.heavy + 5));
            }
            ok = ok && cuda_ok(cudaStreamUpdateCaptureDependencies(s, &node, nullptr, 1,
                                                                   cudaStreamSetCaptureDependencies));
        }
        n_post += enq_shift(h, b, s);
    }
    if (sections & 4) {
        if (h->ph.force_el == ELBM_FEL_FULL) {
            h->ops.efield2(h->g, h->ph, b, h->L, s);
            n_post += 1;
        }
        h->ops.collide(h->g, h->ph, b, diag_steps > 0 ? 1 : 0, h->L, s);
        n_post += 1;
        if (diag_steps > 0) n_post += fin(h, b, s, D_NPART, FIN_DIAG, 0, 0, diag_steps);
        n_post += enq_inlet(h, b, s);
    }
    return ok;
}

// The step's diagnostics and the Poisson no-convergence counter, copied into
// pinned host memory as the last nodes of a step graph: elbm_step checks the
// status words there after one wait on the stream, and elbm_fields serves
// ELBM_F_DIAG from the copy, with no synchronous copies per step.
constexpr int kPinDiag = 16;
bool enqueue_status(elbm_handle *h, cudaStream_t s)
{
    return cuda_ok(cudaMemcpyAsync(h->pin + kPinDiag, h->b.diag, ELBM_NDIAG * sizeof(double), cudaMemcpyDeviceToHost,
                                   s)) &&
           cuda_ok(cudaMemcpyAsync(h->pin + 9, h->b.scal + S_NOCONV, sizeof(double), cudaMemcpyDeviceToHost, s));
}

bool capture_step(elbm_handle *h, int parity, cudaGraphExec_t *out, int sections = 7)
{
    cudaStream_t s = h->cap;
    cudaGraph_t graph = nullptr;
    if (!cuda_ok(cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal))) return false;
    int n_pre = 0, n_body = 0, n_post = 0;
    bool ok = enqueue_step(h, parity, s, sections, n_pre, n_body, n_post);
    if (sections == 7) ok = ok && enqueue_status(h, s);
    ok = cuda_ok(cudaStreamEndCapture(s, &graph)) && ok;
    if (ok) ok = cuda_ok(cudaGraphInstantiate(out, graph, 0));
    if (graph) cudaGraphDestroy(graph);
    cudaGetLastError();
    if (parity == 0) {  // kernels per section, counted once
        h->n_pre += n_pre;
        h->n_body += n_body;
        h->n_post += n_post;
    }
    return ok;
}

// The batch's step for one A/B parity: every instance's step as a parallel
// branch (fork from one event, join into the batch's capture stream). With
// pipelining, an instance at an odd position runs its collision of this step
// and then the moments and potential solve of the next one, so that its
// latency-bound solve overlaps the other instances' collisions and the
// reverse; its prologue (prologue = true) is the first step's moments and
// solve alone.
bool capture_batch(elbm_handle *B, int parity, cudaGraphExec_t *out, bool prologue = false, int steps = 1)
{
    cudaStream_t s = B->cap;
    cudaGraph_t graph = nullptr;
    if (!cuda_ok(cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal))) return false;
    bool ok = cuda_ok(cudaEventRecord(B->ev_fork, s));
    int n_pre = 0, n_body = 0, n_post = 0;
    for (int i = 0; i < B->n_sub && ok; i++) {
        elbm_handle *h = B->sub[i];
        const bool ahead = B->pipe && (i & 1);
        if (prologue && !ahead) continue;
        ok = cuda_ok(cudaStreamWaitEvent(h->cap, B->ev_fork, 0));
        for (int k = 0; k < (prologue ? 1 : steps); k++) {  // consecutive steps: one chain
            const int par = parity ^ (k & 1);
            // diagnostics once, on the last step, closing all `steps` of them
            const int dsteps = k == steps - 1 ? steps : 0;
            if (prologue) {
                ok = ok && enqueue_step(h, par, h->cap, 3, n_pre, n_body, n_post);
            } else if (ahead) {
                ok = ok && enqueue_step(h, par, h->cap, 4, n_pre, n_body, n_post, dsteps);
                ok = ok && enqueue_step(h, par ^ 1, h->cap, 3, n_pre, n_body, n_post);
            } else {
                ok = ok && enqueue_step(h, par, h->cap, 7, n_pre, n_body, n_post, dsteps);
            }
        }
        if (!prologue) ok = ok && enqueue_status(h, h->cap);
        ok = ok && cuda_ok(cudaEventRecord(B->ev_join[i], h->cap));
        ok = ok && cuda_ok(cudaStreamWaitEvent(s, B->ev_join[i], 0));
    }
    if (prologue || steps > 1) parity = 1;  // kernel counts belong to the one-step graphs
    ok = cuda_ok(cudaStreamEndCapture(s, &graph)) && ok;
    std::vector<const void *> heavy;
    for (int i = 0; i < B->n_sub; i++) heavy.insert(heavy.end(), B->sub[i]->ops.heavy, B->sub[i]->ops.heavy + 5);
    ok = ok && prioritize(graph, heavy);
    if (ok) ok = cuda_ok(cudaGraphInstantiate(out, graph, cudaGraphInstantiateFlagUseNodePriority));
    if (graph) cudaGraphDestroy(graph);
    cudaGetLastError();
    if (parity == 0) {
        B->n_pre = n_pre;
        B->n_body = n_body;
        B->n_post = n_post;
    }
    return ok;
}

// ---------------------------------------------------------------------------
// Launch-shape autotuner: the block shape of the site kernels (128 threads,
// bx x by) chosen by timing the collision launch on the handle's own state;
// cached per lattice size, precision and alpha settings for the process.
// ---------------------------------------------------------------------------
constexpr int kShapes[5][2] = {{128, 1}, {64, 2}, {32, 4}, {16, 8}, {8, 16}};

void set_launch(Launch &L, int bx, int by, const elbm_params *p)
{
    L.block = dim3(bx, by, 1);
    L.grid = dim3((p->nx + bx - 1) / bx, (p->ny + by - 1) / by, p->nz);
    L.nblocks = (int)(L.grid.x * L.grid.y * L.grid.z);
}

long long max_blocks_over_shapes(const elbm_params *p)
{
    long long m = 0;
    for (auto &c : kShapes) {
        long long nb = (long long)((p->nx + c[0] - 1) / c[0]) * ((p->ny + c[1] - 1) / c[1]) * p->nz;
        if (nb > m) m = nb;
    }
    return m;
}

std::mutex g_tune_mutex;
std::map<std::array<int, 8>, int> g_tune_cache;

bool autotune(elbm_handle *h)
{
    const elbm_params *p = &h->p;
    const std::array<int, 8> key = {p->nx, p->ny, p->nz, p->precision, h->ph.aprec, p->alpha_mode,
                                    p->charge_model, h->g.has_mask};
    {
        std::lock_guard<std::mutex> lock(g_tune_mutex);
        auto it = g_tune_cache.find(key);
        if (it != g_tune_cache.end()) {
            set_launch(h->L, kShapes[it->second][0], kShapes[it->second][1], p);
            return true;
        }
    }
    cudaEvent_t e0, e1;
    if (!cuda_ok(cudaEventCreate(&e0))) return false;
    if (!cuda_ok(cudaEventCreate(&e1))) { cudaEventDestroy(e0); return false; }
    int best = -1;
    float best_ms = 1e30f;
    bool ok = true;
    for (int c = 0; c < 5 && ok; c++) {
        if (kShapes[c][0] > 32 && kShapes[c][0] / 2 >= p->nx) continue;  // half the block idle
        set_launch(h->L, kShapes[c][0], kShapes[c][1], p);
        if (h->L.grid.y > 65535) continue;
        h->ops.collide(h->g, h->ph, h->b, 1, h->L, h->s);  // warm-up
        ok = cuda_ok(cudaEventRecord(e0, h->s));
        for (int r = 0; r < 3; r++) h->ops.collide(h->g, h->ph, h->b, 1, h->L, h->s);
        ok = ok && cuda_ok(cudaEventRecord(e1, h->s)) && cuda_ok(cudaEventSynchronize(e1));
        float ms = 0.f;
        ok = ok && cuda_ok(cudaEventElapsedTime(&ms, e0, e1));
        if (ok && ms < best_ms) { best_ms = ms; best = c; }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (!ok || best < 0) return false;
    set_launch(h->L, kShapes[best][0], kShapes[best][1], p);
    std::lock_guard<std::mutex> lock(g_tune_mutex);
    g_tune_cache[key] = best;
    return true;
}

}  // namespace

extern "C" {

const char *elbm_strerror(int st)
{
    switch (st) {
    case ELBM_OK: return "ok";
    case ELBM_W_POISSON_NOCONV: return "Poisson solve reached its sweep cap";
    case ELBM_E_INVAL: return "invalid argument";
    case ELBM_E_NOMEM: return "out of memory";
    case ELBM_E_CUDA: return "CUDA runtime error";
    case ELBM_E_NUMERIC: return "non-finite value or non-positive density";
    case ELBM_E_STATE: return "request not possible in this state";
    default: return "unknown status";
    }
}

int elbm_velocity_set(int *c, double *w)
{
    for (int p = 0; p < Q; p++) {
        if (c) { c[3 * p] = cx(p); c[3 * p + 1] = cy(p); c[3 * p + 2] = cz(p); }
        if (w) w[p] = wq(p);
    }
    return Q;
}

int elbm_velocity_set_of(int velset, int *c, double *w)
{
    if (velset == ELBM_VSET_D3Q19) return elbm_velocity_set(c, w);
    if (velset == ELBM_VSET_D2Q9) return vset_d2q9(c, w);
    return ELBM_E_INVAL;
}

elbm_status elbm_init(const elbm_params *p, const elbm_init_fields *in, int n_instances,
                      elbm_handle **out)
{
    if (!out) return ELBM_E_INVAL;
    *out = nullptr;
    if (validate(p, in, n_instances)) return ELBM_E_INVAL;
    elbm_handle *h = new (std::nothrow) elbm_handle;
    if (!h) return ELBM_E_NOMEM;
    std::memset(h, 0, sizeof(*h));
    h->p = *p;
    h->s = (cudaStream_t)p->cuda_stream;
    const long long N = (long long)p->nx * p->ny * p->nz;

    Geom &g = h->g;
    g.nx = p->nx; g.ny = p->ny; g.nz = p->nz; g.N = N;
    for (int a = 0; a < 3; a++) g.per[a] = p->face_bc[2 * a] == ELBM_FACE_PERIODIC;
    for (int f = 0; f < 6; f++) g.phi_kind[f] = p->phi_bc[f];
    h->Q = p->velset == ELBM_VSET_D2Q9 ? vset_d2q9(nullptr, nullptr) : Q;
    if (p->velset == ELBM_VSET_D2Q9) {
        // the one-site-thick z axis: no population crosses it (c_z = 0) and
        // the potential has no flux through its faces
        g.per[2] = 0;
        g.phi_kind[4] = g.phi_kind[5] = ELBM_PHI_NEUMANN;
    }
    g.ncol = ncolors_of(g.per, p->nx, p->ny, p->nz);
    g.phi_axis = p->phi_axis;
    // reduced precision: the potential plane holds its deviation from the
    // linear profile between the electrodes (both faces of phi_axis Dirichlet)
    g.phi_lin = p->precision != ELBM_PREC_FP64 && p->charge_model != ELBM_CHARGE_NONE &&
                p->phi_bc[2 * p->phi_axis] == ELBM_PHI_DIRICHLET && p->phi_bc[2 * p->phi_axis + 1] == ELBM_PHI_DIRICHLET;

    long long n_fluid = N, n_solid = 0;
    if (in->mask) {
        n_fluid = 0;
        for (long long i = 0; i < N; i++) {
            if (in->mask[i] > ELBM_NODE_OUTLET) { delete h; return ELBM_E_INVAL; }
            if (in->mask[i] == ELBM_NODE_FLUID) n_fluid++;
            if (in->mask[i] == ELBM_NODE_SOLID) n_solid++;
            if (in->mask[i] != ELBM_NODE_FLUID) g.has_mask = 1;
        }
    }
    h->has_dirichlet = n_solid > 0;
    for (int f = 0; f < 6; f++)
        if (g.phi_kind[f] == ELBM_PHI_DIRICHLET) h->has_dirichlet = 1;  // the faces that take part

    Phys &ph = h->ph;
    Cst<double> &k = ph.cd;
    k.G = p->G; k.Gw = p->Gw; k.rho0 = p->rho0; k.irho0 = 1.0 / p->rho0;
    k.kap = p->eps_kappa / p->rho0;
    k.sig_g = p->sigma_gas; k.dsig = p->sigma_liq - p->sigma_gas;
    k.itw = p->theta_width > 0.0 ? 1.0 / p->theta_width : 0.0;
    k.itau_q = 1.0 / (0.5 + p->Dq / CS2Q);
    for (int a = 0; a < 3; a++) k.E[a] = p->E_ext[a];
    k.Qb = p->Q_b; k.Qs = p->Q_s; k.iKd = 1.0 / p->K_d; k.xib = p->xi_b; k.xis = p->xi_s;
    k.omega = p->sor_omega;
    k.eq_tol = p->alpha_eq_tol;
    k.htol = p->alpha_h_tol > 0.0 ? p->alpha_h_tol : 1e-10;
    const int nax[3] = {p->nx, p->ny, p->nz};
    k.phi_lo = p->phi_lo; k.phi_hi = p->phi_hi; k.phi_solid = p->phi_solid;
    k.phi_slope = (p->phi_hi - p->phi_lo) / (nax[p->phi_axis] + 1.0);
    k.nu0 = p->nu0; k.nu_inf = p->nu_inf; k.lam = p->lambda; k.nexp = 0.5 * (p->n_carreau - 1.0);
    Cst<float> &kf = ph.cf;
    {
        const double *src = (const double *)&k;
        float *dst = (float *)&kf;
        for (size_t i = 0; i < sizeof(Cst<double>) / sizeof(double); i++) dst[i] = (float)src[i];
    }
    ph.tol = p->poisson_tol;
    ph.rho_in = p->rho_in; ph.rho_out = p->rho_out;
    ph.n_fluid = (double)n_fluid;
    ph.n_unknown = (double)(N - n_solid);
    ph.charge_model = p->charge_model; ph.force_el = p->force_el; ph.alpha_mode = p->alpha_mode;
    ph.aprec = p->precision == ELBM_PREC_FP64 ? ELBM_APREC_FP64 : p->alpha_precision;
    ph.store_macro = p->store_macro; ph.neutralize = p->neutralize;
    ph.newtonian = (p->n_carreau == 1.0 || p->lambda == 0.0 || p->nu0 == p->nu_inf) ? 1 : 0;
    ph.eps_face = p->eps_face;
    ph.carreau_lagged = p->carreau_lagged;
    // adaptive inlet (Sec. III B): the inlet nodes with their initial
    // velocities, the direction d of their sum, the profile's mean along d,
    // and the number of fluid region sites
    std::vector<int> in_idx;
    std::vector<double> in_u0;
    if (in->inlet_region) {
        if (!in->u_in || !in->mask) { delete h; return ELBM_E_INVAL; }
        double d[3] = {0, 0, 0};
        long long nreg = 0;
        for (long long i = 0; i < N; i++) {
            if (in->mask[i] == ELBM_NODE_INLET) {
                in_idx.push_back((int)i);
                for (int a = 0; a < 3; a++) {
                    in_u0.push_back(in->u_in[3 * i + a]);
                    d[a] += in->u_in[3 * i + a];
                }
            }
            if (in->inlet_region[i] && in->mask[i] == ELBM_NODE_FLUID) nreg++;
        }
        const double dn = std::sqrt(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]);
        if (in_idx.empty() || nreg == 0 || !(dn > 0.0)) { delete h; return ELBM_E_INVAL; }
        double m0 = 0.0;
        for (int a = 0; a < 3; a++) ph.in_d[a] = d[a] / dn;
        for (size_t t = 0; t < in_idx.size(); t++)
            m0 += in_u0[3 * t] * ph.in_d[0] + in_u0[3 * t + 1] * ph.in_d[1] + in_u0[3 * t + 2] * ph.in_d[2];
        m0 /= (double)in_idx.size();
        if (m0 == 0.0) { delete h; return ELBM_E_INVAL; }
        ph.adaptive = 1;
        ph.n_inlet = (int)in_idx.size();
        ph.in_m0 = m0;
        ph.n_region = (double)nreg;
    }

    Launch &L = h->L;
    int bx = p->nx >= 128 ? 128 : ((p->nx + 31) / 32) * 32;
    int by = 128 / bx;
    L.block = dim3(bx, by, 1);
    L.grid = dim3((p->nx + bx - 1) / bx, (p->ny + by - 1) / by, p->nz);
    L.nblocks = (int)(L.grid.x * L.grid.y * L.grid.z);
    if (L.grid.y > 65535 || L.grid.z > 65535) { delete h; return ELBM_E_INVAL; }
    {
        Launch &H = h->Lh;
        const int nh = g.ncol == 3 ? p->nx : (p->nx + 1) / 2;  // three colours: one thread per site
        int hx = nh >= 128 ? 128 : ((nh + 31) / 32) * 32;
        int hy = 128 / hx;
        H.block = dim3(hx, hy, 1);
        H.grid = dim3((nh + hx - 1) / hx, (p->ny + hy - 1) / hy, p->nz);
        H.nblocks = (int)(H.grid.x * H.grid.y * H.grid.z);
    }

    // multigrid hierarchy: halve while every extent is even (and stays even on
    // periodic axes) and at least 4; then, while the coarsest level has more
    // than kCoarseCells cells, halve to (n + 1)/2 cells per axis, the last
    // cell of an odd extent a single child (its span kept in last[])
    h->nlev = 0;
    if (p->charge_model != ELBM_CHARGE_NONE && p->poisson_solver == ELBM_POISSON_MG) {
        int n[3] = {p->nx, p->ny, p->nz}, last[3] = {1, 1, 1};
        auto set_level = [&](int l) {
            MGLevel &v = h->lev[l];
            v.nx = n[0]; v.ny = n[1]; v.nz = n[2];
            v.N = (long long)n[0] * n[1] * n[2];
            v.irr = 0;
            for (int a = 0; a < 3; a++) {
                v.last[a] = last[a];
                if (last[a] != (1 << l)) v.irr = 1;
            }
            v.ncol = ncolors_of(g.per, n[0], n[1], n[2]);
        };
        set_level(0);
        int L = 1;
        while (L < kMaxLevels) {
            bool ok = true;
            for (int a = 0; a < 3; a++) {
                if ((n[a] & 1) || n[a] < 4) ok = false;
                if (g.per[a] && ((n[a] / 2) & 1)) ok = false;
            }
            if (!ok) break;
            for (int a = 0; a < 3; a++) { n[a] /= 2; last[a] *= 2; }
            set_level(L);
            L++;
        }
        while (L < kMaxLevels && h->lev[L - 1].N > kCoarseCells) {
            bool ok = true;
            for (int a = 0; a < 3; a++)
                if (n[a] < 4) ok = false;
            if (!ok) break;
            const int S = 1 << (L - 1);  // span of the regular cells of level L - 1
            for (int a = 0; a < 3; a++) {
                if (!(n[a] & 1)) last[a] += S;  // the last pair: a regular cell and the last one
                n[a] = (n[a] + 1) / 2;
            }
            set_level(L);
            L++;
        }
        if (L < 2) { delete h; return ELBM_E_INVAL; }
        h->nlev = L;
        // tail: from the first level (>= 1) with at most kTailCells cells
        int lt = 1;
        while (lt < L - 1 && h->lev[lt].N > kTailCells) lt++;
        if (h->lev[lt].N > kTailCells || L - lt > kTailMaxLevels) { delete h; return ELBM_E_INVAL; }
        h->lt = lt;
        MGTail &t = h->tail;
        t.nt = L - lt;
        t.lt = lt;
        t.total = 0;
        for (int k = 0; k < t.nt; k++) {
            t.nx[k] = h->lev[lt + k].nx; t.ny[k] = h->lev[lt + k].ny; t.nz[k] = h->lev[lt + k].nz;
            t.N[k] = h->lev[lt + k].N;
            for (int a = 0; a < 3; a++) t.last[k][a] = h->lev[lt + k].last[a];
            t.irr[k] = h->lev[lt + k].irr;
            t.ncol[k] = h->lev[lt + k].ncol;
            t.off[k] = t.total;
            t.total += t.N[k];
        }
        t.coarse_sweeps = kCoarseSweeps;
        h->mg = p->precision == ELBM_PREC_FP64 ? mgops_fp64() : mgops_fp32();
        h->mg.prepare();
    }

    const bool d2 = p->velset == ELBM_VSET_D2Q9;
    switch (p->precision) {
    case ELBM_PREC_FP64: h->ops = d2 ? ops_fp64_d2q9() : ops_fp64(); h->pop_bytes = 8; h->sc_bytes = 8; h->g_bytes = 8; break;
    case ELBM_PREC_FP32: h->ops = d2 ? ops_fp32_d2q9() : ops_fp32(); h->pop_bytes = 4; h->sc_bytes = 4; h->g_bytes = 4; break;
    default: h->ops = ops_bf16(); h->pop_bytes = 2; h->sc_bytes = 4; h->g_bytes = 4; break;
    }

    Bufs &b = h->b;
    bool ok = true;
    // Device memory: the buffers are laid out twice by plan(), first to size
    // one allocation (the arena), then to hand out 256-byte aligned pieces of
    // it; the arena is zeroed once. One cudaMalloc / cudaFree per handle
    // instead of one per buffer.
    char *carve_base = nullptr;
    size_t carve_off = 0;
    auto alloc = [&](void **ptr, size_t bytes) {
        const size_t at = (carve_off + 255) & ~size_t(255);
        *ptr = carve_base ? (void *)(carve_base + at) : nullptr;
        carve_off = at + bytes;
    };
    const bool transport = p->charge_model == ELBM_CHARGE_TRANSPORT;
    const bool masks = h->nlev > 0 && n_solid > 0;  // coarse conductor masks
    long long part_blocks = p->autotune ? max_blocks_over_shapes(p) : L.nblocks;
    if (h->Lh.nblocks > part_blocks) part_blocks = h->Lh.nblocks;  // the pair-wise residual's partials
    auto plan = [&]() {
        alloc(&b.fA, (size_t)h->Q * N * h->pop_bytes);
        alloc(&b.fB, (size_t)h->Q * N * h->pop_bytes);
        if (p->precision == ELBM_PREC_BF16) {
            alloc((void **)&b.rA, (size_t)N * sizeof(float));
            alloc((void **)&b.rB, (size_t)N * sizeof(float));
        }
        if (transport) {
            alloc(&b.gA, (size_t)Q7 * N * h->g_bytes);
            alloc(&b.gB, (size_t)Q7 * N * h->g_bytes);
        }
        alloc(&b.rho, (size_t)N * h->sc_bytes);
        alloc(&b.q, (size_t)N * h->sc_bytes);
        alloc(&b.phi, (size_t)N * h->sc_bytes);
        alloc(&b.psi, (size_t)N * h->sc_bytes);
        if (transport) alloc(&b.sig, (size_t)N * h->sc_bytes);
        // extrapolated warm start in reduced precision (FP64 keeps phi(t-1), the
        // start the FP64 oracle uses, so that the two solves agree to 1e-12)
        if (p->charge_model != ELBM_CHARGE_NONE && p->poisson_fixed_sweeps == 0 && p->precision != ELBM_PREC_FP64)
            alloc(&b.phi_old, (size_t)N * h->sc_bytes);
        if (p->store_macro) {
            alloc(&b.ux, (size_t)N * h->sc_bytes);
            alloc(&b.uy, (size_t)N * h->sc_bytes);
            alloc(&b.uz, (size_t)N * h->sc_bytes);
        }
        // viscosity plane: exported, or the previous step's nu of the lagged reading
        if (p->store_macro || p->carreau_lagged) alloc(&b.nu, (size_t)N * h->sc_bytes);
        if (p->force_el == ELBM_FEL_FULL) alloc(&b.E2, (size_t)N * h->sc_bytes);
        if (p->store_macro) alloc(&b.alpha, (size_t)N * h->sc_bytes);
        // reduced precision: the low part of a root the float-float guard certified
        if (p->store_macro && p->precision != ELBM_PREC_FP64) alloc((void **)&b.alpha_lo, (size_t)N * sizeof(float));
        if (p->alpha_mode == ELBM_ALPHA_LEARNED) {
            void *img = nullptr;
            alloc(&img, sizeof(MlpSmem));
            b.mlpimg = img;
        }
        if (g.has_mask) alloc((void **)&b.mask, (size_t)N);
        if (g.has_mask || !g.per[0] || !g.per[1] || !g.per[2]) {
            void *bb = nullptr;
            alloc(&bb, (size_t)N * sizeof(unsigned));
            b.bbits = (const unsigned *)bb;
        }
        if (p->charge_model == ELBM_CHARGE_CONSERVED || p->charge_model == ELBM_CHARGE_XI) {
            alloc(&b.nh, (size_t)4 * N * h->sc_bytes);
            if (p->charge_model == ELBM_CHARGE_CONSERVED) alloc(&b.ab, (size_t)2 * N * h->sc_bytes);
        }
        for (int l = 1; l < h->nlev; l++) {
            alloc(&h->lev[l].e, (size_t)h->lev[l].N * h->sc_bytes);
            alloc(&h->lev[l].b, (size_t)h->lev[l].N * h->sc_bytes);
            alloc(&h->lev[l].eps, (size_t)h->lev[l].N * h->sc_bytes);
        }
        if (masks) {
            for (int l = 1; l < h->lt; l++) {
                void *d = nullptr;
                alloc(&d, (size_t)h->lev[l].N);
                h->lev[l].m = (const unsigned char *)d;
            }
            void *dt = nullptr;
            alloc(&dt, (size_t)h->tail.total);
            h->tail.m = (const unsigned char *)dt;
            h->lev[h->lt].m = (const unsigned char *)dt;  // the tail's first level is level lt
        }
        alloc((void **)&b.part, (size_t)part_blocks * (D_NPART + 1) * sizeof(double));
        if (ph.adaptive) {
            alloc((void **)&b.region, (size_t)N);
            alloc((void **)&b.inlet_idx, (size_t)ph.n_inlet * sizeof(int));
            alloc((void **)&b.inlet_u0, (size_t)ph.n_inlet * 3 * sizeof(double));
        }
        alloc((void **)&b.scal, S_NSCAL * sizeof(double));
        alloc((void **)&b.scalf, S_NSCAL * sizeof(float));
        alloc((void **)&b.colres, kMaxCols * sizeof(double));
        alloc((void **)&b.ticket, 4 * sizeof(unsigned int));  // the ticket; [2..3] the sticky record
        b.sticky = b.ticket + 2;
        alloc((void **)&b.diag, ELBM_NDIAG * sizeof(double));
    };
    plan();
    const size_t arena_bytes = carve_off;
    if (!cuda_ok(cudaMalloc(&h->arena, arena_bytes))) { h->arena = nullptr; ok = false; }
    ok = ok && cuda_ok(cudaMemsetAsync(h->arena, 0, arena_bytes, h->s));
    if (ok) {
        carve_base = (char *)h->arena;
        carve_off = 0;
        plan();
    }
    if (ok && p->alpha_mode == ELBM_ALPHA_LEARNED) {
        k_mlp_image<<<1, 128, 0, h->s>>>(p->mlp, (MlpSmem *)const_cast<void *>(b.mlpimg));
        ok = cuda_ok(cudaGetLastError());
    }
    // conductor masks of the coarse levels: a cell is a conductor (its
    // correction held at 0) when any of its 8 children is one
    if (masks && ok) {
        std::vector<std::vector<unsigned char>> hm(h->nlev);
        hm[0].resize(N);
        for (long long i = 0; i < N; i++) hm[0][i] = in->mask[i] == ELBM_NODE_SOLID;
        for (int l = 1; l < h->nlev; l++) {
            const MGLevel &F = h->lev[l - 1], &C = h->lev[l];
            hm[l].assign(C.N, 0);
            for (int Z = 0; Z < C.nz; Z++)
                for (int Y = 0; Y < C.ny; Y++)
                    for (int X = 0; X < C.nx; X++) {
                        unsigned char any = 0;
                        for (int c = 0; c < 8; c++) {
                            const int cx = 2 * X + (c & 1), cy = 2 * Y + ((c >> 1) & 1), cz = 2 * Z + (c >> 2);
                            if (cx < F.nx && cy < F.ny && cz < F.nz)
                                any |= hm[l - 1][cx + (long long)F.nx * (cy + (long long)F.ny * cz)];
                        }
                        hm[l][X + (long long)C.nx * (Y + (long long)C.ny * Z)] = any;
                    }
        }
        for (int l = 1; l < h->lt && ok; l++)
            ok = cuda_ok(cudaMemcpyAsync(const_cast<unsigned char *>(h->lev[l].m), hm[l].data(), (size_t)h->lev[l].N,
                                         cudaMemcpyHostToDevice, h->s));
        for (int k = 0; k < h->tail.nt && ok; k++)
            ok = cuda_ok(cudaMemcpyAsync(const_cast<unsigned char *>(h->tail.m) + h->tail.off[k],
                                         hm[h->lt + k].data(), (size_t)h->tail.N[k], cudaMemcpyHostToDevice, h->s));
        ok = ok && cuda_ok(cudaStreamSynchronize(h->s));  // hm is freed at the end of this scope
    }
    if (h->nlev > 0) h->tail.top = h->lev[h->lt];
    if (ok && !cuda_ok(cudaMallocHost((void **)&h->pin, (kPinDiag + ELBM_NDIAG) * sizeof(double)))) ok = false;
    if (ok && p->profile)
        for (int i = 0; i < 5; i++)
            if (!cuda_ok(cudaEventCreate(&h->ev[i]))) ok = false;
    if (!ok) { free_bufs(h); delete h; return ELBM_E_NOMEM; }

    // upload the initial fields into temporaries and build f(r, 0)
    double *d_rho0 = nullptr, *d_u0 = nullptr, *d_f0 = nullptr, *d_uin = nullptr, *d_q0 = nullptr;
    const size_t n_up = (in->rho0 ? N : 0) + (in->u0 ? 3 * N : 0) + (in->f0 ? (size_t)h->Q * N : 0) +
                        (in->u_in ? 3 * N : 0) + (transport && in->q0 ? N : 0);
    double *d_up = nullptr;  // one temporary for all of them
    if (ok && n_up > 0 && !cuda_ok(cudaMalloc((void **)&d_up, n_up * sizeof(double)))) { d_up = nullptr; ok = false; }
    size_t up_off = 0;
    auto up = [&](double **dst, const double *src, size_t n) {
        if (!ok || !src) return;
        *dst = d_up + up_off;
        up_off += n;
        if (!cuda_ok(cudaMemcpyAsync(*dst, src, n * sizeof(double), cudaMemcpyHostToDevice, h->s))) ok = false;
    };
    up(&d_rho0, in->rho0, N);
    up(&d_u0, in->u0, 3 * N);
    up(&d_f0, in->f0, (size_t)h->Q * N);
    up(&d_uin, in->u_in, 3 * N);
    if (transport) up(&d_q0, in->q0, N);
    if (ok && b.mask && !cuda_ok(cudaMemcpyAsync(b.mask, in->mask, N, cudaMemcpyHostToDevice, h->s))) ok = false;
    if (ok && b.bbits) {
        h->ops.bounce_bits(g, b, L, h->s);
        ok = cuda_ok(cudaGetLastError());
    }
    if (ok && ph.adaptive) {
        ok = cuda_ok(cudaMemcpyAsync(const_cast<unsigned char *>(b.region), in->inlet_region, N, cudaMemcpyHostToDevice,
                                     h->s)) &&
             cuda_ok(cudaMemcpyAsync(const_cast<int *>(b.inlet_idx), in_idx.data(), in_idx.size() * sizeof(int),
                                     cudaMemcpyHostToDevice, h->s)) &&
             cuda_ok(cudaMemcpyAsync(const_cast<double *>(b.inlet_u0), in_u0.data(), in_u0.size() * sizeof(double),
                                     cudaMemcpyHostToDevice, h->s));
    }
    if (ok) {
        h->ops.init_pop(g, ph, b, d_rho0, d_u0, d_f0, d_uin, d_q0, L, h->s);
        if (!cuda_ok(cudaGetLastError()) || !cuda_ok(cudaStreamSynchronize(h->s))) ok = false;
    }
    if (d_up) cudaFree(d_up);
    if (!ok) { free_bufs(h); delete h; return ELBM_E_CUDA; }

    if (p->autotune && !autotune(h)) { free_bufs(h); delete h; return ELBM_E_CUDA; }

    // Poisson loop control: a unit is one V-cycle, or ce SOR sweeps between tests
    h->ce = (h->nlev > 0 || p->poisson_fixed_sweeps > 0) ? 1
            : (p->poisson_check_every > 0 ? p->poisson_check_every : 8);
    h->units_max = (p->poisson_maxit + h->ce - 1) / h->ce;
    // one CUDA graph per A/B parity, captured on the first elbm_step (an
    // instance stepped only inside a batch never needs its own)
    h->use_graph = 0;
    h->want_graph = p->graph && p->diag_every == 1;
    *out = h;
    return ELBM_OK;
}

elbm_status elbm_batch_create(elbm_handle *const *inst, int n, int flags, void *stream, elbm_handle **out)
{
    if (!out) return ELBM_E_INVAL;
    *out = nullptr;
    const int span = (flags >> 8) == 0 ? 1 : (flags >> 8);
    if (!inst || n < 1 || (flags & ~(ELBM_BATCH_PIPELINE | 0xFF00)) || span > 16) return ELBM_E_INVAL;
    for (int i = 0; i < n; i++) {
        if (!inst[i] || inst[i]->n_sub > 0) return ELBM_E_INVAL;
        if (inst[i]->p.diag_every != 1 || inst[i]->p.profile) return ELBM_E_INVAL;
        for (int j = 0; j < i; j++)
            if (inst[j] == inst[i]) return ELBM_E_INVAL;
    }
    elbm_handle *B = new (std::nothrow) elbm_handle;
    if (!B) return ELBM_E_NOMEM;
    std::memset(B, 0, sizeof(*B));
    B->s = (cudaStream_t)stream;
    B->n_sub = n;
    B->pipe = (flags & ELBM_BATCH_PIPELINE) && n > 1;
    B->span = span;
    B->sub = new (std::nothrow) elbm_handle *[n];
    B->sub_step0 = new (std::nothrow) long long[n];
    B->ev_join = new (std::nothrow) cudaEvent_t[n]();
    bool ok = B->sub && B->sub_step0 && B->ev_join;
    for (int i = 0; ok && i < n; i++) {
        B->sub[i] = inst[i];
        B->sub_step0[i] = inst[i]->step;
        elbm_handle *h = inst[i];
        if (!h->cap) ok = cuda_ok(cudaStreamCreateWithFlags(&h->cap, cudaStreamNonBlocking));
        if (ok && !h->cap2) ok = cuda_ok(cudaStreamCreateWithFlags(&h->cap2, cudaStreamNonBlocking));
        ok = ok && cuda_ok(cudaEventCreateWithFlags(&B->ev_join[i], cudaEventDisableTiming));
    }
    ok = ok && cuda_ok(cudaStreamCreateWithFlags(&B->cap, cudaStreamNonBlocking));
    ok = ok && cuda_ok(cudaEventCreateWithFlags(&B->ev_fork, cudaEventDisableTiming));
    ok = ok && capture_batch(B, 0, &B->bexec[0]) && capture_batch(B, 1, &B->bexec[1]);
    if (span > 1)
        ok = ok && capture_batch(B, 0, &B->bspan[0], false, span) && capture_batch(B, 1, &B->bspan[1], false, span);
    if (ok && B->pipe) {  // the odd positions' first moments and potential solve, once
        cudaGraphExec_t pro = nullptr;
        ok = capture_batch(B, 0, &pro, true);
        ok = ok && cuda_ok(cudaGraphLaunch(pro, B->s)) && cuda_ok(cudaStreamSynchronize(B->s));
        if (pro) cudaGraphExecDestroy(pro);
    }
    if (!ok) {
        cudaGetLastError();
        elbm_free(B);
        return ELBM_E_CUDA;
    }
    *out = B;
    return ELBM_OK;
}

// The instance's step graphs, captured once; any capture failure keeps the
// host loop. The graphs are laid out for the buffers of an even step, so an
// instance already stepped an odd number of times (in a batch) is captured
// with A and B swapped back.
void ensure_graphs(elbm_handle *h)
{
    if (!h->want_graph || h->graph_tried) return;
    h->graph_tried = 1;
    bool g_ok = (h->cap || cuda_ok(cudaStreamCreateWithFlags(&h->cap, cudaStreamNonBlocking))) &&
                (h->cap2 || cuda_ok(cudaStreamCreateWithFlags(&h->cap2, cudaStreamNonBlocking)));
    const Bufs cur = h->b;
    if (h->step & 1) swap_ab(h->b);
    h->n_pre = h->n_body = h->n_post = 0;
    if (h->p.profile) {
        for (int par = 0; par < 2 && g_ok; par++)
            for (int sec = 0; sec < 3 && g_ok; sec++) g_ok = capture_step(h, par, &h->gsec[par][sec], 1 << sec);
    } else {
        g_ok = g_ok && capture_step(h, 0, &h->gexec[0]) && capture_step(h, 1, &h->gexec[1]);
    }
    h->b = cur;
    h->use_graph = g_ok ? 1 : 0;
    cudaGetLastError();
}

elbm_status elbm_step(elbm_handle *h, int nsteps)
{
    if (!h || nsteps < 0) return ELBM_E_INVAL;
    if (h->n_sub > 0) {
        for (int i = 0; i < h->n_sub; i++)
            if (h->sub[i]->step - h->sub_step0[i] != h->step) return ELBM_E_STATE;
        for (int k = 0; k < nsteps;) {
            const int m = (h->span > 1 && nsteps - k >= h->span) ? h->span : 1;  // steps in this launch
            if (!cuda_ok(cudaGraphLaunch(m > 1 ? h->bspan[h->step & 1] : h->bexec[h->step & 1], h->s)))
                return ELBM_E_CUDA;
            for (int j = 0; j < m; j++) {
                for (int i = 0; i < h->n_sub; i++) {
                    swap_ab(h->sub[i]->b);
                    h->sub[i]->step++;
                }
                h->step++;
            }
            k += m;
        }
        if (!cuda_ok(cudaStreamSynchronize(h->s))) return ELBM_E_CUDA;
        elbm_status worst = ELBM_OK;
        if (nsteps > 0) {
            for (int i = 0; i < h->n_sub; i++) {
                elbm_handle *q = h->sub[i];
                const double v[2] = {q->pin[kPinDiag + 15], q->pin[9]};  // copied by the graph's last nodes
                q->diag_mirror = 1;
                if (v[0] != 0.0) worst = ELBM_E_NUMERIC;
                if (v[1] > q->noconv_seen) {
                    q->noconv_seen = v[1];
                    if (worst == ELBM_OK) worst = ELBM_W_POISSON_NOCONV;
                }
            }
        }
        return worst;
    }
    const bool prof = h->p.profile != 0;
    if (nsteps > 0) ensure_graphs(h);
    for (int i = 0; i < nsteps; i++) {
        if (h->use_graph && prof) {
            cudaGraphExec_t *gs = h->gsec[h->step & 1];
            cudaEventRecord(h->ev[0], h->s);
            if (!cuda_ok(cudaGraphLaunch(gs[0], h->s))) return ELBM_E_CUDA;
            cudaEventRecord(h->ev[1], h->s);
            if (!cuda_ok(cudaGraphLaunch(gs[1], h->s))) return ELBM_E_CUDA;
            cudaEventRecord(h->ev[2], h->s);
            if (!cuda_ok(cudaGraphLaunch(gs[2], h->s))) return ELBM_E_CUDA;
            cudaEventRecord(h->ev[3], h->s);
            cudaEventRecord(h->ev[4], h->s);
        } else if (h->use_graph) {
            if (!cuda_ok(cudaGraphLaunch(h->gexec[h->step & 1], h->s))) return ELBM_E_CUDA;
        } else {
            bool diag = h->p.diag_every > 0 && (((h->step + 1) % h->p.diag_every) == 0 || i == nsteps - 1);
            elbm_status st = step_host(h, diag);
            if (st != ELBM_OK) return st;
        }
        if (prof) {
            if (!cuda_ok(cudaEventSynchronize(h->ev[4]))) return ELBM_E_CUDA;
            float ms[4];
            for (int k = 0; k < 4; k++) cudaEventElapsedTime(&ms[k], h->ev[k], h->ev[k + 1]);
            for (int k = 0; k < 4; k++) h->pass_ms[k] += ms[k];
            if (!cuda_ok(cudaMemcpy(h->pin, h->b.scal + S_ITER, sizeof(double), cudaMemcpyDeviceToHost)))
                return ELBM_E_CUDA;
            h->prof_steps += 1;
            h->prof_collide += 1;
            h->prof_sweeps += h->pin[0] * h->ce;
            if (h->use_graph) h->launches += h->n_pre + h->n_post + h->pin[0] * h->n_body;
        }
        swap_ab(h->b);
        h->step++;
    }
    if (!cuda_ok(cudaStreamSynchronize(h->s))) return ELBM_E_CUDA;
    if (nsteps > 0) {
        double v[2] = {0.0, 0.0};
        h->diag_mirror = h->use_graph && !prof;
        if (h->diag_mirror) {  // copied by the step graph's last nodes
            v[0] = h->pin[kPinDiag + 15];
            v[1] = h->pin[9];
            if (v[0] != 0.0) return ELBM_E_NUMERIC;
        } else {
            if (h->p.diag_every > 0 || h->use_graph) {
                if (!cuda_ok(cudaMemcpy(&v[0], h->b.diag + 15, sizeof(double), cudaMemcpyDeviceToHost)))
                    return ELBM_E_CUDA;
                if (v[0] != 0.0) return ELBM_E_NUMERIC;
            }
            if (!cuda_ok(cudaMemcpy(&v[1], h->b.scal + S_NOCONV, sizeof(double), cudaMemcpyDeviceToHost)))
                return ELBM_E_CUDA;
        }
        if (v[1] > h->noconv_seen) { h->noconv_seen = v[1]; return ELBM_W_POISSON_NOCONV; }
    }
    return ELBM_OK;
}

size_t elbm_fields_size(const elbm_handle *h, unsigned mask)
{
    if (!h) return 0;
    size_t N = (size_t)h->g.N, n = 0;
    if (mask & ELBM_F_RHO) n += N;
    if (mask & ELBM_F_U) n += 3 * N;
    if (mask & ELBM_F_PHI) n += N;
    if (mask & ELBM_F_Q) n += N;
    if (mask & ELBM_F_ALPHA) n += N;
    if (mask & ELBM_F_NU) n += N;
    if (mask & ELBM_F_POP) n += (size_t)h->Q * N;
    if (mask & ELBM_F_GPOP) n += (size_t)Q7 * N;
    if (mask & ELBM_F_DIAG) n += ELBM_NDIAG;
    return n;
}

elbm_status elbm_fields(elbm_handle *h, unsigned mask, double *out, size_t out_len)
{
    if (h && h->n_sub > 0) return ELBM_E_STATE;
    if (!h || !out) return ELBM_E_INVAL;
    if (mask & ~0x1FFu) return ELBM_E_INVAL;
    if (out_len < elbm_fields_size(h, mask)) return ELBM_E_INVAL;
    if ((mask & (ELBM_F_U | ELBM_F_ALPHA | ELBM_F_NU)) && !h->p.store_macro) return ELBM_E_STATE;
    if ((mask & ELBM_F_GPOP) && h->p.charge_model != ELBM_CHARGE_TRANSPORT) return ELBM_E_STATE;
    const long long N = h->g.N;
    size_t need = 0;
    if (mask & (ELBM_F_RHO | ELBM_F_U | ELBM_F_PHI | ELBM_F_Q | ELBM_F_ALPHA | ELBM_F_NU)) need = (size_t)N;
    if (mask & ELBM_F_POP) need = (size_t)h->Q * N;
    if (mask & ELBM_F_GPOP) need = need > (size_t)Q7 * N ? need : (size_t)Q7 * N;
    if (need > h->xtmp_n) {  // grow the export scratch (kept: repeated reads allocate nothing)
        if (h->xtmp) cudaFree(h->xtmp);
        h->xtmp = nullptr;
        h->xtmp_n = 0;
        if (!cuda_ok(cudaMalloc((void **)&h->xtmp, need * sizeof(double)))) return ELBM_E_NOMEM;
        h->xtmp_n = need;
    }
    double *tmp = need ? h->xtmp : nullptr;
    elbm_status st = ELBM_OK;
    size_t off = 0;
    auto plane = [&](const void *src, const float *lo = nullptr, bool profile = false) {
        if (st != ELBM_OK) return;
        h->ops.export_plane(src, tmp, N, h->s);
        if (lo) h->ops.add_plane(lo, tmp, N, h->s);
        if (profile && h->g.phi_lin)
            k_add_profile<<<(unsigned)((N + 255) / 256), 256, 0, h->s>>>(tmp, h->g, h->ph.cd.phi_lo, h->ph.cd.phi_slope,
                                                                        h->b.mask);
        if (!cuda_ok(cudaMemcpyAsync(out + off, tmp, N * sizeof(double), cudaMemcpyDeviceToHost, h->s)) ||
            !cuda_ok(cudaStreamSynchronize(h->s)))
            st = ELBM_E_CUDA;
        off += N;
    };
    if (mask & ELBM_F_RHO) plane(h->b.rho);
    if ((mask & ELBM_F_U) && st == ELBM_OK) {
        const void *c3[3] = {h->b.ux, h->b.uy, h->b.uz};
        double *buf = (double *)std::malloc(N * sizeof(double));
        if (!buf) st = ELBM_E_NOMEM;
        for (int a = 0; a < 3 && st == ELBM_OK; a++) {
            h->ops.export_plane(c3[a], tmp, N, h->s);
            if (!cuda_ok(cudaMemcpyAsync(buf, tmp, N * sizeof(double), cudaMemcpyDeviceToHost, h->s)) ||
                !cuda_ok(cudaStreamSynchronize(h->s))) { st = ELBM_E_CUDA; break; }
            for (long long i = 0; i < N; i++) out[off + 3 * i + a] = buf[i];
        }
        std::free(buf);
        off += 3 * N;
    }
    if (mask & ELBM_F_PHI) plane(h->b.phi, nullptr, true);
    if (mask & ELBM_F_Q) plane(h->b.q);
    if (mask & ELBM_F_ALPHA) plane(h->b.alpha, h->b.alpha_lo);
    if (mask & ELBM_F_NU) plane(h->b.nu);
    if ((mask & ELBM_F_POP) && st == ELBM_OK) {
        h->ops.export_pop(h->g, h->b, tmp, h->L, h->s);
        if (!cuda_ok(cudaMemcpyAsync(out + off, tmp, (size_t)h->Q * N * sizeof(double), cudaMemcpyDeviceToHost, h->s)) ||
            !cuda_ok(cudaStreamSynchronize(h->s)))
            st = ELBM_E_CUDA;
        off += (size_t)h->Q * N;
    }
    if ((mask & ELBM_F_GPOP) && st == ELBM_OK) {
        h->ops.export_gpop(h->g, h->b, tmp, h->L, h->s);
        if (!cuda_ok(cudaMemcpyAsync(out + off, tmp, (size_t)Q7 * N * sizeof(double), cudaMemcpyDeviceToHost, h->s)) ||
            !cuda_ok(cudaStreamSynchronize(h->s)))
            st = ELBM_E_CUDA;
        off += (size_t)Q7 * N;
    }
    if ((mask & ELBM_F_DIAG) && st == ELBM_OK) {
        if (h->diag_mirror) {  // the last step graph copied them to pinned memory
            std::memcpy(out + off, h->pin + kPinDiag, ELBM_NDIAG * sizeof(double));
        } else if (!cuda_ok(cudaMemcpyAsync(out + off, h->b.diag, ELBM_NDIAG * sizeof(double), cudaMemcpyDeviceToHost,
                                            h->s)) ||
                   !cuda_ok(cudaStreamSynchronize(h->s))) {
            st = ELBM_E_CUDA;
        }
        off += ELBM_NDIAG;
    }
    return st;
}

elbm_status elbm_pass_times(const elbm_handle *h, double *out, int n)
{
    if (h && h->n_sub > 0) return ELBM_E_STATE;
    if (!h || !out || n < 0) return ELBM_E_INVAL;
    if (!h->p.profile) return ELBM_E_STATE;
    double v[8] = {h->pass_ms[0], h->pass_ms[1], h->pass_ms[2], h->pass_ms[3], h->prof_steps,
                   h->prof_collide, h->prof_sweeps, h->launches};
    for (int i = 0; i < n && i < 8; i++) out[i] = v[i];
    return ELBM_OK;
}

void elbm_free(elbm_handle *h)
{
    if (!h) return;
    cudaStreamSynchronize(h->s);
    if (h->n_sub > 0) {  // a batch: its graphs and events only, not the instances
        for (int i = 0; i < 2; i++) {
            if (h->bexec[i]) cudaGraphExecDestroy(h->bexec[i]);
            if (h->bspan[i]) cudaGraphExecDestroy(h->bspan[i]);
        }
        if (h->ev_join)
            for (int i = 0; i < h->n_sub; i++)
                if (h->ev_join[i]) cudaEventDestroy(h->ev_join[i]);
        if (h->ev_fork) cudaEventDestroy(h->ev_fork);
        if (h->cap) cudaStreamDestroy(h->cap);
        delete[] h->sub;
        delete[] h->sub_step0;
        delete[] h->ev_join;
        delete h;
        return;
    }
    free_bufs(h);
    delete h;
}

}  // extern "C"
