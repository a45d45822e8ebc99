// elbm_noalloc.cu -- elbm_density_noalloc: the density and total mass of a
// population array, for callers that may not allocate device memory.
//
// Some callers cannot call cudaMalloc: code running while a CUDA stream is
// being captured into a graph (allocation is not a capturable operation),
// hosts that hand the whole device to their own memory pool and forbid any
// other allocation, and latency-bound loops where an allocator call (and
// the device synchronisation it may imply) is not acceptable. This entry
// point serves them: it is a variant of the moments pass (per-site sum of
// the populations with per-block partial sums of the mass) whose scratch
// memory is a fixed array in this file, not a buffer it allocates. The
// caller passes the inputs and outputs as device pointers.
#include <mutex>

#include <cuda_runtime.h>

#include "elbm.h"

namespace {

constexpr int kThreads = 256;
constexpr int kSitesPerThread = 4;
constexpr long long kSitesPerBlock = (long long)kThreads * kSitesPerThread;

// Scratch: one FP64 partial mass per block. Every GPU that loads the
// library holds these 128 KiB until the process exits.
static __device__ __align__(256) double g_noalloc_scratch[ELBM_NOALLOC_MAX_BLOCKS];

// Device address of the scratch array per device. In host code the name
// g_noalloc_scratch is only a host-side stand-in: passing it to a kernel
// would fault or silently touch the wrong memory, so the address is looked
// up with cudaGetSymbolAddress, once per device, with that device current.
// The cached address belongs to the device's primary context: it stays valid
// as long as that context does (a cudaDeviceReset ends it; do not call this
// entry point after one in the same process).
constexpr int kMaxDevices = 64;
double *g_scratch_ptr[kMaxDevices];
std::mutex g_setup_mutex;

__global__ void k_density_noalloc(const double *__restrict__ f, const unsigned char *__restrict__ mask,
                                  long long N, double *__restrict__ rho, double *__restrict__ partial)
{
    __shared__ double warp_part[kThreads / 32];
    const long long base = (long long)blockIdx.x * kSitesPerBlock;
    double m = 0.0;
#pragma unroll
    for (int k = 0; k < kSitesPerThread; k++) {
        long long s = base + (long long)k * kThreads + threadIdx.x;
        if (s >= N) break;
        double r = 0.0;
        if (!mask || mask[s] == ELBM_NODE_FLUID) {
            for (int p = 0; p < 19; p++) r += f[(long long)p * N + s];
            m += r;
        }
        rho[s] = r;
    }
    for (int o = 16; o > 0; o >>= 1) m += __shfl_down_sync(0xffffffffu, m, o);
    if ((threadIdx.x & 31) == 0) warp_part[threadIdx.x >> 5] = m;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int i = 0; i < kThreads / 32; i++) t += warp_part[i];
        partial[blockIdx.x] = t;  // every slot a later pass reads is written here first
    }
}

// Sum the per-block partials in a fixed order (one block): reproducible.
__global__ void k_mass_noalloc(const double *__restrict__ partial, int nblocks, double *__restrict__ mass)
{
    __shared__ double sh[kThreads];
    double acc = 0.0;
    for (int i = threadIdx.x; i < nblocks; i += kThreads) acc += partial[i];
    sh[threadIdx.x] = acc;
    __syncthreads();
    for (int w = kThreads / 2; w > 0; w >>= 1) {
        if (threadIdx.x < w) sh[threadIdx.x] += sh[threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0) *mass = sh[0];
}

}  // namespace

extern "C" elbm_status elbm_density_noalloc(const double *f, const unsigned char *mask, long long n_sites,
                                            double *rho, double *mass, void *stream)
{
    if (!f || !rho || !mass || n_sites <= 0) return ELBM_E_INVAL;
    if (n_sites > ELBM_NOALLOC_MAX_SITES) return ELBM_E_INVAL;  // beyond the fixed scratch
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return ELBM_E_CUDA;
    double *scratch = nullptr;
    {
        std::lock_guard<std::mutex> lock(g_setup_mutex);
        if (!g_scratch_ptr[dev]) {
            void *p = nullptr;
            if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || !p) return ELBM_E_CUDA;
            g_scratch_ptr[dev] = (double *)p;
        }
        scratch = g_scratch_ptr[dev];
    }
    const int nblocks = (int)((n_sites + kSitesPerBlock - 1) / kSitesPerBlock);
    cudaStream_t s = (cudaStream_t)stream;
    // an error left pending by earlier, unrelated work on this thread is not
    // this call's failure: clear it so the check below sees only these launches
    (void)cudaGetLastError();
    k_density_noalloc<<<nblocks, kThreads, 0, s>>>(f, mask, n_sites, rho, scratch);
    k_mass_noalloc<<<1, kThreads, 0, s>>>(scratch, nblocks, mass);
    return cudaGetLastError() == cudaSuccess ? ELBM_OK : ELBM_E_CUDA;
}
