// Kernels of the ELBM step for the paper's D2Q9 set (Sec. II) instantiated for
// ELBM_PREC_FP64 populations, and the set's public population order.
#define ELBM_D2Q9 1
#include "elbm_kernels.cuh"

namespace elbm {
Ops ops_fp64_d2q9() { return Launchers<ELBM_PREC_FP64>::table(); }

int vset_d2q9(int *c, double *w)
{
    for (int p = 0; p < Q; p++) {
        if (c) { c[3 * p] = cx(p); c[3 * p + 1] = cy(p); c[3 * p + 2] = cz(p); }
        if (w) w[p] = wq(p);
    }
    return Q;
}
}  // namespace elbm
