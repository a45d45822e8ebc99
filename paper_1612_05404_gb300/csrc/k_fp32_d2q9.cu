// Kernels of the ELBM step for the paper's D2Q9 set (Sec. II) instantiated for
// ELBM_PREC_FP32 populations.
#define ELBM_D2Q9 1
#include "elbm_kernels.cuh"

namespace elbm {
Ops ops_fp32_d2q9() { return Launchers<ELBM_PREC_FP32>::table(); }
}  // namespace elbm
