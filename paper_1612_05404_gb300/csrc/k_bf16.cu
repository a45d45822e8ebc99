// Kernels of the ELBM step instantiated for ELBM_PREC_BF16 populations.
#include "elbm_kernels.cuh"

namespace elbm {
Ops ops_bf16() { return Launchers<ELBM_PREC_BF16>::table(); }
}  // namespace elbm
