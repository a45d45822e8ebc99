// Kernels of the ELBM step instantiated for ELBM_PREC_FP64 populations.
#include "elbm_kernels.cuh"

namespace elbm {
Ops ops_fp64() { return Launchers<ELBM_PREC_FP64>::table(); }
MGOps mgops_fp64() { return MGLaunchers<ELBM_PREC_FP64>::table(); }
}  // namespace elbm
