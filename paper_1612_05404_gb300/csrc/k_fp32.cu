// Kernels of the ELBM step instantiated for ELBM_PREC_FP32 populations.
#include "elbm_kernels.cuh"

namespace elbm {
Ops ops_fp32() { return Launchers<ELBM_PREC_FP32>::table(); }
MGOps mgops_fp32() { return MGLaunchers<ELBM_PREC_FP32>::table(); }
}  // namespace elbm
