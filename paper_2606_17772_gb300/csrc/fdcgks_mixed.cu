// Mixed-precision instantiation of the FD-CGKS stage kernels: FP32
// reconstruction and flux arithmetic; the state and the S2O4 accumulation as
// float-float pairs; the time coefficients of the interface solution in FP64
// (with expm1) where dt/tau <= 4, where they cancel, and in FP32 above.
#include "fdcgks_kernels.cuh"

namespace fdk {
FDK_INSTANTIATE(float)
}  // namespace fdk
