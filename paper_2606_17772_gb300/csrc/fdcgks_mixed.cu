// Mixed-precision instantiation of the FD-CGKS stage kernels: FP32
// reconstruction and flux arithmetic; the state, the S2O4 accumulation and
// the collision-time coefficients stay FP64.
#include "fdcgks_kernels.cuh"

namespace fdk {
FDK_INSTANTIATE(float)
}  // namespace fdk
