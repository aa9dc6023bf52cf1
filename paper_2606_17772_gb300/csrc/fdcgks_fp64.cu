// FP64 instantiation of the FD-CGKS stage kernels.
#include "fdcgks_kernels.cuh"

namespace fdk {
FDK_INSTANTIATE(double)
}  // namespace fdk
