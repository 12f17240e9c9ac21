// newton_m0.cu -- instantiation of the Newton kernel for mode 0: FP64 (every step in float64).
#include "newton_kernel.cuh"

namespace ipm {
template cudaError_t newton_mode_call<0>(int, int, int, const NewtonArgs*, int, size_t, bool, cudaStream_t, int, int*);
}  // namespace ipm
