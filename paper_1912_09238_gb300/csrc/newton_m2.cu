// newton_m2.cu -- instantiation of the Newton kernel for mode 2: mixed with an FP32 factorisation.
#include "newton_kernel.cuh"

namespace ipm {
template cudaError_t newton_mode_call<2>(int, int, int, const NewtonArgs*, int, size_t, bool, cudaStream_t, int, int*);
}  // namespace ipm
