// newton_m4.cu -- instantiation of the Newton kernel for mode 4: FP64 Hessian with the split factorisation.
#include "newton_kernel.cuh"

namespace ipm {
template cudaError_t newton_mode_call<4>(int, int, int, const NewtonArgs*, int, size_t, bool, cudaStream_t, int, int*);
}  // namespace ipm
