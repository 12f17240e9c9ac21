// newton_m1.cu -- instantiation of the Newton kernel for mode 1: mixed (tensor-core Hessian, FP64 blocked factorisation).
#include "newton_kernel.cuh"

namespace ipm {
template cudaError_t newton_mode_call<1>(int, int, int, const NewtonArgs*, int, size_t, bool, cudaStream_t, int, int*);
}  // namespace ipm
