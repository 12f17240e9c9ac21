// newton_m3.cu -- instantiation of the Newton kernel for mode 3: mixed with the split factorisation (tensor-core trailing updates).
#include "newton_kernel.cuh"

namespace ipm {
template cudaError_t newton_mode_call<3>(int, int, int, const NewtonArgs*, int, size_t, bool, cudaStream_t, int, int*);
}  // namespace ipm
