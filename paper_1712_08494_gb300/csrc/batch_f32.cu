// Batched step instantiated for FP32 populations and arithmetic (double-float
// potential).
#include <cstring>

#include "batch_impl.cuh"

namespace lbeh {
BatchKernels batch_kernels_f32() { return BatchImpl<float, float, true>::get(); }
}  // namespace lbeh
