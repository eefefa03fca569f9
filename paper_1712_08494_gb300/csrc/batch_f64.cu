// Batched step instantiated for FP64 populations and arithmetic.
#include <cstring>

#include "batch_impl.cuh"

namespace lbeh {
BatchKernels batch_kernels_f64() { return BatchImpl<double, double, false>::get(); }
}  // namespace lbeh
