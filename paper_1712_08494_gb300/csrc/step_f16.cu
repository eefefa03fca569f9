// Step kernels instantiated for population storage __half, compute type float.
#include "step_kernels.cuh"

namespace lbeh {
PrecOps ops_f16() { return Launch<__half, float>::ops(); }
}  // namespace lbeh
