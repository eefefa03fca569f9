// Step kernels instantiated for population storage float, compute type float.
#include "step_kernels.cuh"

namespace lbeh {
PrecOps ops_f32() { return Launch<float, float>::ops(); }
}  // namespace lbeh
