// Step kernels instantiated for population storage __nv_bfloat16, compute type float.
#include "step_kernels.cuh"

namespace lbeh {
PrecOps ops_bf16() { return Launch<__nv_bfloat16, float>::ops(); }
}  // namespace lbeh
