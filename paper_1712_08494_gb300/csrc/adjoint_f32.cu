// Adjoint passes instantiated for FP32.
#include "adjoint_kernels.cuh"

namespace lbeh {
AdjOps adj_ops_f32() { return AdjLaunch<float>::ops(); }
}  // namespace lbeh
