// Adjoint passes instantiated for FP64.
#include "adjoint_kernels.cuh"

namespace lbeh {
AdjOps adj_ops_f64() { return AdjLaunch<double>::ops(); }
}  // namespace lbeh
