// Step kernels instantiated for population storage double, compute type double.
#include "step_kernels.cuh"

namespace lbeh {
PrecOps ops_f64() { return Launch<double, double>::ops(); }
}  // namespace lbeh
