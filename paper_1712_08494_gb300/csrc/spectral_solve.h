// Host interface of the spectral Poisson solve (spectral.cu) used by the
// solver front end (poisson.cu).
#pragma once

#include "internal.h"

namespace lbeh {

template <typename T> struct PArgs;
struct Spectral;

// Every axis factors into 2, 3, 5, 7 and is at most 512 long (256 in FP64).
bool spectral_supported(const Dims &d, int fp64);
// Work arrays, transform tables and launch shape of the solve of one box;
// eps_ref is the reference permittivity of the preconditioner.  Null when
// unsupported or out of memory.
Spectral *spectral_create(const Ctx &c, int fp64, double eps_ref);
void spectral_destroy(Spectral *s);
// One cooperative launch: the whole solve for c.phi from c.eps and c.q with the
// solver state, partials and barrier of pa.  Returns 0 or -1.
int spectral_launch_f64(Spectral *s, const Ctx &c, const PArgs<double> &pa, cudaStream_t st);
int spectral_launch_f32(Spectral *s, const Ctx &c, const PArgs<float> &pa, cudaStream_t st);
int spectral_grid(const Spectral *s);  // blocks of the launch

}  // namespace lbeh
