// Batched coupled step: many independent systems of uneven size advanced by
// one persistent launch.  One thread-block cluster owns one system and runs
// the whole timestep on it (Sec. II: macroscopic fields, Poisson solve,
// forces + ion fluxes + collision + streaming, Nernst-Planck update) for all
// requested steps, separated by hardware cluster barriers; clusters never
// wait on each other.  The per-site arithmetic is that of the single-system
// kernels (macro_site, collide_site, np_site, poisson_body), so a system's
// result depends only on its own data and the cluster size: the batched
// launch and one launch per system agree bit for bit.
//
// Included once per precision mode (batch_f64.cu, batch_f32.cu).  Systems in a
// batch carry no colloids.
#pragma once

#include "poisson_dev.cuh"
#include "step_kernels.cuh"

namespace lbeh {

// Device record of one system (read-only during the launch).
template <typename S, typename T> struct BatchRec {
  StepK<T> k;
  S *f[2];
  T *rho, *J, *psi, *eps, *q, *u, *flux;
  T *n[2];
  const T *phi;  // potential in the compute type (high words in the FP32 modes)
  int pois;      // the system has a potential to solve
  PArgs<T> pa;
};

template <typename S, typename T, int NC, bool IONS, bool DFM>
__global__ void __launch_bounds__(kPB, 2)
    k_batch(const BatchRec<S, T> *__restrict__ recs, int *__restrict__ par, int rec0, int nsteps) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ double sh[kPB];
  __shared__ T sht[kPB];
  const ClusterTeam tm;
  unsigned cid;
  asm volatile("mov.u32 %0, %%clusterid.x;" : "=r"(cid));
  const int b = rec0 + int(cid);
  const BatchRec<S, T> &B = recs[b];
  const StepK<T> &k = B.k;
  const long long N = k.d.N;
  const long long r0 = tm.rank(), G = tm.size();
  int cur = par[2 * b], ncur = par[2 * b + 1];
  for (int t = 0; t < nsteps; ++t) {
    const S *f = B.f[cur];
    S *fn = B.f[cur ^ 1];
    const T *n = IONS ? B.n[ncur] : nullptr;
    T *nn = IONS ? B.n[ncur ^ 1] : nullptr;
    for (long long i = r0; i < N; i += G)
      macro_site<S, T, NC, false>(k, f, B.rho, B.J, B.psi, B.eps, B.q, n, nullptr, nullptr, nullptr, i);
    tm.sync();
    if (B.pois) {
      poisson_body<T, DFM>(B.pa, tm, smem_raw, sh, sht);
      tm.sync();
    }
    for (long long i = r0; i < N; i += G)
      collide_site<S, T, NC, false, IONS, false>(k, f, fn, B.rho, B.J, B.psi, B.eps, B.phi, n, nullptr, nullptr,
                                                 nullptr, nullptr, B.u, B.flux, int(i));
    tm.sync();
    if (IONS) {
      for (long long i = r0; i < N; i += G) np_site<T, false>(k, n, nn, B.flux, B.u, nullptr, i);
      tm.sync();
      ncur ^= 1;
    }
    cur ^= 1;
  }
  if (r0 == 0) {
    par[2 * b] = cur;
    par[2 * b + 1] = ncur;
  }
}

template <typename S, typename T, bool DFM> struct BatchImpl {
  using Rec = BatchRec<S, T>;
  static long long fill(const BatchBox &bx, void *out) {
    const Ctx &c = *bx.c;
    Rec r{};
    r.k = make_stepk<T>(c);
    r.f[0] = (S *)c.f[0];
    r.f[1] = (S *)c.f[1];
    r.rho = (T *)c.rho;
    r.J = (T *)c.J;
    r.psi = (T *)c.psi;
    r.eps = (T *)c.eps;
    r.q = (T *)c.q;
    r.u = (T *)c.u;
    r.flux = (T *)c.flux;
    r.n[0] = (T *)c.n[0];
    r.n[1] = (T *)c.n[1];
    r.phi = (const T *)c.phit;
    long long smem = 0;
    if (bx.pois) {
      r.pois = 1;
      smem = poisson_team_args(bx.pois, c, &r.pa, sizeof(r.pa));
      if (smem < 0) return -1;
    }
    std::memcpy(out, &r, sizeof(r));
    return smem;
  }
  static const void *kernel(int ncomp, int nions) {
    if (ncomp == 2)
      return nions ? (const void *)k_batch<S, T, 2, true, DFM> : (const void *)k_batch<S, T, 2, false, DFM>;
    return nions ? (const void *)k_batch<S, T, 1, true, DFM> : (const void *)k_batch<S, T, 1, false, DFM>;
  }
  static BatchKernels get() {
    BatchKernels b;
    b.rec_bytes = sizeof(Rec);
    b.fill = fill;
    b.kernel = kernel;
    return b;
  }
};

}  // namespace lbeh
