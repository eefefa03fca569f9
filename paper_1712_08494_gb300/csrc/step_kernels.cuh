// Kernels of the coupled lattice timestep, templated on the population
// storage type S and the compute type T.  Included once per precision mode.
//
// Per step (Sec. II):
//   k_macro    rho^sigma, psi^sigma = 1 - exp(-rho), eps(c, psi_s), q       (II.B, II.C, II.E)
//   k_virtual  mean fluid density on interface solid nodes (Jansen)        (II.E)
//   [Poisson]  phi from eps, q and the applied field                         (II.B, II.D)
//   k_collide  E = -grad phi + E_ext, ion face fluxes, Shan-Chen fluid-fluid
//              and fluid-ion forces, friction, Kelvin force, physical
//              velocity, forced BGK collision (velocity shift), push
//              streaming with halfway bounce-back and moving-wall term      (II.A-II.E)
//   k_np       finite-volume Nernst-Planck update, upwind advection        (II.B)
#pragma once

#include "internal.h"
#include "dfloat.cuh"

namespace lbeh {

template <typename T> __device__ __forceinline__ T expm1_t(T v);
template <> __device__ __forceinline__ double expm1_t<double>(double v) { return expm1(v); }
template <> __device__ __forceinline__ float expm1_t<float>(float v) { return expm1f(v); }

template <typename T> struct StepK {
  Dims d;
  int ncomp, nions;
  bool solids, has_field, solvation;
  T tau, inv_tau, G, D, inv_2D;
  T gas[2], dmd[2];
  T eps_a, eps_b, eps_p, eps_bar;
  T Eext[3];
  T shift[2];
};

template <typename T> StepK<T> make_stepk(const Ctx &c) {
  StepK<T> k;
  k.d = c.d;
  k.ncomp = c.ncomp;
  k.nions = c.nions;
  k.solids = c.solids;
  k.has_field = c.has_field;
  k.solvation = c.solvation;
  k.tau = T(c.tau);
  k.inv_tau = T(1.0 / c.tau);
  k.G = T(c.G);
  k.D = T(c.D);
  k.inv_2D = c.D > 0 ? T(1.0 / (2.0 * c.D)) : T(0);
  for (int s = 0; s < 2; ++s) {
    k.gas[s] = T(c.gas[s]);
    k.dmd[s] = T(c.dmd[s]);
    k.shift[s] = T(c.shift[s]);
  }
  k.eps_a = T(c.eps_a);
  k.eps_b = T(c.eps_b);
  k.eps_p = T(c.eps_p);
  k.eps_bar = T(c.eps_bar);
  for (int a = 0; a < 3; ++a) k.Eext[a] = T(c.Eext[a]);
  return k;
}

// eps = psi_s eps_p + (1 - psi_s) eps_f(c),  eps_f = [eps_a(1-c) + eps_b(1+c)]/2
template <typename T>
__device__ __forceinline__ T permittivity(const StepK<T> &k, T ra, T rb, T ps) {
  T tot = ra + rb;
  T c = tot > T(0) ? (rb - ra) / tot : T(0);
  T ef = T(0.5) * (k.eps_a * (T(1) - c) + k.eps_b * (T(1) + c));
  return ps * k.eps_p + (T(1) - ps) * ef;
}

// ---------------------------------------------------------------- k_macro
// RO: the populations are read-only for the whole launch (separate kernels),
// so they may go through the non-coherent read path; a kernel that also
// writes them in an earlier phase passes false.
template <bool RO, typename S, typename T>
__device__ __forceinline__ T sload(const S *p, size_t i, T shift) {
  if constexpr (RO) return Store<S, T>::ld(p, i, shift);
  else return Store<S, T>::ldc(p, i, shift);
}

template <typename S, typename T, int NC, bool RO>
__device__ __forceinline__ void macro_site(const StepK<T> &k, const S *__restrict__ f, T *__restrict__ rho,
                                           T *__restrict__ Jout, T *__restrict__ psi, T *__restrict__ eps,
                                           T *__restrict__ q, const T *__restrict__ n, const T *__restrict__ qc,
                                           const T *__restrict__ psi_s, const uint8_t *__restrict__ solid,
                                           const long long i) {
  const long long N = k.d.N;
  T r[2] = {T(0), T(0)};
  T J[3] = {T(0), T(0), T(0)};
  const bool sol = k.solids && solid[i];
  if (!sol) {
    T fl[NC][19];
#pragma unroll
    for (int s = 0; s < NC; ++s) {
      T acc = T(0);
#pragma unroll
      for (int qd = 0; qd < 19; ++qd) {
        fl[s][qd] = sload<RO, S, T>(f, (size_t)(s * 19 + qd) * N + i, wq<T>(qd) * k.shift[s]);
        acc += fl[s][qd];
      }
      r[s] = acc;
    }
    // momentum sum_sigma sum_q f c_q (equal relaxation times: one barycentric velocity)
#pragma unroll
    for (int qd = 1; qd < 19; ++qd) {
      T v = fl[0][qd];
      if (NC == 2) v += fl[1][qd];
      if (cx(qd)) J[0] += T(cx(qd)) * v;
      if (cy(qd)) J[1] += T(cy(qd)) * v;
      if (cz(qd)) J[2] += T(cz(qd)) * v;
    }
  }
  Jout[i] = J[0];
  Jout[N + i] = J[1];
  Jout[2 * N + i] = J[2];
#pragma unroll
  for (int s = 0; s < NC; ++s) {
    rho[s * N + i] = r[s];
    psi[s * N + i] = -expm1_t<T>(-r[s]);
  }
  T ps = k.solids ? psi_s[i] : T(0);
  eps[i] = permittivity(k, r[0], NC == 2 ? r[1] : T(0), ps);
  T qq = k.solids ? qc[i] : T(0);
  if (k.nions) qq += n[i] - n[N + i];
  q[i] = qq;
}

template <typename S, typename T, int NC>
__global__ void __launch_bounds__(256) k_macro(StepK<T> k, const S *__restrict__ f, T *__restrict__ rho,
                                               T *__restrict__ Jout, T *__restrict__ psi, T *__restrict__ eps,
                                               T *__restrict__ q, const T *__restrict__ n,
                                               const T *__restrict__ qc, const T *__restrict__ psi_s,
                                               const uint8_t *__restrict__ solid) {
  const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (i >= k.d.N) return;
  macro_site<S, T, NC, true>(k, f, rho, Jout, psi, eps, q, n, qc, psi_s, solid, i);
}

// ---------------------------------------------------------------- k_virtual
// One block per colloid walks the colloid's bounding box; surface nodes get
// the mean density of their fluid D3Q19 neighbours, and their psi and eps.
template <typename T, int NC>
__global__ void k_virtual(StepK<T> k, T *__restrict__ rho, T *__restrict__ psi, T *__restrict__ eps,
                          const T *__restrict__ psi_s, const uint8_t *__restrict__ solid,
                          const uint8_t *__restrict__ surface, const int *__restrict__ owner,
                          const double *__restrict__ cx, const double *__restrict__ cr) {
  const int j = blockIdx.x;
  const Dims d = k.d;
  const long long N = d.N;
  int lo[3], cnt[3];
  const int dims[3] = {d.nx, d.ny, d.nz};
  for (int a = 0; a < 3; ++a) {
    double X = cx[3 * j + a], r = cr[j];
    lo[a] = int(ceil(X - r - 2.0));
    int hi = int(floor(X + r + 2.0));
    cnt[a] = min(dims[a], hi - lo[a] + 1);
  }
  const long long tot = (long long)cnt[0] * cnt[1] * cnt[2];
  for (long long t = threadIdx.x; t < tot; t += blockDim.x) {
    int ox = int(t % cnt[0]);
    int oy = int((t / cnt[0]) % cnt[1]);
    int oz = int(t / ((long long)cnt[0] * cnt[1]));
    int x = ((lo[0] + ox) % d.nx + d.nx) % d.nx;
    int y = ((lo[1] + oy) % d.ny + d.ny) % d.ny;
    int z = ((lo[2] + oz) % d.nz + d.nz) % d.nz;
    long long i = site(d, x, y, z);
    if (!surface[i] || owner[i] != j) continue;
    long long nb[19];
    neighbours19(d, x, y, z, nb);
    T acc[2] = {T(0), T(0)};
    int c = 0;
#pragma unroll
    for (int qd = 1; qd < 19; ++qd) {
      if (!solid[nb[qd]]) {
        ++c;
#pragma unroll
        for (int s = 0; s < NC; ++s) acc[s] += rho[s * N + nb[qd]];
      }
    }
    T rv[2] = {T(0), T(0)};
#pragma unroll
    for (int s = 0; s < NC; ++s) {
      rv[s] = c > 0 ? acc[s] / T(c) : T(0);
      rho[s * N + i] = rv[s];
      psi[s * N + i] = -expm1_t<T>(-rv[s]);
    }
    eps[i] = permittivity(k, rv[0], NC == 2 ? rv[1] : T(0), psi_s[i]);
  }
}

// ---------------------------------------------------------------- k_collide
// Forces and ion fluxes are formed first from the macro fields written by
// k_macro (no population is live), then each component's populations are
// loaded, relaxed and pushed.  Keeping the populations out of the force
// phase holds the register footprint low enough for several resident blocks
// per SM.  Site indices are 32-bit (boxes below 2^31 sites).
template <typename S, typename T, int NC, bool SOL, bool IONS, bool RO>
__device__ __forceinline__ void collide_site(const StepK<T> &k, const S *__restrict__ f, S *__restrict__ fn,
                                             const T *__restrict__ rhoF, const T *__restrict__ JF,
                                             const T *__restrict__ psiF, const T *__restrict__ eps,
                                             const T *__restrict__ phi, const T *__restrict__ n,
                                             const T *__restrict__ psi_f, const uint8_t *__restrict__ solid,
                                             const int *__restrict__ owner, const double *__restrict__ cv,
                                             T *__restrict__ u_out, T *__restrict__ flux_out, const int i) {
  const int nx = k.d.nx, ny = k.d.ny, nz = k.d.nz;
  const int N = int(k.d.N);
  if (SOL && solid[i]) {
    // a node covered by a moving colloid must not keep the face fluxes and
    // velocity of the step in which it was fluid
#pragma unroll
    for (int a = 0; a < 3; ++a) u_out[a * N + i] = T(0);
    if (IONS)
#pragma unroll
      for (int m = 0; m < 6; ++m) flux_out[m * N + i] = T(0);
    return;
  }
  const int r = i / nx;
  const int x = i - r * nx;
  const int z = r / ny;
  const int y = r - z * ny;
  const int nxy = nx * ny;
  // periodic neighbour offsets along each axis
  const int oxm = (x == 0 ? nx - 1 : -1), oxp = (x + 1 == nx ? 1 - nx : 1);
  const int oym = (y == 0 ? (ny - 1) * nx : -nx), oyp = (y + 1 == ny ? (1 - ny) * nx : nx);
  const int ozm = (z == 0 ? (nz - 1) * nxy : -nxy), ozp = (z + 1 == nz ? (1 - nz) * nxy : nxy);
  auto NB = [&](int q) -> int {
    return i + (cx(q) < 0 ? oxm : (cx(q) > 0 ? oxp : 0)) + (cy(q) < 0 ? oym : (cy(q) > 0 ? oyp : 0)) +
           (cz(q) < 0 ? ozm : (cz(q) > 0 ? ozp : 0));
  };

  // L2 prefetch of the site's populations (read-only launches): their DRAM
  // fetch overlaps the force computation below (+9% on the collide pass)
  if (RO) {
#pragma unroll
    for (int s = 0; s < NC; ++s)
#pragma unroll
      for (int qd = 0; qd < 19; ++qd)
        asm volatile("prefetch.global.L2 [%0];" ::"l"(f + (size_t)(s * 19 + qd) * N + i));
  }
  T rho[2];
  rho[0] = rhoF[i];
  rho[1] = NC == 2 ? rhoF[N + i] : T(0);
  const T J[3] = {JF[i], JF[N + i], JF[2 * N + i]};
  const T rho_tot = rho[0] + (NC == 2 ? rho[1] : T(0));
  const T inv_rho = rho_tot > T(0) ? T(1) / rho_tot : T(0);

  T Phi[2][3] = {{T(0), T(0), T(0)}, {T(0), T(0), T(0)}};

  // Shan-Chen fluid-fluid force (Sec. II.C eq. shanChenForce)
  if (NC == 2 && k.G != T(0)) {
    T Sa[3] = {T(0), T(0), T(0)}, Sb[3] = {T(0), T(0), T(0)};
#pragma unroll
    for (int qd = 1; qd < 19; ++qd) {
      const int j = NB(qd);
      const T pa = wq<T>(qd) * psiF[j];
      const T pb = wq<T>(qd) * psiF[N + j];
      if (cx(qd)) { Sa[0] += T(cx(qd)) * pb; Sb[0] += T(cx(qd)) * pa; }
      if (cy(qd)) { Sa[1] += T(cy(qd)) * pb; Sb[1] += T(cy(qd)) * pa; }
      if (cz(qd)) { Sa[2] += T(cz(qd)) * pb; Sb[2] += T(cz(qd)) * pa; }
    }
    const T ga = -k.G * psiF[i], gb = -k.G * psiF[N + i];
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      Phi[0][a] += ga * Sa[a];
      Phi[1][a] += gb * Sb[a];
    }
  }
  // Shan-Chen fluid-ion (solvation) force on component a (Sec. II.C eq. solvation:force1)
  if (IONS && k.solvation) {
    T Si[3] = {T(0), T(0), T(0)};
#pragma unroll
    for (int s = 0; s < 2; ++s) {
      if (k.gas[s] == T(0)) continue;
      T acc[3] = {T(0), T(0), T(0)};
#pragma unroll
      for (int qd = 1; qd < 19; ++qd) {
        const T v = wq<T>(qd) * n[s * N + NB(qd)];
        if (cx(qd)) acc[0] += T(cx(qd)) * v;
        if (cy(qd)) acc[1] += T(cy(qd)) * v;
        if (cz(qd)) acc[2] += T(cz(qd)) * v;
      }
#pragma unroll
      for (int a = 0; a < 3; ++a) Si[a] += k.gas[s] * acc[a];
    }
    const T pa = psiF[i];
#pragma unroll
    for (int a = 0; a < 3; ++a) Phi[0][a] += -pa * Si[a];
  }

  T Fel[3] = {T(0), T(0), T(0)};
  // axis neighbours in the order +x -x +y -y +z -z
  const int ax[6] = {i + oxp, i + oxm, i + oyp, i + oym, i + ozp, i + ozm};
  if (k.has_field) {
    // E = -grad phi + E_ext at i and at its six axis neighbours
    const T p0 = phi[i];
    T Ei[3];
    Ei[0] = T(-0.5) * (phi[ax[0]] - phi[ax[1]]) + k.Eext[0];
    Ei[1] = T(-0.5) * (phi[ax[2]] - phi[ax[3]]) + k.Eext[1];
    Ei[2] = T(-0.5) * (phi[ax[4]] - phi[ax[5]]) + k.Eext[2];
    // Enb[dir][comp]: along-axis components use the distance-2 points, the
    // transverse ones the face diagonals
    const int x2p = x + 2 >= nx ? x + 2 - nx : x + 2, x2m = x - 2 < 0 ? x - 2 + nx : x - 2;
    const int y2p = y + 2 >= ny ? y + 2 - ny : y + 2, y2m = y - 2 < 0 ? y - 2 + ny : y - 2;
    const int z2p = z + 2 >= nz ? z + 2 - nz : z + 2, z2m = z - 2 < 0 ? z - 2 + nz : z - 2;
    T Enb[6][3];
    Enb[0][0] = T(-0.5) * (phi[i - x + x2p] - p0) + k.Eext[0];
    Enb[1][0] = T(-0.5) * (p0 - phi[i - x + x2m]) + k.Eext[0];
    Enb[2][1] = T(-0.5) * (phi[i + (y2p - y) * nx] - p0) + k.Eext[1];
    Enb[3][1] = T(-0.5) * (p0 - phi[i + (y2m - y) * nx]) + k.Eext[1];
    Enb[4][2] = T(-0.5) * (phi[i + (z2p - z) * nxy] - p0) + k.Eext[2];
    Enb[5][2] = T(-0.5) * (p0 - phi[i + (z2m - z) * nxy]) + k.Eext[2];
    Enb[0][1] = T(-0.5) * (phi[NB(7)] - phi[NB(9)]) + k.Eext[1];
    Enb[0][2] = T(-0.5) * (phi[NB(11)] - phi[NB(13)]) + k.Eext[2];
    Enb[1][1] = T(-0.5) * (phi[NB(10)] - phi[NB(8)]) + k.Eext[1];
    Enb[1][2] = T(-0.5) * (phi[NB(14)] - phi[NB(12)]) + k.Eext[2];
    Enb[2][0] = T(-0.5) * (phi[NB(7)] - phi[NB(10)]) + k.Eext[0];
    Enb[2][2] = T(-0.5) * (phi[NB(15)] - phi[NB(17)]) + k.Eext[2];
    Enb[3][0] = T(-0.5) * (phi[NB(9)] - phi[NB(8)]) + k.Eext[0];
    Enb[3][2] = T(-0.5) * (phi[NB(18)] - phi[NB(16)]) + k.Eext[2];
    Enb[4][0] = T(-0.5) * (phi[NB(11)] - phi[NB(14)]) + k.Eext[0];
    Enb[4][1] = T(-0.5) * (phi[NB(15)] - phi[NB(18)]) + k.Eext[1];
    Enb[5][0] = T(-0.5) * (phi[NB(13)] - phi[NB(12)]) + k.Eext[0];
    Enb[5][1] = T(-0.5) * (phi[NB(17)] - phi[NB(16)]) + k.Eext[1];

    // Kelvin force +(eps - eps_bar)/4 sum_{Q6} |E(i+d)|^2 c_d (Sec. II.C, discrete total force)
    const T de = T(0.25) * (eps[i] - k.eps_bar);
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      const T e2p = Enb[2 * a][0] * Enb[2 * a][0] + Enb[2 * a][1] * Enb[2 * a][1] + Enb[2 * a][2] * Enb[2 * a][2];
      const T e2m = Enb[2 * a + 1][0] * Enb[2 * a + 1][0] + Enb[2 * a + 1][1] * Enb[2 * a + 1][1] +
                    Enb[2 * a + 1][2] * Enb[2 * a + 1][2];
      Fel[a] = de * (e2p - e2m);
    }
    if (IONS) {
      // face fluxes (Sec. II.B eq. ionic-fluxes-disc, Sec. II.E eq. ionic-fluxes-disc-2)
      const T pf_i = SOL ? psi_f[i] : T(1);
      T nt_i[2];
#pragma unroll
      for (int s = 0; s < 2; ++s) nt_i[s] = pf_i > T(0) ? n[s * N + i] / pf_i : T(0);
      const T ra_i = rho[0];
#pragma unroll
      for (int a = 0; a < 3; ++a) {
        const int jp = ax[2 * a], jm = ax[2 * a + 1];
        const T pf_p = SOL ? psi_f[jp] : T(1);
        const T pf_m = SOL ? psi_f[jm] : T(1);
        const T Ep = T(0.5) * (Ei[a] + Enb[2 * a][a]);
        const T Em = T(0.5) * (Enb[2 * a + 1][a] + Ei[a]);
        const T dr_p = rhoF[jp] - ra_i;
        const T dr_m = ra_i - rhoF[jm];
        const T wp = k.D * pf_i * pf_p;
        const T wm = k.D * pf_m * pf_i;
        T tot = T(0);
#pragma unroll
        for (int s = 0; s < 2; ++s) {
          const T zs = s == 0 ? T(1) : T(-1);
          const T ntp = pf_p > T(0) ? n[s * N + jp] / pf_p : T(0);
          const T ntm = pf_m > T(0) ? n[s * N + jm] / pf_m : T(0);
          const T nbp = T(0.5) * (nt_i[s] + ntp);
          const T nbm = T(0.5) * (ntm + nt_i[s]);
          const T Fp = wp * ((ntp - nt_i[s]) - zs * nbp * Ep - k.dmd[s] * nbp * dr_p);
          const T Fm = wm * ((nt_i[s] - ntm) - zs * nbm * Em - k.dmd[s] * nbm * dr_m);
          flux_out[(s * 3 + a) * N + i] = Fp;
          tot += Fp + Fm;
        }
        Fel[a] += -tot * k.inv_2D;  // friction (Sec. II.C eq. frictionforce), faces shared by two cells
      }
    }
  } else if (IONS) {
    // no potential and no applied field: diffusion and solvation fluxes only
    const T pf_i = SOL ? psi_f[i] : T(1);
    T nt_i[2];
#pragma unroll
    for (int s = 0; s < 2; ++s) nt_i[s] = pf_i > T(0) ? n[s * N + i] / pf_i : T(0);
    const T ra_i = rho[0];
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      const int jp = ax[2 * a], jm = ax[2 * a + 1];
      const T pf_p = SOL ? psi_f[jp] : T(1);
      const T pf_m = SOL ? psi_f[jm] : T(1);
      const T dr_p = rhoF[jp] - ra_i;
      const T dr_m = ra_i - rhoF[jm];
      const T wp = k.D * pf_i * pf_p;
      const T wm = k.D * pf_m * pf_i;
      T tot = T(0);
#pragma unroll
      for (int s = 0; s < 2; ++s) {
        const T ntp = pf_p > T(0) ? n[s * N + jp] / pf_p : T(0);
        const T ntm = pf_m > T(0) ? n[s * N + jm] / pf_m : T(0);
        const T nbp = T(0.5) * (nt_i[s] + ntp);
        const T nbm = T(0.5) * (ntm + nt_i[s]);
        const T Fp = wp * ((ntp - nt_i[s]) - k.dmd[s] * nbp * dr_p);
        const T Fm = wm * ((nt_i[s] - ntm) - k.dmd[s] * nbm * dr_m);
        flux_out[(s * 3 + a) * N + i] = Fp;
        tot += Fp + Fm;
      }
      Fel[a] += -tot * k.inv_2D;
    }
  }

  // electric and friction forces shared by mass fraction
#pragma unroll
  for (int s = 0; s < NC; ++s) {
    const T fr = rho[s] * inv_rho;
#pragma unroll
    for (int a = 0; a < 3; ++a) Phi[s][a] += fr * Fel[a];
  }
  T ue[2][3];
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    const T ubar = J[a] * inv_rho;
    const T ps = Phi[0][a] + (NC == 2 ? Phi[1][a] : T(0));
    u_out[a * N + i] = (J[a] + T(0.5) * ps) * inv_rho;
#pragma unroll
    for (int s = 0; s < NC; ++s) ue[s][a] = rho[s] > T(0) ? ubar + k.tau * Phi[s][a] / rho[s] : ubar;
  }

  // forced BGK collision with the shifted equilibrium velocity, push streaming,
  // halfway bounce-back on links to solid nodes (Sec. II.A, II.E)
#pragma unroll
  for (int s = 0; s < NC; ++s) {
    const S *fs = f + (size_t)(s * 19) * N;
    S *fns = fn + (size_t)(s * 19) * N;
    const T sh = k.shift[s];
    T fl[19];
#pragma unroll
    for (int qd = 0; qd < 19; ++qd) fl[qd] = sload<RO, S, T>(fs, (size_t)qd * N + i, wq<T>(qd) * sh);
    const T usq = ue[s][0] * ue[s][0] + ue[s][1] * ue[s][1] + ue[s][2] * ue[s][2];
#pragma unroll
    for (int qd = 0; qd < 19; ++qd) {
      const T cu = T(cx(qd)) * ue[s][0] + T(cy(qd)) * ue[s][1] + T(cz(qd)) * ue[s][2];
      const T feq = wq<T>(qd) * rho[s] * (T(1) + T(3) * cu + T(4.5) * cu * cu - T(1.5) * usq);
      const T fpost = fl[qd] + (feq - fl[qd]) * k.inv_tau;
      if (qd == 0) {
        Store<S, T>::st(fns, (size_t)i, fpost, wq<T>(0) * sh);
      } else {
        const int jn = NB(qd);
        if (SOL && solid[jn]) {
          const int o = owner[jn];
          const T cvd = T(double(cx(qd)) * cv[3 * o] + double(cy(qd)) * cv[3 * o + 1] +
                          double(cz(qd)) * cv[3 * o + 2]);
          const T val = fpost - T(6) * wq<T>(qd) * rho[s] * cvd;
          Store<S, T>::st(fns, (size_t)opp(qd) * N + i, val, wq<T>(qd) * sh);
        } else {
          Store<S, T>::st(fns, (size_t)qd * N + jn, fpost, wq<T>(qd) * sh);
        }
      }
    }
  }
}

// One component keeps about half the live state of two: four resident blocks
// per SM (64 registers) hide more latency there; two components stay at three.
template <typename S, typename T, int NC, bool SOL, bool IONS>
__global__ void __launch_bounds__(256, NC == 1 ? 4 : 3)
    k_collide(StepK<T> k, const S *__restrict__ f, S *__restrict__ fn, const T *__restrict__ rhoF,
              const T *__restrict__ JF, const T *__restrict__ psiF, const T *__restrict__ eps,
              const T *__restrict__ phi, const T *__restrict__ n, const T *__restrict__ psi_f,
              const uint8_t *__restrict__ solid, const int *__restrict__ owner, const double *__restrict__ cv,
              T *__restrict__ u_out, T *__restrict__ flux_out) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= int(k.d.N)) return;
  collide_site<S, T, NC, SOL, IONS, true>(k, f, fn, rhoF, JF, psiF, eps, phi, n, psi_f, solid, owner, cv, u_out,
                                          flux_out, i);
}

// ---------------------------------------------------------------- k_np
template <typename T, bool SOL>
__device__ __forceinline__ void np_site(const StepK<T> &k, const T *__restrict__ n, T *__restrict__ nn,
                                        const T *__restrict__ flux, const T *__restrict__ u,
                                        const uint8_t *__restrict__ solid, const long long i) {
  const Dims d = k.d;
  const long long N = d.N;
  if (SOL && solid[i]) {
    nn[i] = T(0);
    nn[N + i] = T(0);
    return;
  }
  // 32-bit site arithmetic (boxes below 2^31 sites): one unsigned division per
  // axis instead of the 64-bit ones, neighbours by periodic offsets
  const unsigned ii = unsigned(i), unx = unsigned(d.nx), uny = unsigned(d.ny);
  const unsigned r = ii / unx, x = ii - r * unx;
  const unsigned z = r / uny, y = r - z * uny;
  const unsigned nxy = unx * uny;
  const unsigned jm[3] = {x == 0 ? ii + unx - 1u : ii - 1u, y == 0 ? ii + (uny - 1u) * unx : ii - unx,
                          z == 0 ? ii + (unsigned(d.nz) - 1u) * nxy : ii - nxy};
  const unsigned jp[3] = {x + 1u == unx ? ii + 1u - unx : ii + 1u, y + 1u == uny ? ii - (uny - 1u) * unx : ii + unx,
                          z + 1u == unsigned(d.nz) ? ii - (unsigned(d.nz) - 1u) * nxy : ii + nxy};
  bool okp[3], okm[3];
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    okp[a] = !SOL || !solid[jp[a]];
    okm[a] = !SOL || !solid[jm[a]];
  }
  T ui[3], up[3], um[3];
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    ui[a] = u[a * N + i];
    um[a] = u[a * N + jm[a]];  // the cell upstream along +a
    up[a] = u[a * N + jp[a]];  // the cell upstream along -a
  }
#pragma unroll
  for (int s = 0; s < 2; ++s) {
    const T ni = n[s * N + i];
    T div = T(0);
#pragma unroll
    for (int a = 0; a < 3; ++a) div += flux[(s * 3 + a) * N + i] - flux[(s * 3 + a) * N + jm[a]];
    T out = T(0), in = T(0);
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      // +a: i sends max(u_a,0) n_i to i+a; i receives from i-a its max(u_a(i-a),0) n_{i-a}
      if (okp[a]) out += fmax(ui[a], T(0)) * ni;
      if (okm[a]) out += fmax(-ui[a], T(0)) * ni;
    }
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      if (okm[a]) in += fmax(um[a], T(0)) * n[s * N + jm[a]];
      if (okp[a]) in += fmax(-up[a], T(0)) * n[s * N + jp[a]];
    }
    nn[s * N + i] = ((ni + div) - out) + in;
  }
}

template <typename T, bool SOL>
__global__ void __launch_bounds__(256) k_np(StepK<T> k, const T *__restrict__ n, T *__restrict__ nn,
                                            const T *__restrict__ flux, const T *__restrict__ u,
                                            const uint8_t *__restrict__ solid) {
  const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (i >= k.d.N) return;
  np_site<T, SOL>(k, n, nn, flux, u, solid, i);
}

// ---------------------------------------------------------------- init / read-out
template <typename S, typename T, int NC, typename R>
__global__ void k_init_eq(StepK<T> k, S *__restrict__ f, const R *__restrict__ rho, const R *__restrict__ u,
                          const uint8_t *__restrict__ solid) {
  const long long N = k.d.N;
  long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (i >= N) return;
  const bool sol = k.solids && solid[i];
  T uu[3] = {T(0), T(0), T(0)};
  if (u) {
    uu[0] = T(u[i]);
    uu[1] = T(u[N + i]);
    uu[2] = T(u[2 * N + i]);
  }
  const T usq = uu[0] * uu[0] + uu[1] * uu[1] + uu[2] * uu[2];
#pragma unroll
  for (int s = 0; s < NC; ++s) {
    const T r = sol ? T(0) : T(rho[s * N + i]);
#pragma unroll
    for (int qd = 0; qd < 19; ++qd) {
      const T cu = T(cx(qd)) * uu[0] + T(cy(qd)) * uu[1] + T(cz(qd)) * uu[2];
      const T feq = wq<T>(qd) * r * (T(1) + T(3) * cu + T(4.5) * cu * cu - T(1.5) * usq);
      Store<S, T>::st(f, (size_t)(s * 19 + qd) * N + i, feq, wq<T>(qd) * k.shift[s]);
    }
  }
}

template <typename S, typename T, int NC>
__global__ void k_init_f(StepK<T> k, S *__restrict__ f, const double *__restrict__ src,
                         const uint8_t *__restrict__ solid) {
  const long long N = k.d.N;
  long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (i >= N) return;
  const bool sol = k.solids && solid[i];
  for (int s = 0; s < NC; ++s)
    for (int qd = 0; qd < 19; ++qd) {
      size_t j = (size_t)(s * 19 + qd) * N + i;
      Store<S, T>::st(f, j, sol ? T(0) : T(src[j]), wq<T>(qd) * k.shift[s]);
    }
}

template <typename S, typename T, int NC>
__global__ void k_get_f(StepK<T> k, const S *__restrict__ f, double *__restrict__ out,
                        const uint8_t *__restrict__ solid) {
  const long long N = k.d.N;
  long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (i >= N) return;
  const bool sol = k.solids && solid[i];
  for (int s = 0; s < NC; ++s)
    for (int qd = 0; qd < 19; ++qd) {
      size_t j = (size_t)(s * 19 + qd) * N + i;
      out[j] = sol ? 0.0 : double(Store<S, T>::ld(f, j, wq<T>(qd) * k.shift[s]));
    }
}

template <typename S, typename T, int NC>
__global__ void k_get_rho(StepK<T> k, const S *__restrict__ f, double *__restrict__ out,
                          const uint8_t *__restrict__ solid) {
  const long long N = k.d.N;
  long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (i >= N) return;
  const bool sol = k.solids && solid[i];
  for (int s = 0; s < NC; ++s) {
    T acc = T(0);
    if (!sol)
      for (int qd = 0; qd < 19; ++qd)
        acc += Store<S, T>::ld(f, (size_t)(s * 19 + qd) * N + i, wq<T>(qd) * k.shift[s]);
    out[s * N + i] = double(acc);
  }
}

// ---------------------------------------------------------------- observables
// Per-block FP64 partial sums, fixed order (per thread, then a tree).
// Layout: 0,1 mass; 2,3 ions; 4 charge; 5..7 momentum; 8 W; 9..11 W x,y,z;
// 12 W x^2; 13 W z^2; 14,15 unused.  Per thread the sums run in double-float
// words in the FP32 modes (the FP64 rate of the target is a small fraction of
// its FP32 rate) with the products W x, W x^2 formed exactly, in FP64 in the
// FP64 mode; site indices are 32-bit (boxes below 2^31 sites).
//
// The populations stream through shared memory: a block owns chunks of
// kObsChunk consecutive sites (one per thread) and copies every population
// row and both ion rows of its next chunk with 16-byte asynchronous copies
// while it sums the current one, so each SM keeps whole chunks in flight
// instead of the few loads a thread's registers can cover.  Boxes whose rows
// do not start on 16-byte boundaries, and the sites past the last whole
// chunk, are read directly.
constexpr int kObsChunk = 256;

template <typename S, typename T, int NC> struct ObsLayout {
  static constexpr int kRows = NC * 19;
  static constexpr int kPopBytes = kRows * kObsChunk * int(sizeof(S));
  static constexpr int kBufBytes = kPopBytes + 2 * kObsChunk * int(sizeof(T));
  static constexpr int kTreeBytes = kObsLen * kObsChunk * 8;
  static constexpr int kSmem = 2 * kBufBytes > kTreeBytes ? 2 * kBufBytes : kTreeBytes;
};

__device__ __forceinline__ void obs_cp16(unsigned char *dst, const void *src) {
  const unsigned d = unsigned(__cvta_generic_to_shared(dst));
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(d), "l"(src) : "memory");
}
__device__ __forceinline__ void obs_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
__device__ __forceinline__ void obs_wait_older() { asm volatile("cp.async.wait_group 1;\n" ::: "memory"); }
__device__ __forceinline__ void obs_wait_all() { asm volatile("cp.async.wait_all;\n" ::: "memory"); }

// copies of chunk sites [c0, c0 + kObsChunk): population row r to buf row r,
// ion rows after the populations
template <typename S, typename T, int NC>
__device__ __forceinline__ void obs_issue(unsigned char *buf, const S *__restrict__ f, const T *__restrict__ n,
                                          unsigned N, unsigned c0, bool ions) {
  using L = ObsLayout<S, T, NC>;
  constexpr int PV = kObsChunk * int(sizeof(S)) / 16;  // 16-byte pieces of a population row
  constexpr int IV = kObsChunk * int(sizeof(T)) / 16;
  for (int e = threadIdx.x; e < L::kRows * PV; e += blockDim.x) {
    const int r = e / PV, v = e - r * PV;
    obs_cp16(buf + (r * kObsChunk) * int(sizeof(S)) + 16 * v,
             reinterpret_cast<const unsigned char *>(f + (size_t)r * N + c0) + 16 * v);
  }
  if (ions)
    for (int e = threadIdx.x; e < 2 * IV; e += blockDim.x) {
      const int r = e / IV, v = e - r * IV;
      obs_cp16(buf + L::kPopBytes + (r * kObsChunk) * int(sizeof(T)) + 16 * v,
               reinterpret_cast<const unsigned char *>(n + (size_t)r * N + c0) + 16 * v);
    }
}

// one site's contributions; pop(s, q) is population q of component s
template <typename T, int NC, class Acc, class Pop>
__device__ __forceinline__ void obs_site(Acc *acc, const StepK<T> &k, unsigned i, unsigned nx, unsigned ny, bool sol,
                                         T np, T nm, T qcv, const Pop &pop) {
  if (k.nions) {
    acc[2].add(np);
    acc[3].add(nm);
    acc[4].add(np);
    acc[4].add(-nm);
  }
  if (k.solids) acc[4].add(qcv);
  if (sol) return;
  T rt[2] = {T(0), T(0)}, Jt[3] = {T(0), T(0), T(0)};
#pragma unroll
  for (int s = 0; s < NC; ++s)
#pragma unroll
    for (int qd = 0; qd < 19; ++qd) {
      const T v = pop(s, qd);
      rt[s] += v;
      if (cx(qd)) Jt[0] += T(cx(qd)) * v;
      if (cy(qd)) Jt[1] += T(cy(qd)) * v;
      if (cz(qd)) Jt[2] += T(cz(qd)) * v;
    }
  acc[0].add(rt[0]);
  acc[1].add(rt[1]);
  acc[5].add(Jt[0]);
  acc[6].add(Jt[1]);
  acc[7].add(Jt[2]);
  if (NC == 2) {
    const T tot = rt[0] + rt[1];
    const T c = tot > T(0) ? (rt[1] - rt[0]) / tot : T(0);
    if (c > T(0)) {
      const unsigned r = i / nx, x = i - r * nx, z = r / ny, y = r - z * ny;
      acc[8].add(c);
      acc_prod(acc[9], c, T(x));
      acc_prod(acc[10], c, T(y));
      acc_prod(acc[11], c, T(z));
      acc_prod2(acc[12], c, T(x));
      acc_prod2(acc[13], c, T(z));
    }
  }
}

// blockDim.x == kObsChunk; nfull whole chunks are staged (0: none)
template <typename S, typename T, int NC>
__global__ void __launch_bounds__(kObsChunk) k_obs(StepK<T> k, const S *__restrict__ f, const T *__restrict__ n,
                                                   const T *__restrict__ qc, const uint8_t *__restrict__ solid,
                                                   double *__restrict__ partials, unsigned nfull) {
  using L = ObsLayout<S, T, NC>;
  extern __shared__ __align__(16) unsigned char obs_sm[];
  const Dims d = k.d;
  const unsigned N = unsigned(d.N), nx = unsigned(d.nx), ny = unsigned(d.ny);
  const bool ions = k.nions != 0;
  SumAcc<std::is_same<T, float>::value> acc[kObsLen];
  const unsigned t = threadIdx.x;
  unsigned c = blockIdx.x;
  if (c < nfull) obs_issue<S, T, NC>(obs_sm, f, n, N, c * kObsChunk, ions);
  obs_commit();
  for (int b = 0; c < nfull; c += gridDim.x, b ^= 1) {
    unsigned char *cur = obs_sm + b * L::kBufBytes, *nxt = obs_sm + (b ^ 1) * L::kBufBytes;
    if (c + gridDim.x < nfull) obs_issue<S, T, NC>(nxt, f, n, N, (c + gridDim.x) * kObsChunk, ions);
    obs_commit();
    obs_wait_older();  // chunk c has landed
    __syncthreads();
    const S *ps = reinterpret_cast<const S *>(cur);
    const T *ns = reinterpret_cast<const T *>(cur + L::kPopBytes);
    const unsigned i = c * kObsChunk + t;
    obs_site<T, NC>(acc, k, i, nx, ny, k.solids && solid[i], ions ? ns[t] : T(0), ions ? ns[kObsChunk + t] : T(0),
                    k.solids ? qc[i] : T(0), [&](int s, int qd) {
                      return Store<S, T>::ldc(ps, (s * 19 + qd) * kObsChunk + t, wq<T>(qd) * k.shift[s]);
                    });
    __syncthreads();  // buffer cur is refilled in the next iteration
  }
  obs_wait_all();
  for (unsigned i = nfull * kObsChunk + blockIdx.x * kObsChunk + t; i < N; i += gridDim.x * kObsChunk)
    obs_site<T, NC>(acc, k, i, nx, ny, k.solids && solid[i], ions ? n[i] : T(0), ions ? n[N + i] : T(0),
                    k.solids ? qc[i] : T(0), [&](int s, int qd) {
                      return Store<S, T>::ld(f, (size_t)(s * 19 + qd) * N + i, wq<T>(qd) * k.shift[s]);
                    });
  __syncthreads();
  double(*sh)[kObsChunk] = reinterpret_cast<double(*)[kObsChunk]>(obs_sm);
#pragma unroll
  for (int m = 0; m < kObsLen; ++m) sh[m][t] = acc[m].get();
  __syncthreads();
  for (int w = kObsChunk / 2; w > 0; w >>= 1) {
    if (t < unsigned(w))
#pragma unroll
      for (int m = 0; m < kObsLen; ++m) sh[m][t] += sh[m][t + w];
    __syncthreads();
  }
  if (t < unsigned(kObsLen)) partials[blockIdx.x * kObsLen + t] = sh[t][0];
}

// ---------------------------------------------------------------- colloid momentum exchange
// One block per colloid: for fluid nodes of its bounding box and links to its
// solid nodes, the momentum [2 f*_q - 6 w_q rho (c_q.v)] c_q with
// f*_q = fn_{opp(q)} + 6 w_q rho (c_q.v) recovered from the bounced population.
template <typename S, typename T, int NC>
__global__ void k_colloid_bb(StepK<T> k, const S *__restrict__ fn, const T *__restrict__ rhoF,
                             const uint8_t *__restrict__ solid, const int *__restrict__ owner,
                             const uint8_t *__restrict__ surface, const T *__restrict__ qc,
                             const T *__restrict__ phi, const double *__restrict__ ccx, const double *__restrict__ ccr,
                             const double *__restrict__ cv, double *__restrict__ cforce) {
  const int j = blockIdx.x;
  const Dims d = k.d;
  const long long N = d.N;
  int lo[3], cnt[3];
  const int dims[3] = {d.nx, d.ny, d.nz};
  for (int a = 0; a < 3; ++a) {
    double X = ccx[3 * j + a], r = ccr[j];
    lo[a] = int(ceil(X - r - 2.0));
    int hi = int(floor(X + r + 2.0));
    cnt[a] = min(dims[a], hi - lo[a] + 1);
  }
  const double v[3] = {cv[3 * j], cv[3 * j + 1], cv[3 * j + 2]};
  double acc[3] = {0, 0, 0};
  const long long tot = (long long)cnt[0] * cnt[1] * cnt[2];
  for (long long t = threadIdx.x; t < tot; t += blockDim.x) {
    int x = ((lo[0] + int(t % cnt[0])) % d.nx + d.nx) % d.nx;
    int y = ((lo[1] + int((t / cnt[0]) % cnt[1])) % d.ny + d.ny) % d.ny;
    int z = ((lo[2] + int(t / ((long long)cnt[0] * cnt[1]))) % d.nz + d.nz) % d.nz;
    long long i = site(d, x, y, z);
    long long nb[19];
    neighbours19(d, x, y, z, nb);
    if (solid[i]) {
      // electric force q_c E on the colloid's surface charge (Sec. II.E)
      if (k.has_field && surface[i] && owner[i] == j) {
        const double q = double(qc[i]);
        acc[0] += q * (-0.5 * (double(phi[nb[1]]) - double(phi[nb[2]])) + double(k.Eext[0]));
        acc[1] += q * (-0.5 * (double(phi[nb[3]]) - double(phi[nb[4]])) + double(k.Eext[1]));
        acc[2] += q * (-0.5 * (double(phi[nb[5]]) - double(phi[nb[6]])) + double(k.Eext[2]));
      }
      continue;
    }
    for (int qd = 1; qd < 19; ++qd) {
      if (!solid[nb[qd]] || owner[nb[qd]] != j) continue;
      const double cvd = cx(qd) * v[0] + cy(qd) * v[1] + cz(qd) * v[2];
      double dp = 0;
      for (int s = 0; s < NC; ++s) {
        const double r = double(rhoF[s * N + i]);
        const double corr = 6.0 * wq<double>(qd) * r * cvd;
        const double back = double(Store<S, T>::ld(fn, (size_t)(s * 19 + opp(qd)) * N + i,
                                                   wq<T>(qd) * k.shift[s]));
        dp += 2.0 * (back + corr) - corr;
      }
      acc[0] += cx(qd) * dp;
      acc[1] += cy(qd) * dp;
      acc[2] += cz(qd) * dp;
    }
  }
  __shared__ double sh[3][256];
  for (int a = 0; a < 3; ++a) sh[a][threadIdx.x] = acc[a];
  __syncthreads();
  for (int w = blockDim.x / 2; w > 0; w >>= 1) {
    if (threadIdx.x < w)
      for (int a = 0; a < 3; ++a) sh[a][threadIdx.x] += sh[a][threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x < 3) cforce[3 * j + threadIdx.x] = sh[threadIdx.x][0];
}


// ---------------------------------------------------------------- colloid remap (Sec. II.E)
// Walks the bounding box of colloid j at its new position (margin covers one
// lattice step of motion).  Covered nodes (solid now, fluid before) give the
// fluid momentum sum_sigma sum_q f c_q to the colloid; uncovered nodes (fluid
// now, solid before, previously owned by j) are refilled with the equilibrium
// at the mean density of the neighbours that are fluid before and after, at
// the colloid velocity, and the colloid loses that momentum.  dp[j] receives
// the colloid's momentum change.
template <typename S, typename T, int NC>
__global__ void k_remap(StepK<T> k, S *__restrict__ f, const uint8_t *__restrict__ solid,
                        const uint8_t *__restrict__ solid_old, const int *__restrict__ owner,
                        const int *__restrict__ owner_old, const double *__restrict__ ccx,
                        const double *__restrict__ ccr, const double *__restrict__ cv, double *__restrict__ dp) {
  const int j = blockIdx.x;
  const Dims d = k.d;
  const long long N = d.N;
  int lo[3], cnt[3];
  const int dims[3] = {d.nx, d.ny, d.nz};
  for (int a = 0; a < 3; ++a) {
    const double X = ccx[3 * j + a], r = ccr[j];
    lo[a] = int(ceil(X - r - 3.0));
    const int hi = int(floor(X + r + 3.0));
    cnt[a] = min(dims[a], hi - lo[a] + 1);
  }
  const double v[3] = {cv[3 * j], cv[3 * j + 1], cv[3 * j + 2]};
  double acc[3] = {0, 0, 0};
  const long long tot = (long long)cnt[0] * cnt[1] * cnt[2];
  for (long long t = threadIdx.x; t < tot; t += blockDim.x) {
    const int x = ((lo[0] + int(t % cnt[0])) % d.nx + d.nx) % d.nx;
    const int y = ((lo[1] + int((t / cnt[0]) % cnt[1])) % d.ny + d.ny) % d.ny;
    const int z = ((lo[2] + int(t / ((long long)cnt[0] * cnt[1]))) % d.nz + d.nz) % d.nz;
    const long long i = site(d, x, y, z);
    const bool now = solid[i], before = solid_old[i];
    if (now && !before && owner[i] == j) {
      // covered: fluid momentum to the colloid
      for (int s = 0; s < NC; ++s)
        for (int qd = 1; qd < 19; ++qd) {
          const double fv = double(Store<S, T>::ld(f, (size_t)(s * 19 + qd) * N + i, wq<T>(qd) * k.shift[s]));
          acc[0] += cx(qd) * fv;
          acc[1] += cy(qd) * fv;
          acc[2] += cz(qd) * fv;
        }
    } else if (!now && before && owner_old[i] == j) {
      // uncovered: equilibrium refill at the neighbour-mean density
      long long nb[19];
      neighbours19(d, x, y, z, nb);
      double rs[2] = {0.0, 0.0};
      int m = 0;
      for (int qd = 1; qd < 19; ++qd) {
        const long long jn = nb[qd];
        if (solid[jn] || solid_old[jn]) continue;
        ++m;
        for (int s = 0; s < NC; ++s)
          for (int q2 = 0; q2 < 19; ++q2)
            rs[s] += double(Store<S, T>::ld(f, (size_t)(s * 19 + q2) * N + jn, wq<T>(q2) * k.shift[s]));
      }
      const double usq = v[0] * v[0] + v[1] * v[1] + v[2] * v[2];
      for (int s = 0; s < NC; ++s) {
        const double rb = m > 0 ? rs[s] / double(m) : 0.0;
        for (int qd = 0; qd < 19; ++qd) {
          const double cu = cx(qd) * v[0] + cy(qd) * v[1] + cz(qd) * v[2];
          const double feq = wq<double>(qd) * rb * (1.0 + 3.0 * cu + 4.5 * cu * cu - 1.5 * usq);
          Store<S, T>::st(f, (size_t)(s * 19 + qd) * N + i, T(feq), wq<T>(qd) * k.shift[s]);
        }
        acc[0] -= rb * v[0];
        acc[1] -= rb * v[1];
        acc[2] -= rb * v[2];
      }
    }
  }
  __shared__ double sh[3][256];
  for (int a = 0; a < 3; ++a) sh[a][threadIdx.x] = acc[a];
  __syncthreads();
  for (int w = blockDim.x / 2; w > 0; w >>= 1) {
    if (threadIdx.x < w)
      for (int a = 0; a < 3; ++a) sh[a][threadIdx.x] += sh[a][threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x < 3) dp[3 * j + threadIdx.x] = sh[threadIdx.x][0];
}

// Ions of covered nodes go in equal shares to their D3Q19 neighbours that are
// fluid before and after the move.  Pass 1 (one block per colloid, its new
// bounding box): each covered node stores its share n/m (m kept neighbours),
// clears its own ions and flags its kept neighbours.  Pass 2 (whole lattice,
// a flag byte per site): flagged nodes gather the shares of their covered
// neighbours in a fixed order and clear the flag.
template <typename T>
__global__ void k_remap_mark(StepK<T> k, T *__restrict__ n, const uint8_t *__restrict__ solid,
                             const uint8_t *__restrict__ solid_old, const int *__restrict__ owner,
                             const double *__restrict__ ccx, const double *__restrict__ ccr, T *__restrict__ share,
                             uint8_t *__restrict__ flag) {
  const int j = blockIdx.x;
  const Dims d = k.d;
  const long long N = d.N;
  int lo[3], cnt[3];
  const int dims[3] = {d.nx, d.ny, d.nz};
  for (int a = 0; a < 3; ++a) {
    const double X = ccx[3 * j + a], r = ccr[j];
    lo[a] = int(ceil(X - r - 2.0));
    const int hi = int(floor(X + r + 2.0));
    cnt[a] = min(dims[a], hi - lo[a] + 1);
  }
  const long long tot = (long long)cnt[0] * cnt[1] * cnt[2];
  for (long long t = threadIdx.x; t < tot; t += blockDim.x) {
    const int x = ((lo[0] + int(t % cnt[0])) % d.nx + d.nx) % d.nx;
    const int y = ((lo[1] + int((t / cnt[0]) % cnt[1])) % d.ny + d.ny) % d.ny;
    const int z = ((lo[2] + int(t / ((long long)cnt[0] * cnt[1]))) % d.nz + d.nz) % d.nz;
    const long long src = site(d, x, y, z);
    if (!(solid[src] && !solid_old[src] && owner[src] == j)) continue;
    long long sn[19];
    neighbours19(d, x, y, z, sn);
    int m = 0;
    for (int q2 = 1; q2 < 19; ++q2) m += (!solid[sn[q2]] && !solid_old[sn[q2]]) ? 1 : 0;
    for (int s = 0; s < 2; ++s) {
      share[s * N + src] = m > 0 ? n[s * N + src] / T(m) : T(0);
      n[s * N + src] = T(0);
    }
    for (int q2 = 1; q2 < 19; ++q2)
      if (!solid[sn[q2]] && !solid_old[sn[q2]]) flag[sn[q2]] = 1;
  }
}

template <typename T>
__global__ void __launch_bounds__(256) k_remap_ions(StepK<T> k, T *__restrict__ n, const uint8_t *__restrict__ solid,
                                                    const uint8_t *__restrict__ solid_old,
                                                    const T *__restrict__ share, uint8_t *__restrict__ flag) {
  const Dims d = k.d;
  const long long N = d.N;
  long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (i >= N || !flag[i]) return;
  flag[i] = 0;
  int x, y, z;
  coords(d, i, x, y, z);
  long long nb[19];
  neighbours19(d, x, y, z, nb);
  T add[2] = {T(0), T(0)};
  for (int qd = 1; qd < 19; ++qd) {
    const long long src = nb[opp(qd)];  // node i - c_q sends along c_q to i
    if (!(solid[src] && !solid_old[src])) continue;
    for (int s = 0; s < 2; ++s) add[s] += share[s * N + src];
  }
  n[i] += add[0];
  n[N + i] += add[1];
}

// ---------------------------------------------------------------- host launchers
template <typename S, typename T> struct Launch {
  static constexpr int B = 256;

  template <typename R> static void init_eq_from(Ctx &c, const R *rho, const R *u) {
    auto k = make_stepk<T>(c);
    S *f = (S *)c.f[c.cur];
    if (c.ncomp == 2)
      count_launch(), k_init_eq<S, T, 2, R><<<grid_for(c.d.N, B), B, 0, c.s>>>(k, f, rho, u, c.solid);
    else
      count_launch(), k_init_eq<S, T, 1, R><<<grid_for(c.d.N, B), B, 0, c.s>>>(k, f, rho, u, c.solid);
  }
  static void init_eq(Ctx &c, const void *rho, const void *u, int f32) {
    if (f32)
      init_eq_from<float>(c, (const float *)rho, (const float *)u);
    else
      init_eq_from<double>(c, (const double *)rho, (const double *)u);
  }
  static void init_f(Ctx &c, const double *src) {
    auto k = make_stepk<T>(c);
    S *f = (S *)c.f[c.cur];
    if (c.ncomp == 2)
      count_launch(), k_init_f<S, T, 2><<<grid_for(c.d.N, B), B, 0, c.s>>>(k, f, src, c.solid);
    else
      count_launch(), k_init_f<S, T, 1><<<grid_for(c.d.N, B), B, 0, c.s>>>(k, f, src, c.solid);
  }
  static void get_f(Ctx &c, double *out) {
    auto k = make_stepk<T>(c);
    const S *f = (const S *)c.f[c.cur];
    if (c.ncomp == 2)
      count_launch(), k_get_f<S, T, 2><<<grid_for(c.d.N, B), B, 0, c.s>>>(k, f, out, c.solid);
    else
      count_launch(), k_get_f<S, T, 1><<<grid_for(c.d.N, B), B, 0, c.s>>>(k, f, out, c.solid);
  }
  static void get_rho(Ctx &c, double *out) {
    auto k = make_stepk<T>(c);
    const S *f = (const S *)c.f[c.cur];
    if (c.ncomp == 2)
      count_launch(), k_get_rho<S, T, 2><<<grid_for(c.d.N, B), B, 0, c.s>>>(k, f, out, c.solid);
    else
      count_launch(), k_get_rho<S, T, 1><<<grid_for(c.d.N, B), B, 0, c.s>>>(k, f, out, c.solid);
  }
  static void macro(Ctx &c) {
    auto k = make_stepk<T>(c);
    const S *f = (const S *)c.f[c.cur];
    const T *n = (const T *)c.n[c.ncur];
    if (c.ncomp == 2)
      count_launch(), k_macro<S, T, 2><<<grid_for(c.d.N, B), B, 0, c.s>>>(
          k, f, (T *)c.rho, (T *)c.J, (T *)c.psi, (T *)c.eps, (T *)c.q, n, (const T *)c.qc, (const T *)c.psi_s,
          c.solid);
    else
      count_launch(), k_macro<S, T, 1><<<grid_for(c.d.N, B), B, 0, c.s>>>(
          k, f, (T *)c.rho, (T *)c.J, (T *)c.psi, (T *)c.eps, (T *)c.q, n, (const T *)c.qc, (const T *)c.psi_s,
          c.solid);
  }
  static void virt(Ctx &c) {
    if (!c.solids || c.ncoll == 0) return;
    auto k = make_stepk<T>(c);
    if (c.ncomp == 2)
      count_launch(), k_virtual<T, 2><<<c.ncoll, B, 0, c.s>>>(k, (T *)c.rho, (T *)c.psi, (T *)c.eps, (const T *)c.psi_s, c.solid,
                                              c.surface, c.owner, c.cx, c.cr);
    else
      count_launch(), k_virtual<T, 1><<<c.ncoll, B, 0, c.s>>>(k, (T *)c.rho, (T *)c.psi, (T *)c.eps, (const T *)c.psi_s, c.solid,
                                              c.surface, c.owner, c.cx, c.cr);
  }
  template <int NC, bool SOL, bool IONS> static void collide_v(Ctx &c) {
    auto k = make_stepk<T>(c);
    count_launch(), k_collide<S, T, NC, SOL, IONS><<<grid_for(c.d.N, B), B, 0, c.s>>>(
        k, (const S *)c.f[c.cur], (S *)c.f[1 - c.cur], (const T *)c.rho, (const T *)c.J, (const T *)c.psi,
        (const T *)c.eps, (const T *)c.phit, (const T *)c.n[c.ncur], (const T *)c.psi_f, c.solid, c.owner, c.cv,
        (T *)c.u, (T *)c.flux);
  }
  static void collide(Ctx &c) {
    const bool ions = c.nions > 0;
    if (c.ncomp == 2) {
      if (c.solids) { ions ? collide_v<2, true, true>(c) : collide_v<2, true, false>(c); }
      else { ions ? collide_v<2, false, true>(c) : collide_v<2, false, false>(c); }
    } else {
      if (c.solids) { ions ? collide_v<1, true, true>(c) : collide_v<1, true, false>(c); }
      else { ions ? collide_v<1, false, true>(c) : collide_v<1, false, false>(c); }
    }
  }
  static void np(Ctx &c) {
    if (!c.nions) return;
    auto k = make_stepk<T>(c);
    const T *n = (const T *)c.n[c.ncur];
    T *nn = (T *)c.n[1 - c.ncur];
    if (c.solids)
      count_launch(), k_np<T, true><<<grid_for(c.d.N, B), B, 0, c.s>>>(k, n, nn, (const T *)c.flux, (const T *)c.u, c.solid);
    else
      count_launch(), k_np<T, false><<<grid_for(c.d.N, B), B, 0, c.s>>>(k, n, nn, (const T *)c.flux, (const T *)c.u, c.solid);
  }
  // one resident wave of k_obs (at most max_blocks); returns its block count
  template <int NC> static int obs_launch(Ctx &c, double *partials, int max_blocks) {
    using L = ObsLayout<S, T, NC>;
    static int per_dev[64];  // resident blocks per SM, by device ordinal (0: not yet known)
    int dev = 0, nsm = 1;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    int per = dev >= 0 && dev < 64 ? per_dev[dev] : 0;
    if (per == 0) {
      cudaFuncSetAttribute(k_obs<S, T, NC>, cudaFuncAttributeMaxDynamicSharedMemorySize, L::kSmem);
      if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_obs<S, T, NC>, kObsChunk, L::kSmem) != cudaSuccess ||
          per < 1) {
        cudaGetLastError();
        per = 1;
      }
      if (dev >= 0 && dev < 64) per_dev[dev] = per;
    }
    const int nb = std::max(1, std::min(max_blocks, per * std::max(1, nsm)));
    const S *f = (const S *)c.f[c.cur];
    const T *n = (const T *)c.n[c.ncur];
    const unsigned N = unsigned(c.d.N);
    // 16-byte copies need every row to start on a 16-byte boundary
    const bool aligned = (size_t(N) * sizeof(S)) % 16 == 0 && (size_t(N) * sizeof(T)) % 16 == 0 &&
                         reinterpret_cast<uintptr_t>(f) % 16 == 0 && (!c.nions || reinterpret_cast<uintptr_t>(n) % 16 == 0);
    const unsigned nfull = aligned ? N / kObsChunk : 0u;
    count_launch(), k_obs<S, T, NC><<<nb, kObsChunk, L::kSmem, c.s>>>(make_stepk<T>(c), f, n, (const T *)c.qc, c.solid,
                                                                       partials, nfull);
    return nb;
  }
  static int obs_partials(Ctx &c, double *partials, int max_blocks) {
    return c.ncomp == 2 ? obs_launch<2>(c, partials, max_blocks) : obs_launch<1>(c, partials, max_blocks);
  }
  static void colloid_bb(Ctx &c) {
    if (!c.solids || c.ncoll == 0) return;
    auto k = make_stepk<T>(c);
    const S *fn = (const S *)c.f[c.cur];
    if (c.ncomp == 2)
      count_launch(), k_colloid_bb<S, T, 2><<<c.ncoll, B, 0, c.s>>>(
          k, fn, (const T *)c.rho, c.solid, c.owner, c.surface, (const T *)c.qc, (const T *)c.phit, c.cx, c.cr, c.cv,
          c.cforce);
    else
      count_launch(), k_colloid_bb<S, T, 1><<<c.ncoll, B, 0, c.s>>>(
          k, fn, (const T *)c.rho, c.solid, c.owner, c.surface, (const T *)c.qc, (const T *)c.phit, c.cx, c.cr, c.cv,
          c.cforce);
  }
  static void remap(Ctx &c) {
    auto k = make_stepk<T>(c);
    S *f = (S *)c.f[c.cur];
    if (c.ncomp == 2)
      count_launch(), k_remap<S, T, 2><<<c.ncoll, B, 0, c.s>>>(k, f, c.solid, c.solid_old, c.owner, c.owner_old, c.cx,
                                                                c.cr, c.cv, c.cdp);
    else
      count_launch(), k_remap<S, T, 1><<<c.ncoll, B, 0, c.s>>>(k, f, c.solid, c.solid_old, c.owner, c.owner_old, c.cx,
                                                                c.cr, c.cv, c.cdp);
    if (c.nions) {
      T *n = (T *)c.n[c.ncur];
      count_launch(), k_remap_mark<T><<<c.ncoll, B, 0, c.s>>>(k, n, c.solid, c.solid_old, c.owner, c.cx, c.cr,
                                                               (T *)c.remap_share, c.remap_flag);
      count_launch(), k_remap_ions<T><<<grid_for(c.d.N, B), B, 0, c.s>>>(k, n, c.solid, c.solid_old,
                                                                          (const T *)c.remap_share, c.remap_flag);
    }
  }
  static PrecOps ops() {
    PrecOps o;
    o.remap = remap;
    o.init_eq = init_eq;
    o.init_f = init_f;
    o.get_f = get_f;
    o.get_rho = get_rho;
    o.macro = macro;
    o.virt = virt;
    o.collide = collide;
    o.np = np;
    o.obs_partials = obs_partials;
    o.colloid_bb = colloid_bb;
    return o;
  }
};

}  // namespace lbeh
