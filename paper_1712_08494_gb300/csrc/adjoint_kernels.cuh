// Discrete adjoint of one coupled timestep (two fluid components, optional
// ions, no colloids), templated on the compute type T (populations stored in
// T).  Included once per precision mode (adjoint_f64.cu, adjoint_f32.cu).
//
// Forward step at site i (Sec. II), with the fields the forward kernels keep:
//   rho^s = sum_q f^s_q, J = sum_s sum_q f^s_q c_q, psi^s = 1 - exp(-rho^s),
//   eps(rho^a, rho^b), q = n+ - n-                                 (k_macro)
//   A(eps) phi = -(q - qbar) + sum_d eps_{i+d/2} E_ext.c_d           (Poisson)
//   E_i = -(phi_{i+a} - phi_{i-a})/2 + E_ext                          (field)
//   F^s_{i,a} = D[(n_{i+a} - n_i) - z_s (n_i + n_{i+a})/2 (E_{i,a} + E_{i+a,a})/2]
//   Fel_a = (eps_i - eps_bar)/4 (|E_{i+a}|^2 - |E_{i-a}|^2) - sum_s (F^s_{i,a} + F^s_{i-a,a})/(2D)
//   Phi^s = -G psi^s S^{s'} + (rho^s/rho) Fel,  S^s = sum_q w_q psi^s(i+c_q) c_q
//   u_e^s = J/rho + tau Phi^s/rho^s,  u = (J + (Phi^a + Phi^b)/2)/rho
//   f^s_q(i+c_q, t+1) = f^s_q + (feq_q(rho^s, u_e^s) - f^s_q)/tau
//   n^s(t+1) = n^s + sum_a (F_{i,a} - F_{i-a,a}) - upwind out + upwind in (u)
// The adjoint runs the transposes in reverse, every scatter written as a
// gather over the transposed stencil (no atomics):
//   ak_a  streaming + collision + velocity + Nernst-Planck advection + force
//         adjoints at the site; seeds the face, Kelvin and Shan-Chen scatters
//   ak_b  face-flux adjoints F-bar and the adjoint of the face field
//   ak_c  gathers: ion adjoint through the face fluxes, E-bar, psi-bar
//   ak_d  phi-bar = transpose of the central difference; right-hand side of
//         the adjoint Poisson problem A lambda = phi-bar - mean (A symmetric)
//   ak_e  Poisson sensitivities (q-bar = -lambda, face coefficients k-bar and
//         eps-bar), eps -> rho chain, and the final population adjoint
// Parameter derivatives (E_ext, G) are summed per block in FP64 and reduced
// in a fixed order.
#pragma once

#include "internal.h"

namespace lbeh {

template <typename T> struct AdjK {
  Dims d;
  int ions, field;
  T tau, G, D, eps_a, eps_b, eps_bar;
  T Eext[3];
};

template <typename T> struct AdjBufs {
  const T *f;      // forward populations at t [2][19][N]
  const T *n;      // forward ions at t [2][N]
  const T *rho, *J, *psi, *eps, *phi, *u, *flux;  // forward fields of step t
  const T *fbo;    // adjoint populations at t+1 [2][19][N]
  T *fbn;          // adjoint populations at t
  const T *nbo;    // adjoint ions at t+1 [2][N]
  T *nbn;          // adjoint ions at t
  T *rb;           // [2][N] rho-bar per component (total-density terms included)
  T *Jb;           // [3][N]
  T *Felb;         // [3][N]
  T *KC;           // [3][N] (eps_i - eps_bar)/4 Fel-bar
  T *Sb;           // [2][3][N] adjoint of S^a, S^b
  T *psib;         // [2][N] site-local psi-bar
  T *epsb;         // [N] site-local eps-bar
  T *Fb;           // [2][3][N] face-flux adjoints
  T *Efb;          // [3][N] adjoint of the face field (E_{i,a} + E_{i+a,a})/2
  T *Eb;           // [3][N] adjoint of E at the site
  T *qadj;         // [N] right-hand side "charge" of the adjoint Poisson problem (-phi-bar)
  const T *lam;    // [N] adjoint potential lambda
};

__device__ __forceinline__ void nb6(const Dims &d, long long i, long long jp[3], long long jm[3]) {
  int x, y, z;
  coords(d, i, x, y, z);
  jp[0] = site(d, wrapp(x, d.nx), y, z);
  jm[0] = site(d, wrapm(x, d.nx), y, z);
  jp[1] = site(d, x, wrapp(y, d.ny), z);
  jm[1] = site(d, x, wrapm(y, d.ny), z);
  jp[2] = site(d, x, y, wrapp(z, d.nz));
  jm[2] = site(d, x, y, wrapm(z, d.nz));
}

// E at site j (central difference of phi plus the applied field)
template <typename T>
__device__ __forceinline__ void efield(const AdjK<T> &k, const T *phi, long long j, T E[3]) {
  long long jp[3], jm[3];
  nb6(k.d, j, jp, jm);
#pragma unroll
  for (int a = 0; a < 3; ++a) E[a] = T(-0.5) * (phi[jp[a]] - phi[jm[a]]) + k.Eext[a];
}
template <typename T> __device__ __forceinline__ T efield_a(const AdjK<T> &k, const T *phi, long long j, int a) {
  long long jp[3], jm[3];
  nb6(k.d, j, jp, jm);
  return T(-0.5) * (phi[jp[a]] - phi[jm[a]]) + k.Eext[a];
}

__device__ __forceinline__ void block_partials(double v[kAdjPar], double *out) {
  __shared__ double sh[kAdjPar][256];
#pragma unroll
  for (int p = 0; p < kAdjPar; ++p) sh[p][threadIdx.x] = v[p];
  __syncthreads();
  for (int w = blockDim.x / 2; w > 0; w >>= 1) {
    if (threadIdx.x < w)
#pragma unroll
      for (int p = 0; p < kAdjPar; ++p) sh[p][threadIdx.x] += sh[p][threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x < kAdjPar) out[(size_t)blockIdx.x * kAdjPar + threadIdx.x] += sh[threadIdx.x][0];
}

// ------------------------------------------------------------------ ak_a
template <typename T, bool IONS>
__global__ void __launch_bounds__(256, 2) ak_a(AdjK<T> k, AdjBufs<T> B, double *part) {
  const Dims d = k.d;
  const long long N = d.N;
  double acc[kAdjPar] = {0, 0, 0, 0};
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < N; i += (long long)gridDim.x * blockDim.x) {
    int x, y, z;
    coords(d, i, x, y, z);
    long long nb[19];
    neighbours19(d, x, y, z, nb);
    const T rho[2] = {B.rho[i], B.rho[N + i]};
    const T rt = rho[0] + rho[1];
    const T inv_rho = rt > T(0) ? T(1) / rt : T(0);
    const T J[3] = {B.J[i], B.J[N + i], B.J[2 * N + i]};
    const T psi[2] = {B.psi[i], B.psi[N + i]};
    // forward forces
    T S[2][3] = {{T(0), T(0), T(0)}, {T(0), T(0), T(0)}};
    if (k.G != T(0)) {
#pragma unroll
      for (int q = 1; q < 19; ++q) {
        const T pa = wq<T>(q) * B.psi[nb[q]], pb = wq<T>(q) * B.psi[N + nb[q]];
        S[0][0] += T(cx(q)) * pa; S[0][1] += T(cy(q)) * pa; S[0][2] += T(cz(q)) * pa;
        S[1][0] += T(cx(q)) * pb; S[1][1] += T(cy(q)) * pb; S[1][2] += T(cz(q)) * pb;
      }
    }
    T Fel[3] = {T(0), T(0), T(0)}, K[3] = {T(0), T(0), T(0)};
    const T de = T(0.25) * (B.eps[i] - k.eps_bar);
    if (k.field) {
      // |E(i+a)|^2 - |E(i-a)|^2 (axis neighbours: nb[1..6] = +x -x +y -y +z -z)
#pragma unroll
      for (int a = 0; a < 3; ++a) {
        T Ep[3], Em[3];
        efield(k, B.phi, nb[1 + 2 * a], Ep);
        efield(k, B.phi, nb[2 + 2 * a], Em);
        K[a] = (Ep[0] * Ep[0] + Ep[1] * Ep[1] + Ep[2] * Ep[2]) - (Em[0] * Em[0] + Em[1] * Em[1] + Em[2] * Em[2]);
        Fel[a] = de * K[a];
      }
    }
    if (IONS) {
      const T inv_2D = T(0.5) / k.D;
#pragma unroll
      for (int a = 0; a < 3; ++a) {
        const long long jm = nb[2 + 2 * a];
        T tot = T(0);
#pragma unroll
        for (int s = 0; s < 2; ++s) tot += B.flux[(s * 3 + a) * N + i] + B.flux[(s * 3 + a) * N + jm];
        Fel[a] += -tot * inv_2D;
      }
    }
    T Phi[2][3];
#pragma unroll
    for (int s = 0; s < 2; ++s)
#pragma unroll
      for (int a = 0; a < 3; ++a) Phi[s][a] = -k.G * psi[s] * S[1 - s][a] + rho[s] * inv_rho * Fel[a];
    T ue[2][3];
#pragma unroll
    for (int s = 0; s < 2; ++s)
#pragma unroll
      for (int a = 0; a < 3; ++a) ue[s][a] = J[a] * inv_rho + (rho[s] > T(0) ? k.tau * Phi[s][a] / rho[s] : T(0));

    // streaming + collision adjoint
    T rb[2] = {T(0), T(0)}, rtb = T(0);
    T ueb[2][3] = {{T(0), T(0), T(0)}, {T(0), T(0), T(0)}};
    const T keep = T(1) - T(1) / k.tau, itau = T(1) / k.tau;
#pragma unroll
    for (int s = 0; s < 2; ++s) {
      const T usq = ue[s][0] * ue[s][0] + ue[s][1] * ue[s][1] + ue[s][2] * ue[s][2];
#pragma unroll
      for (int q = 0; q < 19; ++q) {
        const T fsb = B.fbo[(size_t)(s * 19 + q) * N + nb[q]];  // population sent to i + c_q
        B.fbn[(size_t)(s * 19 + q) * N + i] = keep * fsb;
        const T eb = fsb * itau;
        const T cu = T(cx(q)) * ue[s][0] + T(cy(q)) * ue[s][1] + T(cz(q)) * ue[s][2];
        rb[s] += eb * wq<T>(q) * (T(1) + T(3) * cu + T(4.5) * cu * cu - T(1.5) * usq);
        const T g = eb * wq<T>(q) * rho[s];
        const T gc = g * (T(3) + T(9) * cu);
        ueb[s][0] += gc * T(cx(q)) - T(3) * g * ue[s][0];
        ueb[s][1] += gc * T(cy(q)) - T(3) * g * ue[s][1];
        ueb[s][2] += gc * T(cz(q)) - T(3) * g * ue[s][2];
      }
    }
    // u_e = J/rho + tau Phi/rho^s
    T Jb[3] = {T(0), T(0), T(0)}, Phib[2][3];
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      const T sb = ueb[0][a] + ueb[1][a];
      Jb[a] += sb * inv_rho;
      rtb -= sb * J[a] * inv_rho * inv_rho;
    }
#pragma unroll
    for (int s = 0; s < 2; ++s) {
      const T ir = rho[s] > T(0) ? T(1) / rho[s] : T(0);
#pragma unroll
      for (int a = 0; a < 3; ++a) {
        Phib[s][a] = k.tau * ueb[s][a] * ir;
        rb[s] -= k.tau * ueb[s][a] * Phi[s][a] * ir * ir;
      }
    }
    // Nernst-Planck advection and the physical velocity
    if (IONS) {
      const T u[3] = {B.u[i], B.u[N + i], B.u[2 * N + i]};
      T ub[3] = {T(0), T(0), T(0)};
#pragma unroll
      for (int s = 0; s < 2; ++s) {
        const T nbi = B.nbo[s * N + i], ni = B.n[s * N + i];
        T out = nbi;
#pragma unroll
        for (int a = 0; a < 3; ++a) {
          const T nbp = B.nbo[s * N + nb[1 + 2 * a]], nbm = B.nbo[s * N + nb[2 + 2 * a]];
          const T ua = u[a];
          out += (ua > T(0) ? ua * (nbp - nbi) : T(0)) + (ua < T(0) ? -ua * (nbm - nbi) : T(0));
          ub[a] += ni * (ua > T(0) ? (nbp - nbi) : (ua < T(0) ? (nbi - nbm) : T(0)));
        }
        B.nbn[s * N + i] = out;
      }
      const T phys[3] = {(J[0] + T(0.5) * (Phi[0][0] + Phi[1][0])) * inv_rho,
                         (J[1] + T(0.5) * (Phi[0][1] + Phi[1][1])) * inv_rho,
                         (J[2] + T(0.5) * (Phi[0][2] + Phi[1][2])) * inv_rho};
#pragma unroll
      for (int a = 0; a < 3; ++a) {
        Jb[a] += ub[a] * inv_rho;
        Phib[0][a] += T(0.5) * ub[a] * inv_rho;
        Phib[1][a] += T(0.5) * ub[a] * inv_rho;
        rtb -= ub[a] * phys[a] * inv_rho;
      }
    }
    // Phi^s = -G psi^s S^{s'} + (rho^s/rho) Fel
    T Felb[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) Felb[a] = (Phib[0][a] * rho[0] + Phib[1][a] * rho[1]) * inv_rho;
    T psib[2] = {T(0), T(0)};
#pragma unroll
    for (int s = 0; s < 2; ++s) {
      T pf = T(0), psc = T(0);
#pragma unroll
      for (int a = 0; a < 3; ++a) {
        pf += Phib[s][a] * Fel[a];
        psc += Phib[s][a] * S[1 - s][a];
        B.Sb[((1 - s) * 3 + a) * N + i] = -k.G * psi[s] * Phib[s][a];
      }
      rb[s] += pf * inv_rho;
      rtb -= pf * rho[s] * inv_rho * inv_rho;
      psib[s] = -k.G * psc;
      acc[3] += -double(psi[s]) * double(psc);
    }
    T eb = T(0);
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      eb += T(0.25) * Felb[a] * K[a];
      B.KC[a * N + i] = de * Felb[a];
      B.Felb[a * N + i] = Felb[a];
      B.Jb[a * N + i] = Jb[a];
    }
    B.epsb[i] = eb;
#pragma unroll
    for (int s = 0; s < 2; ++s) {
      B.rb[s * N + i] = rb[s] + rtb;
      B.psib[s * N + i] = psib[s];
    }
  }
  block_partials(acc, part);
}

// ------------------------------------------------------------------ ak_b
template <typename T>
__global__ void __launch_bounds__(256) ak_b(AdjK<T> k, AdjBufs<T> B) {
  const long long N = k.d.N;
  long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (i >= N) return;
  long long jp[3], jm[3];
  nb6(k.d, i, jp, jm);
  const T inv_2D = T(0.5) / k.D;
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    const long long j = jp[a];
    const T fs = (B.Felb[a * N + i] + B.Felb[a * N + j]) * inv_2D;
    T efb = T(0);
#pragma unroll
    for (int s = 0; s < 2; ++s) {
      const T zs = s == 0 ? T(1) : T(-1);
      const T Fb = B.nbo[s * N + i] - B.nbo[s * N + j] - fs;
      B.Fb[(s * 3 + a) * N + i] = Fb;
      efb += -k.D * Fb * zs * T(0.5) * (B.n[s * N + i] + B.n[s * N + j]);
    }
    B.Efb[a * N + i] = k.field ? efb : T(0);
  }
}

// ------------------------------------------------------------------ ak_c
template <typename T, bool IONS>
__global__ void __launch_bounds__(256, 2) ak_c(AdjK<T> k, AdjBufs<T> B, double *part) {
  const Dims d = k.d;
  const long long N = d.N;
  double acc[kAdjPar] = {0, 0, 0, 0};
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < N; i += (long long)gridDim.x * blockDim.x) {
    int x, y, z;
    coords(d, i, x, y, z);
    long long nb[19];
    neighbours19(d, x, y, z, nb);
    T E[3] = {T(0), T(0), T(0)};
    if (k.field) efield(k, B.phi, i, E);
    T Eb[3] = {T(0), T(0), T(0)};
    if (IONS) {
      // ions through the face fluxes of faces (i, i+a) and (i-a, i)
      T Efp[3], Efm[3];
#pragma unroll
      for (int a = 0; a < 3; ++a) {
        if (k.field) {
          Efp[a] = T(0.5) * (E[a] + efield_a(k, B.phi, nb[1 + 2 * a], a));
          Efm[a] = T(0.5) * (efield_a(k, B.phi, nb[2 + 2 * a], a) + E[a]);
        } else {
          Efp[a] = Efm[a] = T(0);
        }
      }
#pragma unroll
      for (int s = 0; s < 2; ++s) {
        const T zs = s == 0 ? T(1) : T(-1);
        T add = T(0);
#pragma unroll
        for (int a = 0; a < 3; ++a) {
          const T Fbp = B.Fb[(s * 3 + a) * N + i], Fbm = B.Fb[(s * 3 + a) * N + nb[2 + 2 * a]];
          add += k.D * Fbp * (T(-1) - zs * T(0.5) * Efp[a]) + k.D * Fbm * (T(1) - zs * T(0.5) * Efm[a]);
        }
        B.nbn[s * N + i] += add;
      }
      if (k.field)
#pragma unroll
        for (int a = 0; a < 3; ++a) Eb[a] += T(0.5) * (B.Efb[a * N + i] + B.Efb[a * N + nb[2 + 2 * a]]);
    }
    if (k.field) {
      // Kelvin: E_i enters Fel_{i-a,a} with + and Fel_{i+a,a} with -
      T kc = T(0);
#pragma unroll
      for (int a = 0; a < 3; ++a) kc += B.KC[a * N + nb[2 + 2 * a]] - B.KC[a * N + nb[1 + 2 * a]];
#pragma unroll
      for (int b = 0; b < 3; ++b) Eb[b] += T(2) * E[b] * kc;
#pragma unroll
      for (int a = 0; a < 3; ++a) {
        B.Eb[a * N + i] = Eb[a];
        acc[a] += double(Eb[a]);
      }
    }
    // psi-bar: local part plus the transposed Shan-Chen sums, then rho-bar
#pragma unroll
    for (int s = 0; s < 2; ++s) {
      T pb = B.psib[s * N + i];
      if (k.G != T(0)) {
#pragma unroll
        for (int q = 1; q < 19; ++q) {
          const long long src = nb[opp(q)];  // i = src + c_q
          pb += wq<T>(q) * (T(cx(q)) * B.Sb[(s * 3 + 0) * N + src] + T(cy(q)) * B.Sb[(s * 3 + 1) * N + src] +
                            T(cz(q)) * B.Sb[(s * 3 + 2) * N + src]);
        }
      }
      B.rb[s * N + i] += pb * (T(1) - B.psi[s * N + i]);  // d psi / d rho = exp(-rho) = 1 - psi
    }
  }
  block_partials(acc, part);
}

// ------------------------------------------------------------------ ak_d
template <typename T> __global__ void __launch_bounds__(256) ak_d(AdjK<T> k, AdjBufs<T> B) {
  const long long N = k.d.N;
  long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (i >= N) return;
  long long jp[3], jm[3];
  nb6(k.d, i, jp, jm);
  T pb = T(0);
#pragma unroll
  for (int a = 0; a < 3; ++a) pb += T(0.5) * (B.Eb[a * N + jp[a]] - B.Eb[a * N + jm[a]]);
  B.qadj[i] = -pb;
}

// ------------------------------------------------------------------ ak_e
template <typename T, bool IONS>
__global__ void __launch_bounds__(256) ak_e(AdjK<T> k, AdjBufs<T> B, double *part) {
  const Dims d = k.d;
  const long long N = d.N;
  double acc[kAdjPar] = {0, 0, 0, 0};
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < N; i += (long long)gridDim.x * blockDim.x) {
    long long jp[3], jm[3];
    nb6(d, i, jp, jm);
    T rb[2] = {B.rb[i], B.rb[N + i]};
    if (k.field) {
      const T li = B.lam[i], pi = B.phi[i], ei = B.eps[i];
      T eb = B.epsb[i];
#pragma unroll
      for (int a = 0; a < 3; ++a) {
        const T lp = B.lam[jp[a]], lm = B.lam[jm[a]];
        const T pp = B.phi[jp[a]], pm = B.phi[jm[a]];
        const T kp = T(0.5) * (ei + B.eps[jp[a]]), km = T(0.5) * (B.eps[jm[a]] + ei);
        const T kbp = (li - lp) * (k.Eext[a] - pp + pi);
        const T kbm = (lm - li) * (k.Eext[a] - pi + pm);
        eb += T(0.5) * (kbp + kbm);
        acc[a] += double(li) * (double(kp) - double(km));
      }
      if (IONS) {
        B.nbn[i] -= li;
        B.nbn[N + i] += li;
      }
      // eps = (eps_a (1 - c) + eps_b (1 + c))/2,  c = (rho_b - rho_a)/(rho_a + rho_b)
      const T ra = B.rho[i], rbb = B.rho[N + i], rt = ra + rbb;
      if (rt > T(0)) {
        const T dedc = T(0.5) * (k.eps_b - k.eps_a), ir2 = T(1) / (rt * rt);
        rb[0] += eb * dedc * (T(-2) * rbb * ir2);
        rb[1] += eb * dedc * (T(2) * ra * ir2);
      }
    }
    const T Jb[3] = {B.Jb[i], B.Jb[N + i], B.Jb[2 * N + i]};
#pragma unroll
    for (int s = 0; s < 2; ++s)
#pragma unroll
      for (int q = 0; q < 19; ++q) {
        const size_t o = (size_t)(s * 19 + q) * N + i;
        B.fbn[o] += rb[s] + T(cx(q)) * Jb[0] + T(cy(q)) * Jb[1] + T(cz(q)) * Jb[2];
      }
  }
  block_partials(acc, part);
}

// ------------------------------------------------------------------ seeds
// Adjoint of the drop deformation D = (b - a)/(b + a), a = sqrt(M_xx),
// b = sqrt(M_zz), M = second moments of w = max(c, 0) about its centroid:
// dD/dw_i = -b (x - X)^2 / (a (a+b)^2) + a (z - Z)^2 / (b (a+b)^2), then
// through c = (rho_b - rho_a)/(rho_a + rho_b) to every population.
template <typename T>
__global__ void __launch_bounds__(256) ak_seed(AdjK<T> k, const T *__restrict__ f, T *__restrict__ fb, double X,
                                               double Z, double a, double b, double scale) {
  const Dims d = k.d;
  const long long N = d.N;
  long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (i >= N) return;
  double r[2] = {0.0, 0.0};
  for (int s = 0; s < 2; ++s)
    for (int q = 0; q < 19; ++q) r[s] += double(f[(size_t)(s * 19 + q) * N + i]);
  const double rt = r[0] + r[1];
  double g[2] = {0.0, 0.0};
  if (rt > 0.0 && (r[1] - r[0]) > 0.0 && a > 0.0 && b > 0.0) {
    int x, y, z;
    coords(d, i, x, y, z);
    const double ab2 = (a + b) * (a + b);
    const double dw = -b * (x - X) * (x - X) / (a * ab2) + a * (z - Z) * (z - Z) / (b * ab2);
    g[0] = scale * dw * (-2.0 * r[1] / (rt * rt));
    g[1] = scale * dw * (2.0 * r[0] / (rt * rt));
  }
  for (int s = 0; s < 2; ++s)
    for (int q = 0; q < 19; ++q) fb[(size_t)(s * 19 + q) * N + i] += T(g[s]);
}

// ------------------------------------------------------------------ host launchers
template <typename T> struct AdjLaunch {
  static AdjK<T> make(const Ctx &c) {
    AdjK<T> k;
    k.d = c.d;
    k.ions = c.nions > 0;
    k.field = c.has_field;
    k.tau = T(c.tau);
    k.G = T(c.G);
    k.D = T(c.D > 0 ? c.D : 1.0);
    k.eps_a = T(c.eps_a);
    k.eps_b = T(c.eps_b);
    k.eps_bar = T(c.eps_bar);
    for (int a = 0; a < 3; ++a) k.Eext[a] = T(c.Eext[a]);
    return k;
  }
  static AdjBufs<T> bufs(const AdjArgs &a) {
    AdjBufs<T> B;
    B.f = (const T *)a.f;
    B.n = (const T *)a.n;
    B.rho = (const T *)a.rho;
    B.J = (const T *)a.J;
    B.psi = (const T *)a.psi;
    B.eps = (const T *)a.eps;
    B.phi = (const T *)a.phi;
    B.u = (const T *)a.u;
    B.flux = (const T *)a.flux;
    B.fbo = (const T *)a.fbo;
    B.fbn = (T *)a.fbn;
    B.nbo = (const T *)a.nbo;
    B.nbn = (T *)a.nbn;
    B.rb = (T *)a.rb;
    B.Jb = (T *)a.Jb;
    B.Felb = (T *)a.Felb;
    B.KC = (T *)a.KC;
    B.Sb = (T *)a.Sb;
    B.psib = (T *)a.psib;
    B.epsb = (T *)a.epsb;
    B.Fb = (T *)a.Fb;
    B.Efb = (T *)a.Efb;
    B.Eb = (T *)a.Eb;
    B.qadj = (T *)a.qadj;
    B.lam = (const T *)a.lam;
    return B;
  }
  // passes a-d of one reversed step (the adjoint Poisson right-hand side in qadj)
  static void before_solve(const Ctx &c, const AdjArgs &a, double *part) {
    const AdjK<T> k = make(c);
    const AdjBufs<T> B = bufs(a);
    const long long N = c.d.N;
    if (c.nions) {
      count_launch(), ak_a<T, true><<<kAdjBlocks, 256, 0, c.s>>>(k, B, part);
      count_launch(), ak_b<T><<<grid_for(N, 256), 256, 0, c.s>>>(k, B);
      count_launch(), ak_c<T, true><<<kAdjBlocks, 256, 0, c.s>>>(k, B, part);
    } else {
      count_launch(), ak_a<T, false><<<kAdjBlocks, 256, 0, c.s>>>(k, B, part);
      count_launch(), ak_c<T, false><<<kAdjBlocks, 256, 0, c.s>>>(k, B, part);
    }
    if (c.has_field) count_launch(), ak_d<T><<<grid_for(N, 256), 256, 0, c.s>>>(k, B);
  }
  static void after_solve(const Ctx &c, const AdjArgs &a, double *part) {
    const AdjK<T> k = make(c);
    const AdjBufs<T> B = bufs(a);
    if (c.nions)
      count_launch(), ak_e<T, true><<<kAdjBlocks, 256, 0, c.s>>>(k, B, part);
    else
      count_launch(), ak_e<T, false><<<kAdjBlocks, 256, 0, c.s>>>(k, B, part);
  }
  static void seed(const Ctx &c, const void *f, void *fb, const double mom[4], double scale) {
    const AdjK<T> k = make(c);
    count_launch(), ak_seed<T><<<grid_for(c.d.N, 256), 256, 0, c.s>>>(k, (const T *)f, (T *)fb, mom[0], mom[1],
                                                                       mom[2], mom[3], scale);
  }
  static AdjOps ops() {
    AdjOps o;
    o.before_solve = before_solve;
    o.after_solve = after_solve;
    o.seed = seed;
    o.elem = sizeof(T);
    return o;
  }
};

}  // namespace lbeh
