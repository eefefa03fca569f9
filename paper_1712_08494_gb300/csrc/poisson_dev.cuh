// Device side of the variable-permittivity Poisson solve (Sec. II.B eq.
// electric_potential, II.D): multigrid level descriptors, double-float
// arithmetic, red-black smoothing, transfer operators, the single-block tail
// cycle and the whole defect-correction solve of one system by one team of
// blocks.  Shared by the single-system solver and the batched step.
#pragma once

#include <cmath>

#include "internal.h"
#include "dfloat.cuh"

namespace lbeh {

constexpr long long kTailCells = 512;
constexpr size_t kTailSmem = 200 * 1024;
constexpr int kMaxLevels = 16;
constexpr int kNu = 2;  // pre- and post-smoothing sweeps

template <typename T> struct Level {
  int nx = 0, ny = 0, nz = 0;
  long long N = 0;
  int cf[3] = {0, 0, 0};  // coarsened along x, y, z relative to the finer level
  T h[3] = {T(1), T(1), T(1)};  // 1 / H_a^2
  T *k[3] = {nullptr, nullptr, nullptr};
  T *x = nullptr, *x2 = nullptr, *b = nullptr;
  const T *eps = nullptr;  // set: face coefficients (eps_i + eps_{i+a})/2 formed from eps, k unused
  bool rb = false;
  __host__ __device__ Dims dims() const { return Dims{nx, ny, nz, N}; }
};

// face coefficients k_a(i) (p: +a face) and k_a(i-a) (m) of a cell
template <typename T> struct Faces {
  T xp, xm, yp, ym, zp, zm;
};
template <typename T, typename I>
__device__ __forceinline__ Faces<T> faces(const Level<T> &L, I i, I ixp, I ixm, I iyp, I iym, I izp, I izm) {
  Faces<T> f;
  if (L.eps) {
    const T e = L.eps[i];
    f.xp = T(0.5) * (e + L.eps[ixp]);
    f.xm = T(0.5) * (L.eps[ixm] + e);
    f.yp = T(0.5) * (e + L.eps[iyp]);
    f.ym = T(0.5) * (L.eps[iym] + e);
    f.zp = T(0.5) * (e + L.eps[izp]);
    f.zm = T(0.5) * (L.eps[izm] + e);
  } else {
    f.xp = L.k[0][i];
    f.xm = L.k[0][ixm];
    f.yp = L.k[1][i];
    f.ym = L.k[1][iym];
    f.zp = L.k[2][i];
    f.zm = L.k[2][izm];
  }
  // an axis coarsened to a single cell carries no coupling
  if (L.nx == 1) f.xp = f.xm = T(0);
  if (L.ny == 1) f.yp = f.ym = T(0);
  if (L.nz == 1) f.zp = f.zm = T(0);
  return f;
}

template <typename T> struct Tail {
  int n = 0;
  Level<T> L[kMaxLevels];
};

__host__ __device__ inline DF df_split(double v) {
  const float h = float(v);
  return DF{h, float(v - double(h))};
}

// Relative residual sqrt(r2 / b2); zero for a vanishing right-hand side and
// NaN when either sum is not finite (a non-finite input must not pass as a
// vanishing right-hand side).
__host__ __device__ inline double rel_res(double r2, double b2) {
  if (!isfinite(r2) || !isfinite(b2)) return r2 + b2 + NAN;
  return b2 > 0.0 ? sqrt(r2 / b2) : 0.0;
}

// Device-side solver state.
struct PDev {
  double mean_q, mean_phi, bnorm2, rnorm2, relres, tol;
  DF mean_q_df, mean_phi_df;
  int iters, max_iter, cond, notconv;
  long long total_iters;
  int have_prev;  // phi_prev holds the solution of the previous step
  int zero;       // right-hand side vanishes: phi = 0
};


// ---------------------------------------------------------------- level operations
template <typename T>
__device__ __forceinline__ void stencil(const Dims &d, const Level<T> &L, long long i, int x, int y, int z,
                                        const T *__restrict__ xv, T &off, T &diag) {
  const long long ixp = site(d, wrapp(x, d.nx), y, z), ixm = site(d, wrapm(x, d.nx), y, z);
  const long long iyp = site(d, x, wrapp(y, d.ny), z), iym = site(d, x, wrapm(y, d.ny), z);
  const long long izp = site(d, x, y, wrapp(z, d.nz)), izm = site(d, x, y, wrapm(z, d.nz));
  const Faces<T> f = faces(L, i, ixp, ixm, iyp, iym, izp, izm);
  const T kxp = f.xp, kxm = f.xm, kyp = f.yp, kym = f.ym, kzp = f.zp, kzm = f.zm;
  off = L.h[0] * (kxp * xv[ixp] + kxm * xv[ixm]) + L.h[1] * (kyp * xv[iyp] + kym * xv[iym]) +
        L.h[2] * (kzp * xv[izp] + kzm * xv[izm]);
  diag = L.h[0] * (kxp + kxm) + L.h[1] * (kyp + kym) + L.h[2] * (kzp + kzm);
}

// 32-bit cell walks.  Levels hold fewer than 2^31 cells.  A thread visits the
// cells t0, t0 + dt, ... of a row-major range of rows of width w (w = nx for
// every cell of a level, nx/2 for one colour of a red-black level with nx
// even); its position (u, y, z) advances by the stride decomposed once, with
// no per-cell division, and the walk ends when z reaches nz.
struct Walk {
  int u, y, z, du, dy, dz, w, ny;
  __device__ __forceinline__ Walk(long long t0, long long dt, int w_, int ny_) : w(w_), ny(ny_) {
    const unsigned uw = unsigned(w_), uny = unsigned(ny_);
    unsigned r = unsigned(t0) / uw;
    u = int(unsigned(t0) - r * uw);
    y = int(r % uny);
    z = int(r / uny);
    r = unsigned(dt) / uw;
    du = int(unsigned(dt) - r * uw);
    dy = int(r % uny);
    dz = int(r / uny);
  }
  __device__ __forceinline__ void next() {
    u += du;
    int c = u >= w;
    if (c) u -= w;
    y += dy + c;
    c = y >= ny;
    if (c) y -= ny;
    z += dz + c;
  }
};

__device__ __forceinline__ unsigned site32(const Dims &d, int x, int y, int z) {
  return (unsigned(z) * unsigned(d.ny) + unsigned(y)) * unsigned(d.nx) + unsigned(x);
}

// Passes over levels of at least kPfCells cells stream arrays larger than the
// L2; there each thread asks the L2 for the cell kPf iterations ahead of the
// one it works on (prefetch.global.L2 is a hint: it loads nothing into
// registers), which keeps more DRAM requests in flight than the 32 resident
// warps per SM issue on their own.  Smaller levels stay in the L2, where the
// hints would only cost instructions.
constexpr int kPf = 4;
constexpr long long kPfCells = 1LL << 22;
__device__ __forceinline__ void pf_l2(const void *p) { asm volatile("prefetch.global.L2 [%0];" ::"l"(p)); }

// cell (x, y, z) and its six periodic neighbours as 32-bit indices
struct Nbr {
  unsigned i, xp, xm, yp, ym, zp, zm;
};
__device__ __forceinline__ Nbr nbr(const Dims &d, int x, int y, int z) {
  const unsigned nx = unsigned(d.nx), sz = nx * unsigned(d.ny), n = unsigned(d.N);
  Nbr c;
  c.i = site32(d, x, y, z);
  c.xp = x + 1 == d.nx ? c.i - (nx - 1) : c.i + 1;
  c.xm = x == 0 ? c.i + (nx - 1) : c.i - 1;
  c.yp = y + 1 == d.ny ? c.i - (sz - nx) : c.i + nx;
  c.ym = y == 0 ? c.i + (sz - nx) : c.i - nx;
  c.zp = z + 1 == d.nz ? c.i - (n - sz) : c.i + sz;
  c.zm = z == 0 ? c.i + (n - sz) : c.i - sz;
  return c;
}

// the level stencil at a cell given by its neighbour indices: the same
// arithmetic as stencil()
template <typename T>
__device__ __forceinline__ void stencil_n(const Level<T> &L, const Nbr &c, const T *__restrict__ xv, T &off,
                                          T &diag) {
  const Faces<T> f = faces(L, c.i, c.xp, c.xm, c.yp, c.ym, c.zp, c.zm);
  const T kxp = f.xp, kxm = f.xm, kyp = f.yp, kym = f.ym, kzp = f.zp, kzm = f.zm;
  off = L.h[0] * (kxp * xv[c.xp] + kxm * xv[c.xm]) + L.h[1] * (kyp * xv[c.yp] + kym * xv[c.ym]) +
        L.h[2] * (kzp * xv[c.zp] + kzm * xv[c.zm]);
  diag = L.h[0] * (kxp + kxm) + L.h[1] * (kyp + kym) + L.h[2] * (kzp + kzm);
}
template <typename T> __device__ __forceinline__ T diag_n(const Level<T> &L, const Nbr &c) {
  const Faces<T> f = faces(L, c.i, c.xp, c.xm, c.yp, c.ym, c.zp, c.zm);
  return L.h[0] * (f.xp + f.xm) + L.h[1] * (f.yp + f.ym) + L.h[2] * (f.zp + f.zm);
}

// Coarse face coefficient along axis AX of coarse cell (X, Y, Z).  Along a
// coarsened axis the flux between the centres of coarse cells X and X + 1
// crosses three fine faces in series: half of the face inside X (fine 2X |
// 2X+1), the shared face (2X+1 | 2X+2) and half of the face inside X + 1
// (2X+2 | 2X+3); their series conductance over the two fine spacings is
// 2 / (1/(2 k_in) + 1/k_shared + 1/(2 k_next)) -- the harmonic weighting that
// keeps a jump of the permittivity inside a coarse cell from passing as the
// arithmetic mean (fewer cycles on the colloid boxes).  Across the face the
// fine paths are averaged.  Along an axis that is not coarsened the coarse
// face is the fine face.  Axis indices are compile-time constants, so the
// small coordinate arrays stay in registers.
template <int AX, typename T>
__device__ __forceinline__ T coarse_coef(const Level<T> &F, const Level<T> &C, int X, int Y, int Z) {
  constexpr int B1 = (AX + 1) % 3, B2 = (AX + 2) % 3;
  const Dims f = F.dims();
  const int fn[3] = {f.nx, f.ny, f.nz};
  const int p[3] = {C.cf[0] ? 2 * X : X, C.cf[1] ? 2 * Y : Y, C.cf[2] ? 2 * Z : Z};
  // fine face coefficient along AX at fine cell q (face q | q + AX)
  auto kf = [&](const int (&q)[3]) -> T {
    const unsigned fi = site32(f, q[0], q[1], q[2]);
    if (F.eps) {
      int r[3] = {q[0], q[1], q[2]};
      r[AX] = r[AX] + 1 == fn[AX] ? 0 : r[AX] + 1;
      return T(0.5) * (F.eps[fi] + F.eps[site32(f, r[0], r[1], r[2])]);
    }
    return F.k[AX][fi];
  };
  T acc = T(0);
  int cnt = 0;
  for (int t1 = 0; t1 <= C.cf[B1]; ++t1)
    for (int t2 = 0; t2 <= C.cf[B2]; ++t2) {
      int q[3] = {p[0], p[1], p[2]};
      q[B1] += t1;
      q[B2] += t2;
      if (C.cf[AX]) {
        const int x0 = q[AX];
        const T k_in = kf(q);
        q[AX] = x0 + 1;
        const T k_sh = kf(q);
        q[AX] = x0 + 2 == fn[AX] ? 0 : x0 + 2;
        const T k_nx = kf(q);
        acc += T(2) / (T(0.5) / k_in + T(1) / k_sh + T(0.5) / k_nx);
      } else {
        acc += kf(q);
      }
      ++cnt;
    }
  return acc / T(cnt);
}

// Cell t (< N/2) of one colour, colour = (x + y + z) & 1.  Red-black levels
// have every extent even or equal to one; cells pair up along the first axis
// of even extent.
__device__ __forceinline__ long long rb_cell(const Dims &d, int color, long long t, int &x, int &y, int &z) {
  if ((d.nx & 1) == 0) {
    const unsigned hx = unsigned(d.nx / 2);
    const unsigned r = unsigned(t) / hx;
    const int xh = int(unsigned(t) - r * hx);
    z = int(r / unsigned(d.ny));
    y = int(r - unsigned(z) * unsigned(d.ny));
    x = 2 * xh + ((y + z + color) & 1);
  } else if ((d.ny & 1) == 0) {  // nx == 1
    const unsigned hy = unsigned(d.ny / 2);
    const unsigned r = unsigned(t) / hy;
    x = 0;
    z = int(r);
    y = 2 * int(unsigned(t) - r * hy) + ((z + color) & 1);
  } else {  // nx == ny == 1
    x = 0;
    y = 0;
    z = 2 * int(t) + (color & 1);
  }
  return site(d, x, y, z);
}

// one colour of a red-black sweep over the thread range t0, t0+dt, ... < N/2
template <typename T>
__device__ __forceinline__ void rb_range(const Level<T> &L, int color, long long t0, long long dt) {
  const Dims d = L.dims();
  if ((d.nx & 1) == 0) {  // pairs along x: the walk of rb_cell without divisions
    const bool pf = kPf && d.N >= kPfCells;
    Walk wp(t0 + kPf * dt, dt, d.nx / 2, d.ny);
    for (Walk w(t0, dt, d.nx / 2, d.ny); w.z < d.nz; w.next(), wp.next()) {
      if (pf && wp.z < d.nz) {
        const unsigned ip = site32(d, 2 * wp.u + ((wp.y + wp.z + color) & 1), wp.y, wp.z);
        pf_l2(L.x + ip);
        pf_l2(L.b + ip);
        if (L.eps) pf_l2(L.eps + ip);
      }
      const Nbr c = nbr(d, 2 * w.u + ((w.y + w.z + color) & 1), w.y, w.z);
      T off, diag;
      stencil_n(L, c, L.x, off, diag);
      L.x[c.i] = (off - L.b[c.i]) / diag;
    }
    return;
  }
  for (long long t = t0; t < d.N / 2; t += dt) {
    int x, y, z;
    const long long i = rb_cell(d, color, t, x, y, z);
    T off, diag;
    stencil(d, L, i, x, y, z, L.x, off, diag);
    L.x[i] = (off - L.b[i]) / diag;
  }
}

template <typename T>
__device__ __forceinline__ void jacobi_range(const Level<T> &L, T w, long long t0, long long dt) {
  const Dims d = L.dims();
  for (long long i = t0; i < d.N; i += dt) {
    int x, y, z;
    coords(d, i, x, y, z);
    T off, diag;
    stencil(d, L, i, x, y, z, L.x, off, diag);
    L.x2[i] = L.x[i] + w * ((off - L.b[i]) / diag - L.x[i]);
  }
}

// diagonal of the level operator at cell I
template <typename T> __device__ __forceinline__ T diag_at(const Level<T> &L, long long I, int X, int Y, int Z) {
  const Dims c = L.dims();
  const Faces<T> fc = faces(L, I, site(c, wrapp(X, c.nx), Y, Z), site(c, wrapm(X, c.nx), Y, Z),
                            site(c, X, wrapp(Y, c.ny), Z), site(c, X, wrapm(Y, c.ny), Z), site(c, X, Y, wrapp(Z, c.nz)),
                            site(c, X, Y, wrapm(Z, c.nz)));
  return L.h[0] * (fc.xp + fc.xm) + L.h[1] * (fc.yp + fc.ym) + L.h[2] * (fc.zp + fc.zm);
}

// coarse b(I) = mean over children of the fine residual (b - A x).  After a
// red-black sweep that ended with the black colour the residual vanishes on
// black cells (each was just solved exactly for its equation), so only the
// red children are evaluated.  The first half sweep on the coarse level
// starts from x = 0, which sets its red cells to -b/diag: that is done here.
template <typename T>
__device__ __forceinline__ void restrict_range(const Level<T> &F, const Level<T> &C, long long t0, long long dt) {
  const Dims f = F.dims(), c = C.dims();
  for (Walk w(t0, dt, c.nx, c.ny); w.z < c.nz; w.next()) {
    const int X = w.u, Y = w.y, Z = w.z;
    T acc = T(0);
    int cnt = 0;
    for (int tz = 0; tz <= C.cf[2]; ++tz)
      for (int ty = 0; ty <= C.cf[1]; ++ty)
        for (int tx = 0; tx <= C.cf[0]; ++tx) {
          const int x = C.cf[0] ? 2 * X + tx : X, y = C.cf[1] ? 2 * Y + ty : Y, z = C.cf[2] ? 2 * Z + tz : Z;
          ++cnt;
          if (F.rb && ((x + y + z) & 1)) continue;
          const Nbr n = nbr(f, x, y, z);
          T off, diag;
          stencil_n(F, n, F.x, off, diag);
          acc += F.b[n.i] - (off - diag * F.x[n.i]);
        }
    const T bI = acc / T(cnt);
    const Nbr nc = nbr(c, X, Y, Z);
    C.b[nc.i] = bI;
    if (C.rb && !((X + Y + Z) & 1)) C.x[nc.i] = -bI / diag_n(C, nc);
  }
}

// trilinear (cell-centred) prolongation and correction x_f += P x_c
template <typename T>
__device__ __forceinline__ void prolong_range(const Level<T> &F, const Level<T> &C, long long t0, long long dt) {
  const Dims f = F.dims(), c = C.dims();
  const int cd[3] = {c.nx, c.ny, c.nz};
  if (C.cf[0] && C.cf[1] && C.cf[2]) {
    // coarsened along every axis: weights 27/64, 9/64, 3/64, 1/64
    const unsigned cnx = unsigned(c.nx), cny = unsigned(c.ny), fnx = unsigned(f.nx), fny = unsigned(f.ny);
    const bool pf = kPf && f.N >= kPfCells;
    Walk wp(t0 + kPf * dt, dt, f.nx, f.ny);
    for (Walk w(t0, dt, f.nx, f.ny); w.z < f.nz; w.next(), wp.next()) {
      if (pf && wp.z < f.nz) pf_l2(F.x + site32(f, wp.u, wp.y, wp.z));
      const int x = w.u, y = w.y, z = w.z;
      const unsigned i = (unsigned(z) * fny + unsigned(y)) * fnx + unsigned(x);
      const int X0 = x >> 1, Y0 = y >> 1, Z0 = z >> 1;
      const int X1 = (x & 1) ? (X0 + 1 == c.nx ? 0 : X0 + 1) : (X0 == 0 ? c.nx - 1 : X0 - 1);
      const int Y1 = (y & 1) ? (Y0 + 1 == c.ny ? 0 : Y0 + 1) : (Y0 == 0 ? c.ny - 1 : Y0 - 1);
      const int Z1 = (z & 1) ? (Z0 + 1 == c.nz ? 0 : Z0 + 1) : (Z0 == 0 ? c.nz - 1 : Z0 - 1);
      // coarse row starts of the four (Y, Z) combinations
      const unsigned r00 = (unsigned(Z0) * cny + unsigned(Y0)) * cnx, r10 = (unsigned(Z0) * cny + unsigned(Y1)) * cnx;
      const unsigned r01 = (unsigned(Z1) * cny + unsigned(Y0)) * cnx, r11 = (unsigned(Z1) * cny + unsigned(Y1)) * cnx;
      const T *cx = C.x;
      const T v000 = cx[r00 + X0];
      const T v100 = cx[r00 + X1], v010 = cx[r10 + X0], v001 = cx[r01 + X0];
      const T v110 = cx[r10 + X1], v101 = cx[r01 + X1], v011 = cx[r11 + X0];
      const T v111 = cx[r11 + X1];
      F.x[i] += T(0.421875) * v000 + T(0.140625) * ((v100 + v010) + v001) + T(0.046875) * ((v110 + v101) + v011) +
                T(0.015625) * v111;
    }
    return;
  }
  for (long long i = t0; i < f.N; i += dt) {
    int x, y, z;
    coords(f, i, x, y, z);
    const int p[3] = {x, y, z};
    int I0[3], I1[3];
    T w0[3], w1[3];
    for (int a = 0; a < 3; ++a) {
      if (C.cf[a]) {
        const int I = p[a] >> 1;
        I0[a] = I;
        I1[a] = (p[a] & 1) ? (I + 1 == cd[a] ? 0 : I + 1) : (I == 0 ? cd[a] - 1 : I - 1);
        w0[a] = T(0.75);
        w1[a] = T(0.25);
      } else {
        I0[a] = I1[a] = p[a];
        w0[a] = T(1);
        w1[a] = T(0);
      }
    }
    T acc = T(0);
    for (int tz = 0; tz < 2; ++tz)
      for (int ty = 0; ty < 2; ++ty)
        for (int tx = 0; tx < 2; ++tx) {
          const T w = (tx ? w1[0] : w0[0]) * (ty ? w1[1] : w0[1]) * (tz ? w1[2] : w0[2]);
          if (w == T(0)) continue;
          acc += w * C.x[site(c, tx ? I1[0] : I0[0], ty ? I1[1] : I0[1], tz ? I1[2] : I0[2])];
        }
    F.x[i] += acc;
  }
}

// ---------------------------------------------------------------- single-block tail
template <typename T> __device__ void tail_smooth(const Level<T> &L, int sweeps) {
  for (int s = 0; s < sweeps; ++s) {
    if (L.rb) {
      rb_range(L, 0, threadIdx.x, blockDim.x);
      __syncthreads();
      rb_range(L, 1, threadIdx.x, blockDim.x);
      __syncthreads();
    } else {
      jacobi_range(L, T(0.8), threadIdx.x, blockDim.x);
      __syncthreads();
      for (long long i = threadIdx.x; i < L.N; i += blockDim.x) L.x[i] = L.x2[i];
      __syncthreads();
    }
  }
}

// Shared-memory bytes of the tail levels first..n-1 (three face arrays, x, b,
// and x2 where an axis is odd).
template <typename T> __host__ __device__ inline size_t tail_bytes(const Tail<T> &tl, int first) {
  size_t b = 0;
  for (int l = first; l < tl.n; ++l) b += size_t(tl.L[l].rb ? 5 : 6) * tl.L[l].N * sizeof(T);
  return b;
}

// V-cycle over levels first..n-1 of `tl` inside one block, with every level
// held in shared memory: face coefficients and the right-hand side of level
// `first` are loaded, the correction x of level `first` is written back.
// V-cycle over levels first..n-1 of lv inside one block, every level held in
// shared memory (descriptors included): face coefficients and the right-hand
// side of level `first` are loaded, its correction x is written back.
template <typename T>
__device__ void tail_vcycle(const Level<T> *__restrict__ lv, int n, int first, unsigned char *smem_raw, T *sh) {
  __shared__ Level<T> sl[kMaxLevels];
  if (threadIdx.x == 0) {
    T *p = reinterpret_cast<T *>(smem_raw);
    for (int l = first; l < n; ++l) {
      Level<T> L = lv[l];
      const long long m = L.N;
      for (int a = 0; a < 3; ++a) {
        L.k[a] = p;
        p += m;
      }
      L.x = p;
      p += m;
      L.b = p;
      p += m;
      if (!L.rb) {
        L.x2 = p;
        p += m;
      }
      L.eps = nullptr;
      sl[l] = L;
    }
  }
  __syncthreads();
  for (int l = first; l < n; ++l) {
    const Level<T> G = lv[l];
    const Level<T> S = sl[l];
    const Dims dg = G.dims();
    for (Walk w(threadIdx.x, blockDim.x, dg.nx, dg.ny); w.z < dg.nz; w.next()) {
      const Nbr c = nbr(dg, w.u, w.y, w.z);
      const unsigned i = c.i;
      if (G.eps) {
        const T e = G.eps[i];
        S.k[0][i] = T(0.5) * (e + G.eps[c.xp]);
        S.k[1][i] = T(0.5) * (e + G.eps[c.yp]);
        S.k[2][i] = T(0.5) * (e + G.eps[c.zp]);
      } else {
        for (int a = 0; a < 3; ++a) S.k[a][i] = G.k[a][i];
      }
      if (l == first) S.b[i] = G.b[i];
    }
  }
  __syncthreads();
  for (int l = first; l < n; ++l) {
    const Level<T> L = sl[l];
    if (l == n - 1) {
      // coarsest: mean-free right-hand side, fixed relaxation count
      T acc = T(0);
      for (long long i = threadIdx.x; i < L.N; i += blockDim.x) acc += L.b[i];
      sh[threadIdx.x] = acc;
      __syncthreads();
      for (int w = blockDim.x / 2; w > 0; w >>= 1) {
        if (threadIdx.x < w) sh[threadIdx.x] += sh[threadIdx.x + w];
        __syncthreads();
      }
      const T mean = sh[0] / T(L.N);
      __syncthreads();
      for (long long i = threadIdx.x; i < L.N; i += blockDim.x) {
        L.b[i] -= mean;
        L.x[i] = T(0);
      }
      __syncthreads();
      tail_smooth(L, L.rb ? 4 : 30);
    } else {
      for (long long i = threadIdx.x; i < L.N; i += blockDim.x) L.x[i] = T(0);
      __syncthreads();
      tail_smooth(L, kNu);
      const Level<T> Lc = sl[l + 1];
      restrict_range(L, Lc, threadIdx.x, blockDim.x);
      __syncthreads();
    }
  }
  for (int l = n - 2; l >= first; --l) {
    const Level<T> Lf = sl[l], Lc = sl[l + 1];
    prolong_range(Lf, Lc, threadIdx.x, blockDim.x);
    __syncthreads();
    tail_smooth(Lf, kNu);
  }
  {
    const Level<T> G = lv[first], S = sl[first];
    for (long long i = threadIdx.x; i < G.N; i += blockDim.x) G.x[i] = S.x[i];
  }
}

// ---------------------------------------------------------------- persistent solve
// The whole solve in one cooperative launch: initial guess, coefficients, the
// residual test and the defect-correction cycles, separated by grid-wide
// barriers.  Every block evaluates the same fixed-order sums, so all blocks
// take the same branches.  The barrier wait is bounded: a block that gives up
// raises an abort flag and the device status, and every block then returns.
constexpr int kPB = 512;
constexpr long long kSpinLimit = 1LL << 24;  // default polls of a barrier wait (~100 ns each: about two seconds)
constexpr double kTrustTol = 1e-8;  // FP32 residual estimate used only above this tolerance
constexpr double kEstErr = 1e-4;    // bound of its error relative to the last exact residual

struct Bar {
  unsigned long long arrived;  // monotonic arrival count (reset before each launch)
  int abort, pad;
};

__device__ __forceinline__ unsigned long long ld_acquire_u64(const unsigned long long *p) {
  unsigned long long v;
  asm volatile("ld.acquire.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ unsigned long long atom_add_acq_rel_u64(unsigned long long *p, unsigned long long v) {
  unsigned long long o;
  asm volatile("atom.add.acq_rel.gpu.global.u64 %0, [%1], %2;" : "=l"(o) : "l"(p), "l"(v) : "memory");
  return o;
}
__device__ __forceinline__ int ld_acquire_s32(const int *p) {
  int v;
  asm volatile("ld.acquire.gpu.global.s32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

// Grid barrier: thread 0 of every block arrives with an acquire-release add
// on a monotonic counter (releasing the block's writes, ordered by the
// preceding __syncthreads) and polls it with acquire loads until all blocks of
// this barrier generation have arrived.  The wait is bounded; on time-out the block raises
// the abort flag and the status, and every block leaves at its next barrier.
__device__ __forceinline__ bool grid_sync(Bar *bar, int *status, long long spin_limit) {
  __shared__ int ok;
  __syncthreads();
  if (threadIdx.x == 0) {
    const unsigned long long nb = gridDim.x;
    const unsigned long long old = atom_add_acq_rel_u64(&bar->arrived, 1ull);
    const unsigned long long target = (old / nb + 1) * nb;
    long long spins = 0;
    while (ld_acquire_u64(&bar->arrived) < target) {
      if (ld_acquire_s32(&bar->abort)) break;
      if (++spins > spin_limit) {
        atomicExch(&bar->abort, 1);
        atomicOr(status, ST_TIMEOUT);
        break;
      }
      __nanosleep(20);
    }
    ok = !ld_acquire_s32(&bar->abort);
  }
  __syncthreads();
  return ok != 0;
}


// A team is the set of blocks that solves one system: the whole grid of a
// cooperative launch (barrier on a global counter, bounded wait), or one
// thread-block cluster (hardware cluster barrier with release/acquire
// semantics, no polling).
struct GridTeam {
  Bar *bar;
  int *status;
  long long spin_limit;  // polls of a barrier wait before the solve gives up
  __device__ long long rank() const { return blockIdx.x * (long long)blockDim.x + threadIdx.x; }
  __device__ long long size() const { return (long long)gridDim.x * blockDim.x; }
  __device__ int block() const { return blockIdx.x; }
  __device__ int nblocks() const { return gridDim.x; }
  __device__ bool sync() const { return grid_sync(bar, status, spin_limit); }
};

struct ClusterTeam {
  unsigned crank, csize;
  __device__ ClusterTeam() {
    asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(crank));
    asm volatile("mov.u32 %0, %%cluster_nctarank;" : "=r"(csize));
  }
  __device__ long long rank() const { return (long long)crank * blockDim.x + threadIdx.x; }
  __device__ long long size() const { return (long long)csize * blockDim.x; }
  __device__ int block() const { return int(crank); }
  __device__ int nblocks() const { return int(csize); }
  __device__ bool sync() const {
    asm volatile("barrier.cluster.arrive.release;\n\tbarrier.cluster.wait.acquire;" ::: "memory");
    return true;
  }
};

template <typename T> struct PArgs {
  const Level<T> *lv;                          // level table in device memory
  int nlev;
  int tail;                                    // first level relaxed by block 0 in shared memory
  const T *eps, *q;
  double *phi, *prev;                          // FP64 potential (FP64 mode)
  float *phi_hi, *phi_lo, *prev_hi, *prev_lo;  // double-float potential (FP32 modes)
  DF edf[3];
  double ex, ey, ez;
  PDev *st;
  int *status;
  double *part;  // [3][blocks of the team]
  Bar *bar;
  long long spin_limit;  // polls of a grid-barrier wait before time-out (cooperative solve)
};

__device__ __forceinline__ double block_sum_n(double v, double *sh) {
  sh[threadIdx.x] = v;
  __syncthreads();
  for (int w = blockDim.x / 2; w > 0; w >>= 1) {
    if (threadIdx.x < w) sh[threadIdx.x] += sh[threadIdx.x + w];
    __syncthreads();
  }
  const double r = sh[0];
  __syncthreads();
  return r;
}

// fixed-order sum of nb partials, identical in every block
__device__ __forceinline__ double sum_partials(const double *part, int nb, double *sh) {
  double acc = 0.0;
  for (int b = threadIdx.x; b < nb; b += blockDim.x) acc += part[b];
  return block_sum_n(acc, sh);
}

template <typename T, bool DFM>
__device__ __forceinline__ void residual_site(const PArgs<T> &a, const Level<T> &L0, int x, int y, int z,
                                              double qbar, DF qbar_df, SumAcc<DFM> &ar, SumAcc<DFM> &ab,
                                              SumAcc<DFM> &ap) {
  const Nbr c = nbr(L0.dims(), x, y, z);
  const unsigned i = c.i, ixp = c.xp, ixm = c.xm, iyp = c.yp, iym = c.ym, izp = c.zp, izm = c.zm;
  const Faces<T> fc = faces(L0, i, ixp, ixm, iyp, iym, izp, izm);
  const T kxp = fc.xp, kxm = fc.xm, kyp = fc.yp, kym = fc.ym, kzp = fc.zp, kzm = fc.zm;
  if constexpr (DFM) {
    // sum_k k_k (phi_k - phi_i): exact differences of the high words
    // (two_sum) plus the differences of the low words, the high products
    // exact with their FMA error terms, high parts summed with compensation
    // (about 2^-46 of the largest flux term, as in general double-float
    // arithmetic, at less than half its operations)
    const float *hi = a.phi_hi, *lo = a.phi_lo;
    const float h0 = hi[i], l0 = lo[i];
    const unsigned nb[6] = {ixp, ixm, iyp, iym, izp, izm};
    const float kk[6] = {float(kxp), float(kxm), float(kyp), float(kym), float(kzp), float(kzm)};
    float ahi = 0.f, alo = 0.f;
#pragma unroll
    for (int k = 0; k < 6; ++k) {
      const DF dd = two_sum(hi[nb[k]], -h0);
      const float dlo = __fadd_rn(dd.lo, __fsub_rn(lo[nb[k]], l0));
      const float prod = __fmul_rn(dd.hi, kk[k]);
      const float plo = __fmaf_rn(dlo, kk[k], __fmaf_rn(dd.hi, kk[k], -prod));
      const DF t = two_sum(ahi, prod);
      ahi = t.hi;
      alo = __fadd_rn(alo, __fadd_rn(t.lo, plo));
    }
    DF b = two_sum(qbar_df.hi, -float(a.q[i]));
    b.lo = __fadd_rn(b.lo, qbar_df.lo);
    if (a.edf[0].hi != 0.f) b = df_add(b, df_mul(a.edf[0], two_sum(kxp, -kxm)));
    if (a.edf[1].hi != 0.f) b = df_add(b, df_mul(a.edf[1], two_sum(kyp, -kym)));
    if (a.edf[2].hi != 0.f) b = df_add(b, df_mul(a.edf[2], two_sum(kzp, -kzm)));
    const DF r = two_sum(b.hi, -ahi);
    const float rf = __fadd_rn(r.hi, __fadd_rn(r.lo, __fsub_rn(b.lo, alo)));
    L0.b[i] = T(rf);
    ar.add(rf * rf);
    ab.add(b.hi * b.hi);
    ap.add(h0);
  } else {
    const double *phi = a.phi;
    const double p = phi[i];
    double b = -(double(a.q[i]) - qbar);
    if (a.ex != 0.0) b += a.ex * (double(kxp) - double(kxm));
    if (a.ey != 0.0) b += a.ey * (double(kyp) - double(kym));
    if (a.ez != 0.0) b += a.ez * (double(kzp) - double(kzm));
    const double Ap = double(kxp) * (phi[ixp] - p) - double(kxm) * (p - phi[ixm]) + double(kyp) * (phi[iyp] - p) -
                      double(kym) * (p - phi[iym]) + double(kzp) * (phi[izp] - p) - double(kzm) * (p - phi[izm]);
    const double r = b - Ap;
    L0.b[i] = T(r);
    ar.add(r * r);
    ab.add(b * b);
    ap.add(p);
  }
}

// residual pass + fixed-order sums in every block; returns false on abort
template <typename T, bool DFM, class Team>
__device__ bool residual_pass(const PArgs<T> &a, const Team &tm, const Level<T> &L0, double qbar, DF qbar_df,
                              double *sh, double &r2, double &b2, double &ps, bool pf_always = false) {
  const long long G = tm.size();
  SumAcc<DFM> sr, sb, sp;
  const Dims d = L0.dims();
  const bool pf = kPf && (pf_always || d.N >= kPfCells);
  Walk wp(tm.rank() + kPf * G, G, L0.nx, L0.ny);
  for (Walk w(tm.rank(), G, L0.nx, L0.ny); w.z < L0.nz; w.next(), wp.next()) {
    if (pf && wp.z < d.nz) {
      const unsigned ip = site32(d, wp.u, wp.y, wp.z);
      if (L0.eps) pf_l2(L0.eps + ip);
      pf_l2(a.q + ip);
      if constexpr (DFM) {
        pf_l2(a.phi_hi + ip);
        pf_l2(a.phi_lo + ip);
      } else {
        pf_l2(a.phi + ip);
      }
    }
    residual_site<T, DFM>(a, L0, w.u, w.y, w.z, qbar, qbar_df, sr, sb, sp);
  }
  const double ar = block_sum_n(sr.get(), sh);
  const double ab = block_sum_n(sb.get(), sh);
  const double ap = block_sum_n(sp.get(), sh);
  const int nb = tm.nblocks();
  if (threadIdx.x == 0) {
    a.part[tm.block()] = ar;
    a.part[nb + tm.block()] = ab;
    a.part[2 * nb + tm.block()] = ap;
  }
  if (!tm.sync()) return false;
  r2 = sum_partials(a.part, nb, sh);
  b2 = sum_partials(a.part + nb, nb, sh);
  ps = sum_partials(a.part + 2 * nb, nb, sh);
  return true;
}

// The whole solve of one system by one team: initial guess, coefficients,
// the residual test and the defect-correction cycles, separated by team
// barriers.  Every block of the team evaluates the same fixed-order sums, so
// all blocks take the same branches.  smem_raw holds the tail levels, sh and
// sht kPB-element block scratch.
template <typename T, bool DFM, class Team>
__device__ void poisson_body(const PArgs<T> &a, const Team &tm, unsigned char *smem_raw, double *sh, T *sht) {
  const long long G = tm.size();
  const long long gt = tm.rank();
  const Level<T> L0 = a.lv[0];  // descriptors by value: stores cannot alias them
  const Dims d = L0.dims();
  const long long N = d.N;
  PDev *st = a.st;
  const int have_prev = st->have_prev;

  // initial guess, level-0 face coefficients, sum of q
  SumAcc<DFM> sq;
  for (long long i = gt; i < N; i += G) {
    if constexpr (DFM) {
      const DF p{a.phi_hi[i], a.phi_lo[i]};
      if (have_prev) {
        const DF g = df_sub(DF{2.f * p.hi, 2.f * p.lo}, DF{a.prev_hi[i], a.prev_lo[i]});
        a.phi_hi[i] = g.hi;
        a.phi_lo[i] = g.lo;
      }
      a.prev_hi[i] = p.hi;
      a.prev_lo[i] = p.lo;
    } else {
      const double p = a.phi[i];
      if (have_prev) a.phi[i] = 2.0 * p - a.prev[i];
      a.prev[i] = p;
    }
    if (!L0.eps) {
      int x, y, z;
      coords(d, i, x, y, z);
      const T e = a.eps[i];
      L0.k[0][i] = T(0.5) * (e + a.eps[site(d, wrapp(x, d.nx), y, z)]);
      L0.k[1][i] = T(0.5) * (e + a.eps[site(d, x, wrapp(y, d.ny), z)]);
      L0.k[2][i] = T(0.5) * (e + a.eps[site(d, x, y, wrapp(z, d.nz))]);
    }
    sq.add(a.q[i]);
  }
  const double accq = block_sum_n(sq.get(), sh);
  if (threadIdx.x == 0) a.part[tm.block()] = accq;
  if (!tm.sync()) return;
  const double qbar = sum_partials(a.part, tm.nblocks(), sh) / double(N);
  const DF qbar_df = df_split(qbar);
  // coarse face coefficients, level by level
  for (int l = 1; l < a.nlev; ++l) {
    const Level<T> F = a.lv[l - 1], C = a.lv[l];
    const Dims f = F.dims(), c = C.dims();
    for (Walk w(gt, G, c.nx, c.ny); w.z < c.nz; w.next()) {
      const unsigned I = site32(c, w.u, w.y, w.z);
      C.k[0][I] = coarse_coef<0>(F, C, w.u, w.y, w.z);
      C.k[1][I] = coarse_coef<1>(F, C, w.u, w.y, w.z);
      C.k[2][I] = coarse_coef<2>(F, C, w.u, w.y, w.z);
    }
    if (!tm.sync()) return;
  }
  // residual test
  double r2, b2, ps;
  if (!residual_pass<T, DFM>(a, tm, L0, qbar, qbar_df, sh, r2, b2, ps)) return;
  const double tol = st->tol;
  const int max_iter = st->max_iter;
  const double bn = b2;
  double rr = rel_res(r2, bn);
  int it = 0;
  // In the FP32 modes the level-0 residual is carried from cycle to cycle in
  // FP32 (r <- r - A e); that estimate is accurate to about 1e-5 of the
  // starting residual, so below kTrustTol the exact double-float residual
  // re-anchors it before convergence is accepted.
  bool exact = true;
  const bool carry = DFM && tol >= kTrustTol;
  double rr0 = rr;
  for (;;) {
  while (rr >= tol && it < max_iter) {
    exact = !carry;
    // V-cycle on the correction: levels above the tail, red-black smoothing
    for (int l = 0; l < a.tail; ++l) {
      const Level<T> Ll = a.lv[l];
      const Level<T> Lc = a.lv[l + 1];
      for (int s = 0; s < kNu; ++s) {
        // first red half sweep from x = 0: x = -b/diag, done by the
        // restriction that produced the right-hand side on coarse levels
        if (s > 0) {
          rb_range(Ll, 0, gt, G);
          if (!tm.sync()) return;
        } else if (l == 0) {
          const Dims dl = Ll.dims();
          if ((dl.nx & 1) == 0) {
            const bool pf = kPf && dl.N >= kPfCells;
            Walk wp(gt + kPf * G, G, dl.nx / 2, dl.ny);
            for (Walk w(gt, G, dl.nx / 2, dl.ny); w.z < dl.nz; w.next(), wp.next()) {
              if (pf && wp.z < dl.nz) {
                const unsigned ip = site32(dl, 2 * wp.u + ((wp.y + wp.z) & 1), wp.y, wp.z);
                pf_l2(Ll.b + ip);
                if (Ll.eps) pf_l2(Ll.eps + ip);
              }
              const Nbr c = nbr(dl, 2 * w.u + ((w.y + w.z) & 1), w.y, w.z);
              Ll.x[c.i] = -Ll.b[c.i] / diag_n(Ll, c);
            }
          } else {
            for (long long t = gt; t < Ll.N / 2; t += G) {
              int x, y, z;
              const long long i = rb_cell(dl, 0, t, x, y, z);
              Ll.x[i] = -Ll.b[i] / diag_at(Ll, i, x, y, z);
            }
          }
          if (!tm.sync()) return;
        }
        rb_range(Ll, 1, gt, G);
        if (!tm.sync()) return;
      }
      restrict_range(Ll, Lc, gt, G);
      if (!tm.sync()) return;
    }
    if (tm.block() == 0) tail_vcycle(a.lv, a.nlev, a.tail, smem_raw, sht);
    if (!tm.sync()) return;
    for (int l = a.tail - 1; l >= 0; --l) {
      const Level<T> Ll = a.lv[l];
      const Level<T> Lc = a.lv[l + 1];
      prolong_range(Ll, Lc, gt, G);
      if (!tm.sync()) return;
      for (int s = 0; s < kNu; ++s) {
        rb_range(Ll, 0, gt, G);
        if (!tm.sync()) return;
        rb_range(Ll, 1, gt, G);
        if (!tm.sync()) return;
      }
    }
    // phi += correction; the residual follows the correction
    if (carry) {
      // FP32 modes: r <- r - A e on the FP32 level-0 residual (its rounding error is
      // relative to |A e| ~ |r|), phi += e in double-float; the double-float residual
      // of the first pass fixes the starting point of each solve
      SumAcc<DFM> sr, sp;
      const bool pf = kPf && d.N >= kPfCells;
      Walk wp(gt + kPf * G, G, d.nx, d.ny);
      for (Walk w(gt, G, d.nx, d.ny); w.z < d.nz; w.next(), wp.next()) {
        if (pf && wp.z < d.nz) {
          const unsigned ip = site32(d, wp.u, wp.y, wp.z);
          pf_l2(L0.x + ip);
          pf_l2(L0.b + ip);
          if (L0.eps) pf_l2(L0.eps + ip);
          pf_l2(a.phi_hi + ip);
          pf_l2(a.phi_lo + ip);
        }
        const Nbr c = nbr(d, w.u, w.y, w.z);
        const unsigned i = c.i, ixp = c.xp, ixm = c.xm, iyp = c.yp, iym = c.ym, izp = c.zp, izm = c.zm;
        const T *e = L0.x;
        const T ei = e[i];
        const Faces<T> fc = faces(L0, i, ixp, ixm, iyp, iym, izp, izm);
        const T Ae = fc.xp * (e[ixp] - ei) + fc.xm * (e[ixm] - ei) + fc.yp * (e[iyp] - ei) + fc.ym * (e[iym] - ei) +
                     fc.zp * (e[izp] - ei) + fc.zm * (e[izm] - ei);
        // every cell, black ones included: after the black half sweep their
        // residual is zero only up to the FP32 rounding of the update, which
        // scales with the correction and must stay visible to later cycles
        const T r = L0.b[i] - Ae;
        L0.b[i] = r;
        sr.add(r * r);
        const DF s = df_add(DF{a.phi_hi[i], a.phi_lo[i]}, DF{float(ei), 0.f});
        a.phi_hi[i] = s.hi;
        a.phi_lo[i] = s.lo;
        sp.add(s.hi);
      }
      const double ar = block_sum_n(sr.get(), sh);
      const double ap = block_sum_n(sp.get(), sh);
      const int nb = tm.nblocks();
      if (threadIdx.x == 0) {
        a.part[tm.block()] = ar;
        a.part[2 * nb + tm.block()] = ap;
      }
      if (!tm.sync()) return;
      r2 = sum_partials(a.part, nb, sh);
      ps = sum_partials(a.part + 2 * nb, nb, sh);
    } else {
      for (long long i = gt; i < N; i += G) {
        if constexpr (DFM) {
          const DF s = df_add(DF{a.phi_hi[i], a.phi_lo[i]}, DF{float(L0.x[i]), 0.f});
          a.phi_hi[i] = s.hi;
          a.phi_lo[i] = s.lo;
        } else {
          a.phi[i] += double(L0.x[i]);
        }
      }
      if (!tm.sync()) return;
      if (!residual_pass<T, DFM>(a, tm, L0, qbar, qbar_df, sh, r2, b2, ps)) return;
    }
    rr = rel_res(r2, bn);
    ++it;
  }
  if (exact || rr + kEstErr * rr0 < tol) break;
  if (!residual_pass<T, DFM>(a, tm, L0, qbar, qbar_df, sh, r2, b2, ps)) return;
  rr = rel_res(r2, bn);
  rr0 = rr;
  exact = true;
  if (rr < tol || it >= max_iter) break;
  }
  const bool zero = bn == 0.0;
  const double mean_phi = ps / double(N);
  const DF mean_df = df_split(mean_phi);
  for (long long i = gt; i < N; i += G) {
    if constexpr (DFM) {
      DF v{0.f, 0.f};
      if (!zero) v = df_sub(DF{a.phi_hi[i], a.phi_lo[i]}, mean_df);
      a.phi_hi[i] = v.hi;
      a.phi_lo[i] = v.lo;
    } else {
      a.phi[i] = zero ? 0.0 : a.phi[i] - mean_phi;
    }
  }
  if (gt == 0) {
    st->mean_q = qbar;
    st->mean_phi = mean_phi;
    st->bnorm2 = bn;
    st->rnorm2 = r2;
    st->relres = rr;
    st->iters = it;
    st->total_iters += it;
    const int fail = !(rr < tol);  // not converged, or not finite
    st->notconv = fail;
    st->cond = 0;
    st->zero = zero;
    st->have_prev = 1;
    if (fail) atomicOr(a.status, ST_POISSON);
    if (!isfinite(rr)) atomicOr(a.status, ST_NONFINITE);
  }
}

}  // namespace lbeh
