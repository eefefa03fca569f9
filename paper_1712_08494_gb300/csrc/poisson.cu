// Variable-permittivity Poisson solve (Sec. II.B eq. electric_potential, II.D).
//
// Discrete problem (periodic, seven-point flux form, written for the total
// potential phi_I - E_ext.x so that the applied field polarises eps):
//   sum_{d in Q6} k_{i+d/2} (phi_{i+d} - phi_i) = b_i,
//   b = -(q - qbar) + sum_{d in Q6} k_{i+d/2} (E_ext.c_d),  k_{i+d/2} = (eps_i + eps_{i+d})/2,
// with mean(phi) = 0.  The paper inverts the constant-coefficient part by FFT
// and lags the variable part; here the same equation is solved to a residual
// tolerance by geometric multigrid used as a defect-correction iteration:
// the residual b - A phi is formed in FP64 against the FP64 potential, a
// V(2,2) cycle in the compute type (FP32 or FP64) approximates the
// correction, and phi is updated in FP64.  Cell-centred grids: coarse face
// coefficients are means of the fine faces they cover, restriction averages
// the children, prolongation is trilinear, smoothing is red-black
// Gauss-Seidel (damped Jacobi where an axis is odd), and the coarsest grid is
// relaxed by one thread block.
#include <cmath>
#include <utility>
#include <vector>

#include "internal.h"

namespace lbeh {

template <typename T> struct Level {
  int nx = 0, ny = 0, nz = 0;
  long long N = 0;
  int cf[3] = {0, 0, 0};  // coarsened along x, y, z relative to the finer level
  T h[3] = {T(1), T(1), T(1)};  // 1 / H_a^2
  T *k[3] = {nullptr, nullptr, nullptr};
  T *x = nullptr, *x2 = nullptr, *b = nullptr;
  bool rb = false;
  __host__ __device__ Dims dims() const { return Dims{nx, ny, nz, N}; }
};

struct Poisson {
  int fp64 = 0;
  std::vector<Level<double>> Ld;
  std::vector<Level<float>> Lf;
  double *b0 = nullptr;       // FP64 right-hand side
  double *part = nullptr;     // reduction partials (+ result slot)
  std::vector<void *> allocs;
};

// ---------------------------------------------------------------- kernels
template <typename T>
__global__ void k_coef0(Dims d, const T *__restrict__ eps, T *__restrict__ kx, T *__restrict__ ky,
                        T *__restrict__ kz) {
  long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (i >= d.N) return;
  int x, y, z;
  coords(d, i, x, y, z);
  const T e = eps[i];
  kx[i] = T(0.5) * (e + eps[site(d, wrapp(x, d.nx), y, z)]);
  ky[i] = T(0.5) * (e + eps[site(d, x, wrapp(y, d.ny), z)]);
  kz[i] = T(0.5) * (e + eps[site(d, x, y, wrapp(z, d.nz))]);
}

// coarse face (I + a/2) covers the fine faces (2I+1 + a/2) along a, averaged
// over the transverse children
template <typename T>
__global__ void k_coef_coarsen(Dims f, Dims c, int cfx, int cfy, int cfz, const T *__restrict__ fk0,
                               const T *__restrict__ fk1, const T *__restrict__ fk2, T *__restrict__ ck0,
                               T *__restrict__ ck1, T *__restrict__ ck2) {
  long long I = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (I >= c.N) return;
  int X, Y, Z;
  coords(c, I, X, Y, Z);
  const int cf[3] = {cfx, cfy, cfz};
  const int base[3] = {cfx ? 2 * X : X, cfy ? 2 * Y : Y, cfz ? 2 * Z : Z};
  const T *fk[3] = {fk0, fk1, fk2};
  T *ck[3] = {ck0, ck1, ck2};
  for (int a = 0; a < 3; ++a) {
    T acc = T(0);
    int cnt = 0;
    // along a: the last fine cell of the coarse cell; transverse: all children
    const int ra = cf[a] ? 1 : 0;
    const int b1 = (a + 1) % 3, b2 = (a + 2) % 3;
    for (int t1 = 0; t1 <= cf[b1]; ++t1)
      for (int t2 = 0; t2 <= cf[b2]; ++t2) {
        int p[3];
        p[a] = base[a] + ra;
        p[b1] = base[b1] + t1;
        p[b2] = base[b2] + t2;
        acc += fk[a][site(f, p[0], p[1], p[2])];
        ++cnt;
      }
    ck[a][I] = acc / T(cnt);
  }
}

template <typename T>
__device__ __forceinline__ void stencil(const Dims &d, const Level<T> &L, long long i, int x, int y, int z,
                                        const T *__restrict__ xv, T &off, T &diag) {
  const long long ixp = site(d, wrapp(x, d.nx), y, z), ixm = site(d, wrapm(x, d.nx), y, z);
  const long long iyp = site(d, x, wrapp(y, d.ny), z), iym = site(d, x, wrapm(y, d.ny), z);
  const long long izp = site(d, x, y, wrapp(z, d.nz)), izm = site(d, x, y, wrapm(z, d.nz));
  const T kxp = L.k[0][i], kxm = L.k[0][ixm];
  const T kyp = L.k[1][i], kym = L.k[1][iym];
  const T kzp = L.k[2][i], kzm = L.k[2][izm];
  off = L.h[0] * (kxp * xv[ixp] + kxm * xv[ixm]) + L.h[1] * (kyp * xv[iyp] + kym * xv[iym]) +
        L.h[2] * (kzp * xv[izp] + kzm * xv[izm]);
  diag = L.h[0] * (kxp + kxm) + L.h[1] * (kyp + kym) + L.h[2] * (kzp + kzm);
}

// red-black Gauss-Seidel half sweep; `zero` treats the current iterate as 0
template <typename T> __global__ void k_rb(Level<T> L, int color, int zero) {
  const Dims d = L.dims();
  long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (t >= d.N / 2) return;
  const int hx = d.nx / 2;
  long long r = t / hx;
  const int xh = int(t - r * hx);
  const int z = int(r / d.ny);
  const int y = int(r - (long long)z * d.ny);
  const int x = 2 * xh + ((y + z + color) & 1);
  const long long i = site(d, x, y, z);
  if (zero) {
    // first sweep from x = 0: red nodes see zero neighbours
    const long long ixm = site(d, wrapm(x, d.nx), y, z), iym = site(d, x, wrapm(y, d.ny), z),
                    izm = site(d, x, y, wrapm(z, d.nz));
    const T diag = L.h[0] * (L.k[0][i] + L.k[0][ixm]) + L.h[1] * (L.k[1][i] + L.k[1][iym]) +
                   L.h[2] * (L.k[2][i] + L.k[2][izm]);
    L.x[i] = -L.b[i] / diag;
    return;
  }
  T off, diag;
  stencil(d, L, i, x, y, z, L.x, off, diag);
  L.x[i] = (off - L.b[i]) / diag;
}

template <typename T> __global__ void k_zero(T *p, long long n) {
  long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (i < n) p[i] = T(0);
}

// damped Jacobi: x2 = x + w ((off - b)/diag - x)
template <typename T> __global__ void k_jacobi(Level<T> L, T w) {
  const Dims d = L.dims();
  long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (i >= d.N) return;
  int x, y, z;
  coords(d, i, x, y, z);
  T off, diag;
  stencil(d, L, i, x, y, z, L.x, off, diag);
  L.x2[i] = L.x[i] + w * ((off - L.b[i]) / diag - L.x[i]);
}

// fused residual + restriction: coarse b(I) = mean over children of (b - A x)
template <typename T> __global__ void k_restrict(Level<T> F, Level<T> C) {
  const Dims f = F.dims(), c = C.dims();
  long long I = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (I >= c.N) return;
  int X, Y, Z;
  coords(c, I, X, Y, Z);
  T acc = T(0);
  int cnt = 0;
  for (int tz = 0; tz <= C.cf[2]; ++tz)
    for (int ty = 0; ty <= C.cf[1]; ++ty)
      for (int tx = 0; tx <= C.cf[0]; ++tx) {
        const int x = C.cf[0] ? 2 * X + tx : X, y = C.cf[1] ? 2 * Y + ty : Y, z = C.cf[2] ? 2 * Z + tz : Z;
        const long long i = site(f, x, y, z);
        T off, diag;
        stencil(f, F, i, x, y, z, F.x, off, diag);
        acc += F.b[i] - (off - diag * F.x[i]);
        ++cnt;
      }
  C.b[I] = acc / T(cnt);
}

// trilinear (cell-centred) prolongation and correction x_f += P x_c
template <typename T> __global__ void k_prolong(Level<T> F, Level<T> C) {
  const Dims f = F.dims(), c = C.dims();
  long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (i >= f.N) return;
  int x, y, z;
  coords(f, i, x, y, z);
  const int p[3] = {x, y, z};
  const int cd[3] = {c.nx, c.ny, c.nz};
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

// coarsest grid: one block, mean-free right-hand side, fixed relaxation count
template <typename T> __global__ void __launch_bounds__(1024) k_coarsest(Level<T> L, int iters) {
  const Dims d = L.dims();
  __shared__ T sh[1024];
  T acc = T(0);
  for (long long i = threadIdx.x; i < d.N; i += blockDim.x) acc += L.b[i];
  sh[threadIdx.x] = acc;
  __syncthreads();
  for (int w = blockDim.x / 2; w > 0; w >>= 1) {
    if (threadIdx.x < w) sh[threadIdx.x] += sh[threadIdx.x + w];
    __syncthreads();
  }
  const T mean = sh[0] / T(d.N);
  __syncthreads();
  for (long long i = threadIdx.x; i < d.N; i += blockDim.x) {
    L.b[i] -= mean;
    L.x[i] = T(0);
  }
  __syncthreads();
  for (int it = 0; it < iters; ++it) {
    if (L.rb) {
      for (int color = 0; color < 2; ++color) {
        for (long long i = threadIdx.x; i < d.N; i += blockDim.x) {
          int x, y, z;
          coords(d, i, x, y, z);
          if (((x + y + z) & 1) != color) continue;
          T off, diag;
          stencil(d, L, i, x, y, z, L.x, off, diag);
          L.x[i] = (off - L.b[i]) / diag;
        }
        __syncthreads();
      }
    } else {
      for (long long i = threadIdx.x; i < d.N; i += blockDim.x) {
        int x, y, z;
        coords(d, i, x, y, z);
        T off, diag;
        stencil(d, L, i, x, y, z, L.x, off, diag);
        L.x2[i] = L.x[i] + T(0.8) * ((off - L.b[i]) / diag - L.x[i]);
      }
      __syncthreads();
      for (long long i = threadIdx.x; i < d.N; i += blockDim.x) L.x[i] = L.x2[i];
      __syncthreads();
    }
  }
}

// b0 = -q + sum_d k (E_ext.c_d)   (the mean of q is removed afterwards)
template <typename T>
__global__ void k_rhs(Dims d, const T *__restrict__ q, const T *__restrict__ kx, const T *__restrict__ ky,
                      const T *__restrict__ kz, double ex, double ey, double ez, double *__restrict__ b0) {
  long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (i >= d.N) return;
  int x, y, z;
  coords(d, i, x, y, z);
  double src = 0.0;
  if (ex != 0.0) src += ex * (double(kx[i]) - double(kx[site(d, wrapm(x, d.nx), y, z)]));
  if (ey != 0.0) src += ey * (double(ky[i]) - double(ky[site(d, x, wrapm(y, d.ny), z)]));
  if (ez != 0.0) src += ez * (double(kz[i]) - double(kz[site(d, x, y, wrapm(z, d.nz))]));
  b0[i] = -double(q[i]) + src;
}

__global__ void k_add_const(double *__restrict__ a, long long n, const double *__restrict__ sum, double scale) {
  long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (i < n) a[i] -= sum[0] * scale;
}

// FP64 residual r0 = b0 - A phi; r (compute type) = r0; per-block partials of r0^2
template <typename T>
__global__ void __launch_bounds__(256) k_residual0(Level<T> L, const double *__restrict__ phi,
                                                   const double *__restrict__ b0, double *__restrict__ part) {
  const Dims d = L.dims();
  __shared__ double sh[256];
  double acc = 0.0;
  for (long long i = blockIdx.x * 256LL + threadIdx.x; i < d.N; i += (long long)gridDim.x * 256) {
    int x, y, z;
    coords(d, i, x, y, z);
    const long long ixp = site(d, wrapp(x, d.nx), y, z), ixm = site(d, wrapm(x, d.nx), y, z);
    const long long iyp = site(d, x, wrapp(y, d.ny), z), iym = site(d, x, wrapm(y, d.ny), z);
    const long long izp = site(d, x, y, wrapp(z, d.nz)), izm = site(d, x, y, wrapm(z, d.nz));
    const double p = phi[i];
    const double Ap = double(L.k[0][i]) * (phi[ixp] - p) - double(L.k[0][ixm]) * (p - phi[ixm]) +
                      double(L.k[1][i]) * (phi[iyp] - p) - double(L.k[1][iym]) * (p - phi[iym]) +
                      double(L.k[2][i]) * (phi[izp] - p) - double(L.k[2][izm]) * (p - phi[izm]);
    const double r = b0[i] - Ap;
    L.b[i] = T(r);
    acc += r * r;
  }
  sh[threadIdx.x] = acc;
  __syncthreads();
  for (int w = 128; w > 0; w >>= 1) {
    if (threadIdx.x < w) sh[threadIdx.x] += sh[threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x == 0) part[blockIdx.x] = sh[0];
}

template <typename T>
__global__ void k_update_phi(double *__restrict__ phi, const T *__restrict__ x, long long n) {
  long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (i < n) phi[i] += double(x[i]);
}

__global__ void k_zero_d(double *p, long long n) {
  long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (i < n) p[i] = 0.0;
}

// ---------------------------------------------------------------- host
template <typename T> static std::vector<Level<T>> &levels(Poisson *p);
template <> std::vector<Level<double>> &levels<double>(Poisson *p) { return p->Ld; }
template <> std::vector<Level<float>> &levels<float>(Poisson *p) { return p->Lf; }

template <typename T> static T *alloc(Poisson *p, long long n) {
  void *ptr = nullptr;
  if (cudaMalloc(&ptr, n * sizeof(T)) != cudaSuccess) return nullptr;
  p->allocs.push_back(ptr);
  return (T *)ptr;
}

template <typename T> static bool setup(Poisson *p, const Dims &d) {
  auto &L = levels<T>(p);
  Level<T> l0;
  l0.nx = d.nx;
  l0.ny = d.ny;
  l0.nz = d.nz;
  l0.N = d.N;
  L.push_back(l0);
  while (true) {
    const Level<T> &f = L.back();
    int cf[3] = {f.nx % 2 == 0 && f.nx >= 4, f.ny % 2 == 0 && f.ny >= 4, f.nz % 2 == 0 && f.nz >= 4};
    if (!(cf[0] || cf[1] || cf[2]) || f.N <= 64) break;
    Level<T> c;
    c.nx = cf[0] ? f.nx / 2 : f.nx;
    c.ny = cf[1] ? f.ny / 2 : f.ny;
    c.nz = cf[2] ? f.nz / 2 : f.nz;
    c.N = (long long)c.nx * c.ny * c.nz;
    for (int a = 0; a < 3; ++a) {
      c.cf[a] = cf[a];
      c.h[a] = cf[a] ? f.h[a] * T(0.25) : f.h[a];
    }
    L.push_back(c);
  }
  for (auto &l : L) {
    for (int a = 0; a < 3; ++a)
      if (!(l.k[a] = alloc<T>(p, l.N))) return false;
    if (!(l.x = alloc<T>(p, l.N)) || !(l.x2 = alloc<T>(p, l.N)) || !(l.b = alloc<T>(p, l.N))) return false;
    l.rb = (l.nx % 2 == 0) && (l.ny % 2 == 0) && (l.nz % 2 == 0);
  }
  return true;
}

Poisson *poisson_create(const Ctx &c, int fp64) {
  Poisson *p = new Poisson;
  p->fp64 = fp64;
  bool ok = fp64 ? setup<double>(p, c.d) : setup<float>(p, c.d);
  p->b0 = alloc<double>(p, c.d.N);
  p->part = alloc<double>(p, kRedBlocks + 8);
  if (!ok || !p->b0 || !p->part) {
    poisson_destroy(p);
    return nullptr;
  }
  return p;
}

void poisson_destroy(Poisson *p) {
  if (!p) return;
  for (void *a : p->allocs) cudaFree(a);
  delete p;
}

template <typename T> static void smooth(Level<T> &l, int sweeps, bool from_zero, cudaStream_t s) {
  const int B = 256;
  if (l.rb) {
    for (int k = 0; k < sweeps; ++k) {
      const bool z = from_zero && k == 0;
      count_launch(), k_rb<T><<<grid_for(l.N / 2, B), B, 0, s>>>(l, 0, z ? 1 : 0);
      count_launch(), k_rb<T><<<grid_for(l.N / 2, B), B, 0, s>>>(l, 1, 0);
    }
  } else {
    if (from_zero) count_launch(), k_zero<T><<<grid_for(l.N, B), B, 0, s>>>(l.x, l.N);
    for (int k = 0; k < sweeps; ++k) {
      count_launch(), k_jacobi<T><<<grid_for(l.N, B), B, 0, s>>>(l, T(0.8));
      std::swap(l.x, l.x2);
    }
  }
}

template <typename T> static void vcycle(std::vector<Level<T>> &L, size_t li, cudaStream_t s) {
  const int B = 256;
  Level<T> &l = L[li];
  if (li + 1 == L.size()) {
    const int iters = l.rb ? 40 : 120;
    count_launch(), k_coarsest<T><<<1, 1024, 0, s>>>(l, iters);
    return;
  }
  if (l.rb) {
    // the first red half sweep writes every red node; black nodes must start at 0
    count_launch(), k_zero<T><<<grid_for(l.N, B), B, 0, s>>>(l.x, l.N);
  }
  smooth(l, 2, true, s);
  Level<T> &c = L[li + 1];
  count_launch(), k_restrict<T><<<grid_for(c.N, B), B, 0, s>>>(l, c);
  vcycle(L, li + 1, s);
  count_launch(), k_prolong<T><<<grid_for(l.N, B), B, 0, s>>>(l, L[li + 1]);
  smooth(l, 2, false, s);
}

template <typename T> static int solve(Poisson *p, Ctx &c, double tol, int max_iter, double *relres) {
  const int B = 256;
  auto &L = levels<T>(p);
  const Dims d = c.d;
  cudaStream_t s = c.s;
  Level<T> &l0 = L[0];
  count_launch(), k_coef0<T><<<grid_for(d.N, B), B, 0, s>>>(d, (const T *)c.eps, l0.k[0], l0.k[1], l0.k[2]);
  for (size_t li = 1; li < L.size(); ++li) {
    Level<T> &f = L[li - 1], &cc = L[li];
    count_launch(), k_coef_coarsen<T><<<grid_for(cc.N, B), B, 0, s>>>(f.dims(), cc.dims(), cc.cf[0], cc.cf[1], cc.cf[2], f.k[0],
                                                      f.k[1], f.k[2], cc.k[0], cc.k[1], cc.k[2]);
  }
  count_launch(), k_rhs<T><<<grid_for(d.N, B), B, 0, s>>>(d, (const T *)c.q, l0.k[0], l0.k[1], l0.k[2], c.Eext[0], c.Eext[1],
                                          c.Eext[2], p->b0);
  // remove the mean (qbar) with a fixed-order sum
  sum_f64(p->b0, d.N, p->part, s);
  count_launch(), k_add_const<<<grid_for(d.N, B), B, 0, s>>>(p->b0, d.N, p->part + kRedBlocks, 1.0 / double(d.N));
  const double bn = std::sqrt(dot_f64(p->b0, p->b0, d.N, p->part, s));
  if (bn == 0.0) {
    count_launch(), k_zero_d<<<grid_for(d.N, B), B, 0, s>>>(c.phi, d.N);
    *relres = 0.0;
    return 0;
  }
  int it = 0;
  double rr = 0.0;
  while (true) {
    count_launch(), k_residual0<T><<<kRedBlocks, 256, 0, s>>>(l0, c.phi, p->b0, p->part);
    reduce_partials_final(p->part, kRedBlocks, 1, p->part + kRedBlocks, s);
    double h = 0.0;
    cudaMemcpyAsync(&h, p->part + kRedBlocks, sizeof(double), cudaMemcpyDeviceToHost, s);
    if (cudaStreamSynchronize(s) != cudaSuccess) return -1;
    rr = std::sqrt(h) / bn;
    if (rr < tol || it >= max_iter) break;
    vcycle(L, 0, s);
    count_launch(), k_update_phi<T><<<grid_for(d.N, B), B, 0, s>>>(c.phi, l0.x, d.N);
    ++it;
  }
  // mean-free potential
  sum_f64(c.phi, d.N, p->part, s);
  count_launch(), k_add_const<<<grid_for(d.N, B), B, 0, s>>>(c.phi, d.N, p->part + kRedBlocks, 1.0 / double(d.N));
  *relres = rr;
  return rr < tol ? it : -(it + 2);
}

int poisson_solve(Poisson *p, Ctx &c, double tol, int max_iter, double *relres) {
  return p->fp64 ? solve<double>(p, c, tol, max_iter, relres) : solve<float>(p, c, tol, max_iter, relres);
}

}  // namespace lbeh
