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
// Gauss-Seidel (damped Jacobi where an axis is odd).  All levels of at most
// kTailCells cells are cycled inside one thread block.
//
// Control: the relative residual is computed and tested on the device.  In
// eager mode the host reads the test after each cycle; inside a captured
// CUDA graph the test drives a conditional WHILE node, so a whole timestep
// runs without host round trips.
#include <algorithm>
#include <cmath>
#include <utility>
#include <vector>

#include "internal.h"

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
  bool rb = false;
  __host__ __device__ Dims dims() const { return Dims{nx, ny, nz, N}; }
};

template <typename T> struct Tail {
  int n = 0;
  Level<T> L[kMaxLevels];
};

// Device-side solver state.
struct PDev {
  double mean_q, mean_phi, bnorm2, rnorm2, relres, tol;
  int iters, max_iter, cond, notconv;
  long long total_iters;
  int have_prev;  // phi_prev holds the solution of the previous step
  int zero;       // right-hand side vanishes: phi = 0
};

struct Poisson {
  int fp64 = 0;
  int nred = 0;               // blocks of the FP64 reduction passes (fixed per size)
  std::vector<Level<double>> Ld;
  std::vector<Level<float>> Lf;
  double *phi_prev = nullptr; // solution of the previous step (initial guess extrapolation)
  double *part = nullptr;     // reduction partials
  PDev *dev = nullptr;
  std::vector<void *> allocs;
  int body_launches = 0;      // kernels of one cycle (launch accounting in graphs)
};

// ---------------------------------------------------------------- level operations
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

// one colour of a red-black sweep over the thread range t0, t0+dt, ... < N/2
template <typename T>
__device__ __forceinline__ void rb_range(const Level<T> &L, int color, long long t0, long long dt) {
  const Dims d = L.dims();
  const unsigned hx = unsigned(d.nx / 2);
  for (long long t = t0; t < d.N / 2; t += dt) {
    const unsigned r = unsigned(t) / hx;
    const int xh = int(unsigned(t) - r * hx);
    const int z = int(r / unsigned(d.ny));
    const int y = int(r - unsigned(z) * unsigned(d.ny));
    const int x = 2 * xh + ((y + z + color) & 1);
    const long long i = site(d, x, y, z);
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

// coarse b(I) = mean over children of the fine residual (b - A x)
template <typename T>
__device__ __forceinline__ void restrict_range(const Level<T> &F, const Level<T> &C, long long t0, long long dt) {
  const Dims f = F.dims(), c = C.dims();
  for (long long I = t0; I < c.N; I += dt) {
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
}

// trilinear (cell-centred) prolongation and correction x_f += P x_c
template <typename T>
__device__ __forceinline__ void prolong_range(const Level<T> &F, const Level<T> &C, long long t0, long long dt) {
  const Dims f = F.dims(), c = C.dims();
  const int cd[3] = {c.nx, c.ny, c.nz};
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

// ---------------------------------------------------------------- multi-block kernels
template <typename T> __global__ void k_rb(Level<T> L, int color) {
  rb_range(L, color, blockIdx.x * (long long)blockDim.x + threadIdx.x, (long long)gridDim.x * blockDim.x);
}
template <typename T> __global__ void k_jacobi(Level<T> L, T w) {
  jacobi_range(L, w, blockIdx.x * (long long)blockDim.x + threadIdx.x, (long long)gridDim.x * blockDim.x);
}
template <typename T> __global__ void k_restrict(Level<T> F, Level<T> C) {
  restrict_range(F, C, blockIdx.x * (long long)blockDim.x + threadIdx.x, (long long)gridDim.x * blockDim.x);
}
template <typename T> __global__ void k_prolong(Level<T> F, Level<T> C) {
  prolong_range(F, C, blockIdx.x * (long long)blockDim.x + threadIdx.x, (long long)gridDim.x * blockDim.x);
}
template <typename T> __global__ void k_zero(T *p, long long n) {
  long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (i < n) p[i] = T(0);
}

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
template <typename T> __global__ void k_coef_coarsen(Level<T> F, Level<T> C) {
  const Dims f = F.dims(), c = C.dims();
  long long I = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (I >= c.N) return;
  int X, Y, Z;
  coords(c, I, X, Y, Z);
  const int base[3] = {C.cf[0] ? 2 * X : X, C.cf[1] ? 2 * Y : Y, C.cf[2] ? 2 * Z : Z};
  for (int a = 0; a < 3; ++a) {
    T acc = T(0);
    int cnt = 0;
    const int ra = C.cf[a] ? 1 : 0;
    const int b1 = (a + 1) % 3, b2 = (a + 2) % 3;
    for (int t1 = 0; t1 <= C.cf[b1]; ++t1)
      for (int t2 = 0; t2 <= C.cf[b2]; ++t2) {
        int p[3];
        p[a] = base[a] + ra;
        p[b1] = base[b1] + t1;
        p[b2] = base[b2] + t2;
        acc += F.k[a][site(f, p[0], p[1], p[2])];
        ++cnt;
      }
    C.k[a][I] = acc / T(cnt);
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
template <typename T> __global__ void __launch_bounds__(1024) k_tail(Tail<T> tl, int first) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ T sh[1024];
  Tail<T> sl = tl;  // same levels, arrays redirected to shared memory
  {
    T *p = reinterpret_cast<T *>(smem_raw);
    for (int l = first; l < tl.n; ++l) {
      Level<T> &L = sl.L[l];
      const long long n = L.N;
      for (int a = 0; a < 3; ++a) {
        L.k[a] = p;
        p += n;
      }
      L.x = p;
      p += n;
      L.b = p;
      p += n;
      if (!L.rb) {
        L.x2 = p;
        p += n;
      }
    }
  }
  for (int l = first; l < tl.n; ++l) {
    const long long n = tl.L[l].N;
    for (long long i = threadIdx.x; i < n; i += blockDim.x) {
      for (int a = 0; a < 3; ++a) sl.L[l].k[a][i] = tl.L[l].k[a][i];
      if (l == first) sl.L[l].b[i] = tl.L[l].b[i];
    }
  }
  __syncthreads();
  for (int l = first; l < sl.n; ++l) {
    const Level<T> &L = sl.L[l];
    if (l == sl.n - 1) {
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
      tail_smooth(L, L.rb ? 16 : 48);
    } else {
      for (long long i = threadIdx.x; i < L.N; i += blockDim.x) L.x[i] = T(0);
      __syncthreads();
      tail_smooth(L, kNu);
      restrict_range(L, sl.L[l + 1], threadIdx.x, blockDim.x);
      __syncthreads();
    }
  }
  for (int l = sl.n - 2; l >= first; --l) {
    prolong_range(sl.L[l], sl.L[l + 1], threadIdx.x, blockDim.x);
    __syncthreads();
    tail_smooth(sl.L[l], kNu);
  }
  for (long long i = threadIdx.x; i < tl.L[first].N; i += blockDim.x) tl.L[first].x[i] = sl.L[first].x[i];
}

// ---------------------------------------------------------------- FP64 driver kernels
__device__ __forceinline__ double block_sum256(double v, double *sh) {
  sh[threadIdx.x] = v;
  __syncthreads();
  for (int w = 128; w > 0; w >>= 1) {
    if (threadIdx.x < w) sh[threadIdx.x] += sh[threadIdx.x + w];
    __syncthreads();
  }
  const double r = sh[0];
  __syncthreads();
  return r;
}

// level-0 face coefficients from eps, and per-block partial sums of q
template <typename T>
__global__ void __launch_bounds__(256) k_coef0_qsum(Dims d, const T *__restrict__ eps, const T *__restrict__ q,
                                                    T *__restrict__ kx, T *__restrict__ ky, T *__restrict__ kz,
                                                    double *__restrict__ part) {
  __shared__ double sh[256];
  double acc = 0.0;
  for (long long i = blockIdx.x * 256LL + threadIdx.x; i < d.N; i += (long long)gridDim.x * 256) {
    int x, y, z;
    coords(d, i, x, y, z);
    const T e = eps[i];
    kx[i] = T(0.5) * (e + eps[site(d, wrapp(x, d.nx), y, z)]);
    ky[i] = T(0.5) * (e + eps[site(d, x, wrapp(y, d.ny), z)]);
    kz[i] = T(0.5) * (e + eps[site(d, x, y, wrapp(z, d.nz))]);
    acc += double(q[i]);
  }
  const double r = block_sum256(acc, sh);
  if (threadIdx.x == 0) part[blockIdx.x] = r;
}

// fixed-order sum of the partials, times scale, into *out
__global__ void __launch_bounds__(256) k_sum_partials(const double *__restrict__ part, int nb,
                                                      double *__restrict__ out, double scale) {
  __shared__ double sh[256];
  double acc = 0.0;
  for (int b = threadIdx.x; b < nb; b += 256) acc += part[b];
  const double r = block_sum256(acc, sh);
  if (threadIdx.x == 0) *out = r * scale;
}

// FP64 residual r = b - A phi with b = -(q - qbar) + sum_d k (E_ext.c_d)
// formed on the fly; r (compute type) becomes the level-0 right-hand side.
// Per-block partials: [0] r^2, [1] b^2, [2] phi.
template <typename T>
__global__ void __launch_bounds__(256) k_residual0(Level<T> L, const double *__restrict__ phi,
                                                   const T *__restrict__ q, const PDev *__restrict__ st,
                                                   double ex, double ey, double ez, double *__restrict__ part,
                                                   int nb) {
  const Dims d = L.dims();
  __shared__ double sh[256];
  const double qbar = st->mean_q;
  double ar = 0.0, ab = 0.0, ap = 0.0;
  for (long long i = blockIdx.x * 256LL + threadIdx.x; i < d.N; i += (long long)gridDim.x * 256) {
    int x, y, z;
    coords(d, i, x, y, z);
    const long long ixp = site(d, wrapp(x, d.nx), y, z), ixm = site(d, wrapm(x, d.nx), y, z);
    const long long iyp = site(d, x, wrapp(y, d.ny), z), iym = site(d, x, wrapm(y, d.ny), z);
    const long long izp = site(d, x, y, wrapp(z, d.nz)), izm = site(d, x, y, wrapm(z, d.nz));
    const double kxp = double(L.k[0][i]), kxm = double(L.k[0][ixm]);
    const double kyp = double(L.k[1][i]), kym = double(L.k[1][iym]);
    const double kzp = double(L.k[2][i]), kzm = double(L.k[2][izm]);
    double b = -(double(q[i]) - qbar);
    if (ex != 0.0) b += ex * (kxp - kxm);
    if (ey != 0.0) b += ey * (kyp - kym);
    if (ez != 0.0) b += ez * (kzp - kzm);
    const double p = phi[i];
    const double Ap = kxp * (phi[ixp] - p) - kxm * (p - phi[ixm]) + kyp * (phi[iyp] - p) - kym * (p - phi[iym]) +
                      kzp * (phi[izp] - p) - kzm * (p - phi[izm]);
    const double r = b - Ap;
    L.b[i] = T(r);
    ar += r * r;
    ab += b * b;
    ap += p;
  }
  double v = block_sum256(ar, sh);
  if (threadIdx.x == 0) part[blockIdx.x] = v;
  v = block_sum256(ab, sh);
  if (threadIdx.x == 0) part[nb + blockIdx.x] = v;
  v = block_sum256(ap, sh);
  if (threadIdx.x == 0) part[2 * nb + blockIdx.x] = v;
}

// relative residual, loop condition, iteration count, status, mean of phi
__global__ void __launch_bounds__(256) k_check(const double *__restrict__ part, int nb, PDev *__restrict__ st,
                                               int *__restrict__ status, int first, long long n,
                                               cudaGraphConditionalHandle handle, int use_handle) {
  __shared__ double sh[256];
  double a0 = 0.0, a1 = 0.0, a2 = 0.0;
  for (int b = threadIdx.x; b < nb; b += 256) {
    a0 += part[b];
    a1 += part[nb + b];
    a2 += part[2 * nb + b];
  }
  const double r2 = block_sum256(a0, sh);
  const double b2 = block_sum256(a1, sh);
  const double ps = block_sum256(a2, sh);
  if (threadIdx.x == 0) {
    if (first) {
      st->bnorm2 = b2;
      st->iters = 0;
    } else {
      st->iters += 1;
      st->total_iters += 1;
    }
    st->rnorm2 = r2;
    st->mean_phi = ps / double(n);
    const double bn = st->bnorm2;
    const double rr = bn > 0.0 ? sqrt(r2 / bn) : 0.0;
    st->relres = rr;
    st->zero = bn == 0.0;
    const int more = rr >= st->tol && st->iters < st->max_iter;
    st->cond = more;
    const int fail = rr >= st->tol && st->iters >= st->max_iter;
    st->notconv = fail;
    if (fail) atomicOr(status, ST_POISSON);
    if (use_handle) cudaGraphSetConditional(handle, more ? 1u : 0u);
  }
}

// initial guess phi(t) ~ 2 phi(t-1) - phi(t-2) once two solutions exist
__global__ void k_extrapolate(double *__restrict__ phi, double *__restrict__ prev, long long n,
                              const PDev *__restrict__ st) {
  long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (i >= n) return;
  const double p = phi[i];
  if (st->have_prev) phi[i] = 2.0 * p - prev[i];
  prev[i] = p;
}

__global__ void k_mark_prev(PDev *st) { st->have_prev = 1; }

// phi -= mean(phi) (or phi = 0 for a vanishing right-hand side); the
// compute-type copy read by the step kernels
template <typename T>
__global__ void k_center_copy(double *__restrict__ phi, long long n, const PDev *__restrict__ st,
                              T *__restrict__ out) {
  long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (i >= n) return;
  const double v = st->zero ? 0.0 : phi[i] - st->mean_phi;
  phi[i] = v;
  if (out) out[i] = T(v);
}

template <typename T>
__global__ void k_update_phi(double *__restrict__ phi, const T *__restrict__ x, long long n) {
  long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (i < n) phi[i] += double(x[i]);
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
  while ((int)L.size() < kMaxLevels) {
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
  if (cudaFuncSetAttribute(k_tail<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kTailSmem) != cudaSuccess)
    return false;
  return true;
}

Poisson *poisson_create(const Ctx &c, int fp64) {
  Poisson *p = new Poisson;
  p->fp64 = fp64;
  bool ok = fp64 ? setup<double>(p, c.d) : setup<float>(p, c.d);
  p->phi_prev = alloc<double>(p, c.d.N);
  p->nred = int(std::min<long long>(std::max<long long>((c.d.N + 255) / 256, 1), 8192));
  p->part = alloc<double>(p, 3 * p->nred + 8);
  p->dev = alloc<PDev>(p, 1);
  if (!ok || !p->phi_prev || !p->part || !p->dev) {
    poisson_destroy(p);
    return nullptr;
  }
  cudaMemset(p->dev, 0, sizeof(PDev));
  return p;
}

void poisson_destroy(Poisson *p) {
  if (!p) return;
  for (void *a : p->allocs) cudaFree(a);
  delete p;
}

// first level cycled by the single-block tail kernel: the coarse levels of at
// most kTailCells cells whose arrays fit in kTailSmem bytes of shared memory
template <typename T> static size_t tail_start(const std::vector<Level<T>> &L) {
  size_t t = L.size() - 1;
  auto bytes = [&](size_t first) {
    size_t b = 0;
    for (size_t l = first; l < L.size(); ++l) b += size_t(L[l].rb ? 5 : 6) * L[l].N * sizeof(T);
    return b;
  };
  while (t > 0 && L[t - 1].N <= kTailCells && bytes(t - 1) <= kTailSmem) --t;
  return t;
}

template <typename T> static void smooth(Level<T> &l, int sweeps, cudaStream_t s) {
  const int B = 256;
  if (l.rb) {
    for (int k = 0; k < sweeps; ++k) {
      count_launch(), k_rb<T><<<grid_for(l.N / 2, B), B, 0, s>>>(l, 0);
      count_launch(), k_rb<T><<<grid_for(l.N / 2, B), B, 0, s>>>(l, 1);
    }
  } else {
    for (int k = 0; k < sweeps; ++k) {
      count_launch(), k_jacobi<T><<<grid_for(l.N, B), B, 0, s>>>(l, T(0.8));
      std::swap(l.x, l.x2);
    }
  }
}

// One V-cycle for the correction at level 0 (right-hand side in L[0].b).  The
// levels are a copy: Jacobi ping-pong swaps stay local to the cycle, and the
// correction is left in L[0].x of the copy (returned).
template <typename T> static T *vcycle(std::vector<Level<T>> L, cudaStream_t s) {
  const int B = 256;
  const size_t ts = tail_start(L);
  for (size_t l = 0; l < ts; ++l) {
    Level<T> &lv = L[l];
    count_launch(), k_zero<T><<<grid_for(lv.N, B), B, 0, s>>>(lv.x, lv.N);
    smooth(lv, kNu, s);
    count_launch(), k_restrict<T><<<grid_for(L[l + 1].N, B), B, 0, s>>>(lv, L[l + 1]);
  }
  Tail<T> tl;
  tl.n = (int)L.size();
  for (size_t l = 0; l < L.size(); ++l) tl.L[l] = L[l];
  count_launch(), k_tail<T><<<1, 1024, tail_bytes(tl, (int)ts), s>>>(tl, (int)ts);
  for (size_t l = ts; l-- > 0;) {
    count_launch(), k_prolong<T><<<grid_for(L[l].N, B), B, 0, s>>>(L[l], L[l + 1]);
    smooth(L[l], kNu, s);
  }
  return L[0].x;
}

template <typename T>
static int enqueue(Poisson *p, Ctx &c, cudaGraphConditionalHandle handle, bool graph, double *relres) {
  const int B = 256;
  auto &L = levels<T>(p);
  const Dims d = c.d;
  const cudaStream_t s = c.s;
  Level<T> &l0 = L[0];
  count_launch(), k_extrapolate<<<grid_for(d.N, B), B, 0, s>>>(c.phi, p->phi_prev, d.N, p->dev);
  count_launch(), k_coef0_qsum<T><<<p->nred, 256, 0, s>>>(d, (const T *)c.eps, (const T *)c.q, l0.k[0], l0.k[1],
                                                         l0.k[2], p->part);
  count_launch(), k_sum_partials<<<1, 256, 0, s>>>(p->part, p->nred, &p->dev->mean_q, 1.0 / double(d.N));
  for (size_t li = 1; li < L.size(); ++li)
    count_launch(), k_coef_coarsen<T><<<grid_for(L[li].N, B), B, 0, s>>>(L[li - 1], L[li]);
  count_launch(), k_residual0<T><<<p->nred, 256, 0, s>>>(l0, c.phi, (const T *)c.q, p->dev, c.Eext[0], c.Eext[1],
                                                         c.Eext[2], p->part, p->nred);
  count_launch(), k_check<<<1, 256, 0, s>>>(p->part, p->nred, p->dev, c.status, 1, d.N, handle, graph ? 1 : 0);
  auto body = [&](cudaStream_t bs) {
    T *corr = vcycle(L, bs);
    count_launch(), k_update_phi<T><<<grid_for(d.N, B), B, 0, bs>>>(c.phi, corr, d.N);
    count_launch(), k_residual0<T><<<p->nred, 256, 0, bs>>>(l0, c.phi, (const T *)c.q, p->dev, c.Eext[0],
                                                            c.Eext[1], c.Eext[2], p->part, p->nred);
    count_launch(), k_check<<<1, 256, 0, bs>>>(p->part, p->nred, p->dev, c.status, 0, d.N, handle, graph ? 1 : 0);
  };
  PDev hd{};
  if (graph) {
    // conditional WHILE node whose body is one defect-correction cycle
    cudaStreamCaptureStatus cs;
    cudaGraph_t g = nullptr;
    const cudaGraphNode_t *deps = nullptr;
    size_t ndeps = 0;
    if (cudaStreamGetCaptureInfo(s, &cs, nullptr, &g, &deps, nullptr, &ndeps) != cudaSuccess ||
        cs != cudaStreamCaptureStatusActive)
      return -1;
    cudaGraphNodeParams np = {};
    np.type = cudaGraphNodeTypeConditional;
    np.conditional.handle = handle;
    np.conditional.type = cudaGraphCondTypeWhile;
    np.conditional.size = 1;
    cudaGraphNode_t node;
    if (cudaGraphAddNode(&node, g, deps, nullptr, ndeps, &np) != cudaSuccess) return -1;
    cudaGraph_t bodyg = np.conditional.phGraph_out[0];
    cudaStream_t bs;
    if (cudaStreamCreateWithFlags(&bs, cudaStreamNonBlocking) != cudaSuccess) return -1;
    if (cudaStreamBeginCaptureToGraph(bs, bodyg, nullptr, nullptr, 0, cudaStreamCaptureModeRelaxed) != cudaSuccess) {
      cudaStreamDestroy(bs);
      return -1;
    }
    const long long before = g_launches.load();
    body(bs);
    p->body_launches = int(g_launches.load() - before);
    g_launches.fetch_sub(p->body_launches);  // counted per executed cycle instead
    cudaGraph_t out = nullptr;
    const cudaError_t e = cudaStreamEndCapture(bs, &out);
    cudaStreamDestroy(bs);
    if (e != cudaSuccess) return -1;
    if (cudaStreamUpdateCaptureDependencies(s, &node, nullptr, 1, cudaStreamSetCaptureDependencies) != cudaSuccess)
      return -1;
  } else {
    while (true) {
      if (cudaMemcpyAsync(&hd, p->dev, sizeof(PDev), cudaMemcpyDeviceToHost, s) != cudaSuccess) return -1;
      if (cudaStreamSynchronize(s) != cudaSuccess) return -1;
      if (!hd.cond) break;
      body(s);
    }
  }
  // mean-free potential and its compute-type copy
  count_launch(), k_center_copy<T><<<grid_for(d.N, 256), 256, 0, s>>>(
      c.phi, d.N, p->dev, (void *)c.phit == (void *)c.phi ? nullptr : (T *)c.phit);
  count_launch(), k_mark_prev<<<1, 1, 0, s>>>(p->dev);
  if (graph) return 0;
  *relres = hd.relres;
  return hd.notconv ? -(hd.iters + 2) : hd.iters;
}

int poisson_configure(Poisson *p, double tol, int max_iter, cudaStream_t s) {
  PDev h{};
  if (cudaMemcpyAsync(&h, p->dev, sizeof(PDev), cudaMemcpyDeviceToHost, s) != cudaSuccess) return -1;
  if (cudaStreamSynchronize(s) != cudaSuccess) return -1;
  h.tol = tol;
  h.max_iter = max_iter;
  if (cudaMemcpyAsync(p->dev, &h, sizeof(PDev), cudaMemcpyHostToDevice, s) != cudaSuccess) return -1;
  return cudaStreamSynchronize(s) == cudaSuccess ? 0 : -1;
}

int poisson_reset(Poisson *p, cudaStream_t s) {
  // forget the previous solutions (new state loaded)
  const int zero = 0;
  if (cudaMemcpyAsync(&p->dev->have_prev, &zero, sizeof(int), cudaMemcpyHostToDevice, s) != cudaSuccess) return -1;
  return cudaStreamSynchronize(s) == cudaSuccess ? 0 : -1;
}

int poisson_solve(Poisson *p, Ctx &c, double *relres) {
  cudaGraphConditionalHandle none = 0;
  return p->fp64 ? enqueue<double>(p, c, none, false, relres) : enqueue<float>(p, c, none, false, relres);
}

int poisson_capture(Poisson *p, Ctx &c, cudaGraphConditionalHandle handle) {
  double rr = 0;
  return p->fp64 ? enqueue<double>(p, c, handle, true, &rr) : enqueue<float>(p, c, handle, true, &rr);
}

int poisson_read(Poisson *p, cudaStream_t s, PoissonStats *out) {
  PDev h{};
  if (cudaMemcpyAsync(&h, p->dev, sizeof(PDev), cudaMemcpyDeviceToHost, s) != cudaSuccess) return -1;
  if (cudaStreamSynchronize(s) != cudaSuccess) return -1;
  out->iters = h.iters;
  out->relres = h.relres;
  out->total_iters = h.total_iters;
  out->notconv = h.notconv;
  out->body_launches = p->body_launches;
  return 0;
}

}  // namespace lbeh
