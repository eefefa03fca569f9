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
// coefficients combine the fine faces in series along the face normal and
// average them across it (coarse_coef), restriction averages
// the children, prolongation is trilinear, smoothing is red-black
// Gauss-Seidel (damped Jacobi where an axis is odd).  All levels of at most
// kTailCells cells are cycled inside one thread block.
//
// Control: the relative residual is computed and tested on the device.  In
// eager mode the host reads the test after each cycle; inside a captured
// CUDA graph the test drives a conditional WHILE node, so a whole timestep
// runs without host round trips.
#include <algorithm>
#include <type_traits>
#include <cmath>
#include <cstring>
#include <utility>
#include <vector>

#include "internal.h"
#include "poisson_dev.cuh"
#include "spectral_solve.h"

namespace lbeh {

struct Bar;
struct Poisson {
  int fp64 = 0;
  int nred = 0;               // blocks of the FP64 reduction passes (fixed per size)
  int pgrid = 0;              // blocks of the persistent solve (0: not available)
  size_t ptail_smem = 0;      // its dynamic shared memory
  Bar *bar = nullptr;         // its grid barrier
  void *dlevels = nullptr;    // its level table (device)
  std::vector<Level<double>> Ld;
  std::vector<Level<float>> Lf;
  double *phi_prev = nullptr; // solution of the previous step (initial guess extrapolation)
  float *prev_hi = nullptr, *prev_lo = nullptr;  // the same in double-float (FP32 modes)
  double *part = nullptr;     // reduction partials
  PDev *dev = nullptr;
  std::vector<void *> allocs;
  int body_launches = 0;      // kernels of one cycle (launch accounting in graphs)
  Spectral *spec = nullptr;   // spectral solve (replaces the multigrid when set)
  long long spin_limit = kSpinLimit;
};

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

// coarse face coefficients of one level from the finer one (coarse_coef)
template <typename T> __global__ void k_coef_coarsen(Level<T> F, Level<T> C) {
  const Dims c = C.dims();
  long long I = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (I >= c.N) return;
  int X, Y, Z;
  coords(c, I, X, Y, Z);
  C.k[0][I] = coarse_coef<0>(F, C, X, Y, Z);
  C.k[1][I] = coarse_coef<1>(F, C, X, Y, Z);
  C.k[2][I] = coarse_coef<2>(F, C, X, Y, Z);
}

template <typename T> __global__ void __launch_bounds__(1024) k_tail(Tail<T> tl, int first) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ T sh[1024];
  tail_vcycle(tl.L, tl.n, first, smem_raw, sh);
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

// fixed-order sum of the partials, times scale, into *out (and its
// double-float split into *out_df when given)
__global__ void __launch_bounds__(256) k_sum_partials(const double *__restrict__ part, int nb,
                                                      double *__restrict__ out, double scale, DF *out_df) {
  __shared__ double sh[256];
  double acc = 0.0;
  for (int b = threadIdx.x; b < nb; b += 256) acc += part[b];
  const double r = block_sum256(acc, sh);
  if (threadIdx.x == 0) {
    *out = r * scale;
    if (out_df) *out_df = df_split(r * scale);
  }
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
    st->mean_phi_df = df_split(st->mean_phi);
    const double bn = st->bnorm2;
    const double rr = rel_res(r2, bn);
    st->relres = rr;
    st->zero = bn == 0.0;
    const int more = rr >= st->tol && st->iters < st->max_iter;
    st->cond = more;
    const int fail = (rr >= st->tol && st->iters >= st->max_iter) || !isfinite(rr);
    st->notconv = fail;
    if (fail) atomicOr(status, ST_POISSON);
    if (!isfinite(rr)) atomicOr(status, ST_NONFINITE);
    if (use_handle) cudaGraphSetConditional(handle, more ? 1u : 0u);
  }
}

// ---------------------------------------------------------------- double-float driver kernels
// residual r = b - A phi with phi = hi + lo and b = -(q - qbar) + sum_d k (E_ext.c_d)
// in double-float; per-block partials [0] r^2, [1] b^2, [2] phi as in k_residual0
__global__ void __launch_bounds__(256) k_residual_df(Level<float> L, const float *__restrict__ hi,
                                                     const float *__restrict__ lo, const float *__restrict__ q,
                                                     const PDev *__restrict__ st, DF ex, DF ey, DF ez,
                                                     double *__restrict__ part, int nb) {
  const Dims d = L.dims();
  __shared__ double sh[256];
  const DF qbar = st->mean_q_df;
  float ar = 0.f, ab = 0.f, ap = 0.f;
  for (long long i = blockIdx.x * 256LL + threadIdx.x; i < d.N; i += (long long)gridDim.x * 256) {
    int x, y, z;
    coords(d, i, x, y, z);
    const long long ixp = site(d, wrapp(x, d.nx), y, z), ixm = site(d, wrapm(x, d.nx), y, z);
    const long long iyp = site(d, x, wrapp(y, d.ny), z), iym = site(d, x, wrapm(y, d.ny), z);
    const long long izp = site(d, x, y, wrapp(z, d.nz)), izm = site(d, x, y, wrapm(z, d.nz));
    const float kxp = L.k[0][i], kxm = L.k[0][ixm];
    const float kyp = L.k[1][i], kym = L.k[1][iym];
    const float kzp = L.k[2][i], kzm = L.k[2][izm];
    const DF p{hi[i], lo[i]};
    DF Ap = df_mul_f(df_sub(DF{hi[ixp], lo[ixp]}, p), kxp);
    Ap = df_add(Ap, df_mul_f(df_sub(DF{hi[ixm], lo[ixm]}, p), kxm));
    Ap = df_add(Ap, df_mul_f(df_sub(DF{hi[iyp], lo[iyp]}, p), kyp));
    Ap = df_add(Ap, df_mul_f(df_sub(DF{hi[iym], lo[iym]}, p), kym));
    Ap = df_add(Ap, df_mul_f(df_sub(DF{hi[izp], lo[izp]}, p), kzp));
    Ap = df_add(Ap, df_mul_f(df_sub(DF{hi[izm], lo[izm]}, p), kzm));
    DF b = df_sub(qbar, DF{q[i], 0.f});
    if (ex.hi != 0.f) b = df_add(b, df_mul(ex, two_sum(kxp, -kxm)));
    if (ey.hi != 0.f) b = df_add(b, df_mul(ey, two_sum(kyp, -kym)));
    if (ez.hi != 0.f) b = df_add(b, df_mul(ez, two_sum(kzp, -kzm)));
    const DF r = df_sub(b, Ap);
    const float rf = __fadd_rn(r.hi, r.lo);
    L.b[i] = rf;
    ar = __fmaf_rn(rf, rf, ar);
    ab = __fmaf_rn(b.hi, b.hi, ab);
    ap = __fadd_rn(ap, p.hi);
  }
  double v = block_sum256(double(ar), sh);
  if (threadIdx.x == 0) part[blockIdx.x] = v;
  v = block_sum256(double(ab), sh);
  if (threadIdx.x == 0) part[nb + blockIdx.x] = v;
  v = block_sum256(double(ap), sh);
  if (threadIdx.x == 0) part[2 * nb + blockIdx.x] = v;
}

// phi += correction, in double-float
__global__ void k_update_df(float *__restrict__ hi, float *__restrict__ lo, const float *__restrict__ x,
                            long long n) {
  long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (i >= n) return;
  const DF s = df_add(DF{hi[i], lo[i]}, DF{x[i], 0.f});
  hi[i] = s.hi;
  lo[i] = s.lo;
}

// initial guess 2 phi(t-1) - phi(t-2), in double-float
__global__ void k_extrapolate_df(float *__restrict__ hi, float *__restrict__ lo, float *__restrict__ phi_hi,
                                 float *__restrict__ phi_lo, long long n, const PDev *__restrict__ st) {
  long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (i >= n) return;
  const DF p{hi[i], lo[i]};
  if (st->have_prev) {
    const DF g = df_sub(DF{2.f * p.hi, 2.f * p.lo}, DF{phi_hi[i], phi_lo[i]});
    hi[i] = g.hi;
    lo[i] = g.lo;
  }
  phi_hi[i] = p.hi;
  phi_lo[i] = p.lo;
}

// phi -= mean(phi), or phi = 0 for a vanishing right-hand side
__global__ void k_center_df(float *__restrict__ hi, float *__restrict__ lo, long long n,
                            const PDev *__restrict__ st) {
  long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (i >= n) return;
  DF v{0.f, 0.f};
  if (!st->zero) v = df_sub(DF{hi[i], lo[i]}, st->mean_phi_df);
  hi[i] = v.hi;
  lo[i] = v.lo;
}

__global__ void k_df_to_double(const float *__restrict__ hi, const float *__restrict__ lo, double *__restrict__ out,
                               long long n) {
  long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (i < n) out[i] = double(hi[i]) + double(lo[i]);
}

__global__ void k_double_to_df(const double *__restrict__ in, float *__restrict__ hi, float *__restrict__ lo,
                               long long n) {
  long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (i >= n) return;
  const DF v = df_split(in[i]);
  hi[i] = v.hi;
  lo[i] = v.lo;
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

template <typename T, bool DFM>
__global__ void __launch_bounds__(kPB, 2) k_poisson(PArgs<T> a) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ double sh[kPB];
  __shared__ T sht[kPB];
  poisson_body<T, DFM>(a, GridTeam{a.bar, a.status, a.spin_limit}, smem_raw, sh, sht);
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
    // an even axis halves; a two-cell axis coarsens to one cell (no coupling
    // left along it), which keeps thin boxes' coarse operators isotropic
    int cf[3] = {f.nx % 2 == 0, f.ny % 2 == 0, f.nz % 2 == 0};
    // stop at a few cells per axis (4^3 in a cube); thin boxes keep halving
    // their long axes, whose smooth modes a small coarsest level of many
    // cells along one axis would barely relax
    const int ext = std::max(f.nx, std::max(f.ny, f.nz));
    if (!(cf[0] || cf[1] || cf[2]) || (f.N <= 64 && ext <= 4)) break;
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
    l.rb = (l.nx % 2 == 0 || l.nx == 1) && (l.ny % 2 == 0 || l.ny == 1) && (l.nz % 2 == 0 || l.nz == 1) &&
           l.N % 2 == 0;
  }
  if (cudaFuncSetAttribute(k_tail<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kTailSmem) != cudaSuccess)
    return false;
  return true;
}

template <typename T, bool DFM> static void persistent_setup(Poisson *p, const Ctx &c) {
  auto &L = levels<T>(p);
  const size_t ts = tail_start(L);
  for (size_t l = 0; l < ts; ++l)
    if (!L[l].rb) return;  // odd axes above the tail: multi-kernel path
  Tail<T> tl;
  tl.n = (int)L.size();
  for (size_t l = 0; l < L.size(); ++l) tl.L[l] = L[l];
  const size_t smem = tail_bytes(tl, (int)ts);
  if (!raise_smem_limit((const void *)k_poisson<T, DFM>, smem))
    return;
  int dev = 0, nsm = 0, coop = 0, per = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, dev);
  if (!coop || cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_poisson<T, DFM>, kPB, smem) != cudaSuccess ||
      per < 1) {
    cudaGetLastError();
    return;
  }
  // level table in device memory; level 0 forms its face coefficients from eps
  std::vector<Level<T>> tab(L.begin(), L.end());
  if (ts > 0) tab[0].eps = (const T *)c.eps;
  Level<T> *d = alloc<Level<T>>(p, (long long)tab.size());
  if (!d || cudaMemcpy(d, tab.data(), tab.size() * sizeof(Level<T>), cudaMemcpyHostToDevice) != cudaSuccess) return;
  p->dlevels = d;
  p->pgrid = nsm * std::min(per, 2);
  p->ptail_smem = smem;
}

template <typename T, bool DFM> static PArgs<T> fill_args(Poisson *p, const Ctx &c) {
  auto &L = levels<T>(p);
  PArgs<T> a{};
  a.lv = (const Level<T> *)p->dlevels;
  a.nlev = (int)L.size();
  a.tail = L.empty() ? 0 : (int)tail_start(L);  // no levels: spectral solve
  a.eps = (const T *)c.eps;
  a.q = (const T *)c.q;
  if constexpr (DFM) {
    a.phi_hi = (float *)c.phit;
    a.phi_lo = c.phi_lo;
    a.prev_hi = p->prev_hi;
    a.prev_lo = p->prev_lo;
  } else {
    a.phi = c.phi;
    a.prev = p->phi_prev;
  }
  for (int k = 0; k < 3; ++k) a.edf[k] = df_split(c.Eext[k]);
  a.ex = c.Eext[0];
  a.ey = c.Eext[1];
  a.ez = c.Eext[2];
  a.st = p->dev;
  a.status = c.status;
  a.part = p->part;
  a.bar = p->bar;
  a.spin_limit = p->spin_limit;
  return a;
}

template <typename T, bool DFM> static int persistent_launch(Poisson *p, Ctx &c, cudaStream_t s) {
  const PArgs<T> a = fill_args<T, DFM>(p, c);
  if (cudaMemsetAsync(p->bar, 0, sizeof(Bar), s) != cudaSuccess) return -1;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(p->pgrid);
  cfg.blockDim = dim3(kPB);
  cfg.dynamicSmemBytes = p->ptail_smem;
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeCooperative;
  attr[0].val.cooperative = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  count_launch();
  return cudaLaunchKernelEx(&cfg, k_poisson<T, DFM>, a) == cudaSuccess ? 0 : -1;
}

static double eps_range(const Ctx &c, double *lo) {
  double mn = std::min(c.eps_a, c.ncomp == 2 ? c.eps_b : c.eps_a), mx = std::max(c.eps_a, c.ncomp == 2 ? c.eps_b : c.eps_a);
  if (c.ncoll_max > 0) {
    mn = std::min(mn, c.eps_p);
    mx = std::max(mx, c.eps_p);
  }
  *lo = mn;
  return mx;
}

bool poisson_spectral_choice(const Ctx &c, int fp64) {
  if (c.psolver == LBEH_POISSON_MULTIGRID) return false;
  if (!spectral_supported(c.d, fp64)) return false;
  if (c.psolver == LBEH_POISSON_SPECTRAL) return true;
  double lo = 0.0;
  const double hi = eps_range(c, &lo);
  return c.ncoll_max == 0 && lo > 0.0 && hi / lo <= kSpectralMaxContrast;
}

bool poisson_is_spectral(const Poisson *p) { return p->spec != nullptr; }
void poisson_set_wait_limit(Poisson *p, long long polls) { p->spin_limit = polls > 0 ? polls : kSpinLimit; }

Poisson *poisson_create(const Ctx &c, int fp64) {
  Poisson *p = new Poisson;
  p->fp64 = fp64;
  if (poisson_spectral_choice(c, fp64)) {
    double lo = 0.0;
    const double hi = eps_range(c, &lo);
    p->spec = spectral_create(c, fp64, 0.5 * (lo + hi));
    if (!p->spec) {
      delete p;
      return nullptr;
    }
    if (fp64)
      p->phi_prev = alloc<double>(p, c.d.N);
    else {
      p->prev_hi = alloc<float>(p, c.d.N);
      p->prev_lo = alloc<float>(p, c.d.N);
    }
    p->dev = alloc<PDev>(p, 1);
    p->bar = alloc<Bar>(p, 1);
    p->part = alloc<double>(p, 3 * spectral_grid(p->spec) + 8);
    if ((fp64 ? !p->phi_prev : (!p->prev_hi || !p->prev_lo)) || !p->dev || !p->bar || !p->part) {
      poisson_destroy(p);
      return nullptr;
    }
    cudaMemset(p->bar, 0, sizeof(Bar));
    cudaMemset(p->dev, 0, sizeof(PDev));
    return p;
  }
  bool ok = fp64 ? setup<double>(p, c.d) : setup<float>(p, c.d);
  if (fp64) {
    p->phi_prev = alloc<double>(p, c.d.N);
  } else {
    p->prev_hi = alloc<float>(p, c.d.N);
    p->prev_lo = alloc<float>(p, c.d.N);
  }
  p->nred = int(std::min<long long>(std::max<long long>((c.d.N + 255) / 256, 1), 8192));
  p->dev = alloc<PDev>(p, 1);
  p->bar = alloc<Bar>(p, 1);
  if (p->bar) cudaMemset(p->bar, 0, sizeof(Bar));
  // persistent solve: every level above the tail must be red-black colourable
  if (p->bar) {
    if (fp64)
      persistent_setup<double, false>(p, c);
    else
      persistent_setup<float, true>(p, c);
  }
  p->part = alloc<double>(p, 3 * std::max(p->nred, p->pgrid) + 8);
  if (!ok || (fp64 ? !p->phi_prev : (!p->prev_hi || !p->prev_lo)) || !p->part || !p->dev) {
    poisson_destroy(p);
    return nullptr;
  }
  cudaMemset(p->dev, 0, sizeof(PDev));
  return p;
}

void poisson_destroy(Poisson *p) {
  if (!p) return;
  spectral_destroy(p->spec);
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
  constexpr bool DFM = std::is_same<T, float>::value;  // double-float potential
  if (p->spec || p->pgrid > 0) {
    // whole solve in one cooperative launch
    if (p->spec) {
      const PArgs<T> a = fill_args<T, DFM>(p, c);
      int rc;
      if constexpr (DFM)
        rc = spectral_launch_f32(p->spec, c, a, s);
      else
        rc = spectral_launch_f64(p->spec, c, a, s);
      if (rc != 0) return -1;
    } else if (persistent_launch<T, DFM>(p, c, s) != 0) {
      return -1;
    }
    p->body_launches = 0;
    if (graph) return 0;
    PDev hd{};
    if (cudaMemcpyAsync(&hd, p->dev, sizeof(PDev), cudaMemcpyDeviceToHost, s) != cudaSuccess) return -1;
    if (cudaStreamSynchronize(s) != cudaSuccess) return -1;
    *relres = hd.relres;
    return hd.notconv ? -(hd.iters + 2) : hd.iters;
  }
  Level<T> &l0 = L[0];
  float *phi_hi = (float *)c.phit, *phi_lo = c.phi_lo;
  const DF edf[3] = {df_split(c.Eext[0]), df_split(c.Eext[1]), df_split(c.Eext[2])};
  auto residual = [&](cudaStream_t st) {
    if constexpr (DFM)
      count_launch(), k_residual_df<<<p->nred, 256, 0, st>>>(l0, phi_hi, phi_lo, (const float *)c.q, p->dev, edf[0],
                                                             edf[1], edf[2], p->part, p->nred);
    else
      count_launch(), k_residual0<T><<<p->nred, 256, 0, st>>>(l0, c.phi, (const T *)c.q, p->dev, c.Eext[0],
                                                              c.Eext[1], c.Eext[2], p->part, p->nred);
  };
  if constexpr (DFM)
    count_launch(), k_extrapolate_df<<<grid_for(d.N, B), B, 0, s>>>(phi_hi, phi_lo, p->prev_hi, p->prev_lo, d.N,
                                                                    p->dev);
  else
    count_launch(), k_extrapolate<<<grid_for(d.N, B), B, 0, s>>>(c.phi, p->phi_prev, d.N, p->dev);
  count_launch(), k_coef0_qsum<T><<<p->nred, 256, 0, s>>>(d, (const T *)c.eps, (const T *)c.q, l0.k[0], l0.k[1],
                                                         l0.k[2], p->part);
  count_launch(), k_sum_partials<<<1, 256, 0, s>>>(p->part, p->nred, &p->dev->mean_q, 1.0 / double(d.N),
                                                   &p->dev->mean_q_df);
  for (size_t li = 1; li < L.size(); ++li)
    count_launch(), k_coef_coarsen<T><<<grid_for(L[li].N, B), B, 0, s>>>(L[li - 1], L[li]);
  residual(s);
  count_launch(), k_check<<<1, 256, 0, s>>>(p->part, p->nred, p->dev, c.status, 1, d.N, handle, graph ? 1 : 0);
  auto body = [&](cudaStream_t bs) {
    T *corr = vcycle(L, bs);
    if constexpr (DFM)
      count_launch(), k_update_df<<<grid_for(d.N, B), B, 0, bs>>>(phi_hi, phi_lo, (const float *)corr, d.N);
    else
      count_launch(), k_update_phi<T><<<grid_for(d.N, B), B, 0, bs>>>(c.phi, corr, d.N);
    residual(bs);
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
  // mean-free potential (the hi words are the compute-type copy read by the step kernels)
  if constexpr (DFM)
    count_launch(), k_center_df<<<grid_for(d.N, 256), 256, 0, s>>>(phi_hi, phi_lo, d.N, p->dev);
  else
    count_launch(), k_center_copy<T><<<grid_for(d.N, 256), 256, 0, s>>>(c.phi, d.N, p->dev, (T *)nullptr);
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
  // forget the previous solutions (new state loaded); stream-ordered
  return cudaMemsetAsync(&p->dev->have_prev, 0, sizeof(int), s) == cudaSuccess ? 0 : -1;
}

int poisson_solve(Poisson *p, Ctx &c, double *relres) {
  cudaGraphConditionalHandle none = 0;
  return p->fp64 ? enqueue<double>(p, c, none, false, relres) : enqueue<float>(p, c, none, false, relres);
}

int poisson_capture(Poisson *p, Ctx &c, cudaGraphConditionalHandle handle) {
  double rr = 0;
  return p->fp64 ? enqueue<double>(p, c, handle, true, &rr) : enqueue<float>(p, c, handle, true, &rr);
}

// Level table in device memory for a solve by one team (built here when the
// cooperative solve was not set up); -1 when a level above the tail cannot be
// coloured red-black.
template <typename T, bool DFM> static long long team_setup(Poisson *p, const Ctx &c) {
  auto &L = levels<T>(p);
  const size_t ts = tail_start(L);
  for (size_t l = 0; l < ts; ++l)
    if (!L[l].rb) return -1;
  Tail<T> tl;
  tl.n = (int)L.size();
  for (size_t l = 0; l < L.size(); ++l) tl.L[l] = L[l];
  const size_t smem = tail_bytes(tl, (int)ts);
  if (!p->dlevels) {
    std::vector<Level<T>> tab(L.begin(), L.end());
    if (ts > 0) tab[0].eps = (const T *)c.eps;
    Level<T> *d = alloc<Level<T>>(p, (long long)tab.size());
    if (!d || cudaMemcpy(d, tab.data(), tab.size() * sizeof(Level<T>), cudaMemcpyHostToDevice) != cudaSuccess)
      return -1;
    p->dlevels = d;
  }
  return (long long)smem;
}

long long poisson_team_args(Poisson *p, const Ctx &c, void *out, size_t out_bytes) {
  if (p->spec) return -1;  // the batched step cycles the multigrid
  if (p->fp64) {
    if (out_bytes != sizeof(PArgs<double>)) return -1;
    const long long smem = team_setup<double, false>(p, c);
    if (smem < 0) return -1;
    const PArgs<double> a = fill_args<double, false>(p, c);
    std::memcpy(out, &a, sizeof(a));
    return smem;
  }
  if (out_bytes != sizeof(PArgs<float>)) return -1;
  const long long smem = team_setup<float, true>(p, c);
  if (smem < 0) return -1;
  const PArgs<float> a = fill_args<float, true>(p, c);
  std::memcpy(out, &a, sizeof(a));
  return smem;
}

void poisson_state_buffers(Poisson *p, const Ctx &c, std::vector<std::pair<void *, size_t>> &out) {
  if (p->fp64) {
    out.emplace_back(p->phi_prev, 8 * (size_t)c.d.N);
  } else {
    out.emplace_back(p->prev_hi, 4 * (size_t)c.d.N);
    out.emplace_back(p->prev_lo, 4 * (size_t)c.d.N);
  }
  out.emplace_back(p->dev, sizeof(PDev));
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

namespace lbeh {
// the potential as FP64 values (either representation)
void phi_to_double(Ctx &c, double *out) {
  if (c.prec == LBEH_FP64) {
    cudaMemcpyAsync(out, c.phi, 8 * c.d.N, cudaMemcpyDeviceToDevice, c.s);
  } else {
    count_launch(), k_df_to_double<<<grid_for(c.d.N, 256), 256, 0, c.s>>>((const float *)c.phit, c.phi_lo, out, c.d.N);
  }
}
void phi_from_double(Ctx &c, const double *in) {
  if (c.prec == LBEH_FP64) {
    cudaMemcpyAsync(c.phi, in, 8 * c.d.N, cudaMemcpyDeviceToDevice, c.s);
  } else {
    count_launch(), k_double_to_df<<<grid_for(c.d.N, 256), 256, 0, c.s>>>(in, (float *)c.phit, c.phi_lo, c.d.N);
  }
}
}  // namespace lbeh

namespace lbeh {
bool poisson_needs_conditional(const Poisson *p) { return p->pgrid == 0 && !p->spec; }
}  // namespace lbeh
