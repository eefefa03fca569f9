// Spectral solve of the variable-permittivity Poisson equation (Sec. II.B eq.
// electric_potential, Sec. II.D): conjugate gradients on the flux-form
// equation  sum_d k_{i+d/2} (phi_{i+d} - phi_i) = b  preconditioned by the
// constant-coefficient inverse (eps_ref L)^-1 of spectral.cuh, the Fourier
// method of Sec. II.D.  Defect correction around it: the residual
// r = b - A phi is formed in FP64 (FP64 mode) or double-float (FP32 modes)
// against the potential, conjugate gradients in the compute type find the
// correction e of A e = r, and phi += e in the potential's precision.  The
// number of iterations follows the permittivity contrast (condition number of
// the preconditioned operator eps_max / eps_min), not the box size.
//
// The whole solve is one cooperative launch whose phases are separated by the
// bounded grid barrier of poisson_dev.cuh.  One iteration is six phases:
//   U  r -= alpha q, e += alpha p (sums |r|^2, e), Hartley pass along x of r
//      into the work array w;
//   Y  pass along y of w;   Z  pass along z, symbol scaling, pass along z;
//   Y  pass along y;        X  pass along x (w = z = M^-1 r; sum r.z);
//   F  p = z + beta p, q = A z + beta q (sum p.q).
#include <algorithm>
#include <cmath>
#include <vector>

#include "internal.h"
#include "poisson_dev.cuh"
#include "spectral.cuh"
#include "spectral_solve.h"

namespace lbeh {
using namespace lbeh_spectral;

namespace {

constexpr int kSB = 256;  // threads per block of the spectral solve

template <typename T> struct AxisDev {
  int n, nrad, W, ld;
  int rad[kMaxStages];
  const C2<T> *w;  // roots exp(-2 pi i t / n)
  const T *s;      // symbol 2 (1 - cos(2 pi k / n))
};

template <typename T> struct SArgs {
  PArgs<T> pa;  // potential, charge, field, solver state, barrier (residual_site)
  Level<T> L0;  // level-0 descriptor: faces from eps, residual into b (= r)
  AxisDev<T> ax[3];
  Grid3 g;
  T *r, *p, *q, *e, *w;
  T inv_eref_n;  // 1 / (eps_ref N)
};

// One lattice pass along axis A over every tile owned by this block: stage
// the tile through `load`, transform each pair of lines (forward; with `fuse`
// also the symbol scaling and the second transform), write through `store`.
template <typename T, class Load, class Store>
__device__ void tile_pass(const SArgs<T> &a, int A, bool fuse, C2<T> *buf, Load load, Store store) {
  const AxisDev<T> P = a.ax[A];
  const Grid3 g = a.g;
  const int N = P.n, W = P.W, pairs = W >> 1, ld = P.ld;
  C2<T> *bA = buf, *bB = buf + pairs * ld;
  const int nt = tile_count(g, A, W);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
  const int nm = warp < pairs ? (pairs - warp + nw - 1) / nw : 0;  // line pairs of this warp
  for (int t = blockIdx.x; t < nt; t += gridDim.x) {
    for (int el = threadIdx.x; el < W * N; el += blockDim.x) {
      int l, pos;
      if (A == 0) {  // consecutive threads along the row
        l = el / N;
        pos = el - l * N;
      } else {  // consecutive threads along x
        pos = el / W;
        l = el - pos * W;
      }
      bool ok;
      const long long gi = tile_index(g, A, W, t, l, pos, ok);
      reinterpret_cast<T *>(bA + (l >> 1) * ld + pos)[l & 1] = ok ? load(gi) : T(0);
    }
    __syncthreads();
    C2<T> *in = bA, *out = bB;
    for (int rep = 0; rep < (fuse ? 2 : 1); ++rep) {
      int Ns = 1;
      for (int s = 0; s < P.nrad; ++s) {
        const int R = P.rad[s], nb = N / R;
        for (int j = lane; j < nm * nb; j += 32) {
          const int mi = j / nb, jj = j - mi * nb;
          const int m = warp + mi * nw;
          stage_bfly(in + m * ld, out + m * ld, P.w, N, R, Ns, jj);
        }
        __syncwarp();
        Ns *= R;
        C2<T> *tp = in;
        in = out;
        out = tp;
      }
      if (fuse && rep == 0) {
        // Hartley values of both lines, times the inverse symbol, packed again
        for (int mi = 0; mi < nm; ++mi) {
          const int m = warp + mi * nw;
          int kxa, kxb, ky;
          zline_k(g, W, t, 2 * m, kxa, ky);
          zline_k(g, W, t, 2 * m + 1, kxb, ky);
          for (int k = lane; k <= N / 2; k += 32) {
            const Split<T> sp = pair_split(in + m * ld, N, k);
            const int kn = k == 0 ? 0 : N - k;
            const T *sx = a.ax[0].s, *sy = a.ax[1].s, *sz = a.ax[2].s;
            const T sa = kxa < g.nx ? inv_symbol(kxa, ky, k, sx, sy, sz, a.inv_eref_n) : T(0);
            const T sb = kxb < g.nx ? inv_symbol(kxb, ky, k, sx, sy, sz, a.inv_eref_n) : T(0);
            const T sa2 = kxa < g.nx ? inv_symbol(kxa, ky, kn, sx, sy, sz, a.inv_eref_n) : T(0);
            const T sb2 = kxb < g.nx ? inv_symbol(kxb, ky, kn, sx, sy, sz, a.inv_eref_n) : T(0);
            out[m * ld + k] = C2<T>{sp.ak * sa, sp.bk * sb};
            out[m * ld + kn] = C2<T>{sp.an * sa2, sp.bn * sb2};
          }
        }
        __syncwarp();
        C2<T> *tp = in;
        in = out;
        out = tp;
      }
    }
    __syncthreads();
    for (int el = threadIdx.x; el < W * N; el += blockDim.x) {
      int l, pos;
      if (A == 0) {
        l = el / N;
        pos = el - l * N;
      } else {
        pos = el / W;
        l = el - pos * W;
      }
      bool ok;
      const long long gi = tile_index(g, A, W, t, l, pos, ok);
      if (ok) {
        const Split<T> sp = pair_split(in + (l >> 1) * ld, N, pos);
        store(gi, (l & 1) ? sp.bk : sp.ak);
      }
    }
    __syncthreads();
  }
}

// q = A z + beta q, p = z + beta p over the team's cells; returns the block's
// share of p.q
template <typename T, bool DFM>
__device__ double matvec_update(const SArgs<T> &a, const T *z, T beta, bool first, double *sh) {
  const Level<T> L0 = a.L0;
  const Dims d = L0.dims();
  const long long G = (long long)gridDim.x * blockDim.x;
  SumAcc<DFM> acc;
  for (Walk wk(blockIdx.x * (long long)blockDim.x + threadIdx.x, G, d.nx, d.ny); wk.z < d.nz; wk.next()) {
    const Nbr c = nbr(d, wk.u, wk.y, wk.z);
    const Faces<T> f = faces(L0, c.i, c.xp, c.xm, c.yp, c.ym, c.zp, c.zm);
    const T zi = z[c.i];
    const T Az = f.xp * (z[c.xp] - zi) + f.xm * (z[c.xm] - zi) + f.yp * (z[c.yp] - zi) + f.ym * (z[c.ym] - zi) +
                 f.zp * (z[c.zp] - zi) + f.zm * (z[c.zm] - zi);
    const T pn = first ? zi : zi + beta * a.p[c.i];
    const T qn = first ? Az : Az + beta * a.q[c.i];
    a.p[c.i] = pn;
    a.q[c.i] = qn;
    acc.add(pn * qn);
  }
  return block_sum_n(acc.get(), sh);
}

template <typename T, bool DFM>
__global__ void __launch_bounds__(kSB, 2) k_spectral(SArgs<T> a) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ double sh[kSB];
  C2<T> *buf = reinterpret_cast<C2<T> *>(smem_raw);
  const PArgs<T> &pa = a.pa;
  const GridTeam tm{pa.bar, pa.status, pa.spin_limit};
  const Level<T> L0 = a.L0;
  const Dims d = L0.dims();
  const long long N = d.N;
  const long long G = tm.size(), gt = tm.rank();
  const int nb = tm.nblocks();
  PDev *st = pa.st;
  const int have_prev = st->have_prev;

  // initial guess 2 phi(t-1) - phi(t-2), sum of q
  SumAcc<DFM> sq;
  for (long long i = gt; i < N; i += G) {
    if constexpr (DFM) {
      const DF pv{pa.phi_hi[i], pa.phi_lo[i]};
      if (have_prev) {
        const DF gv = df_sub(DF{2.f * pv.hi, 2.f * pv.lo}, DF{pa.prev_hi[i], pa.prev_lo[i]});
        pa.phi_hi[i] = gv.hi;
        pa.phi_lo[i] = gv.lo;
      }
      pa.prev_hi[i] = pv.hi;
      pa.prev_lo[i] = pv.lo;
    } else {
      const double pv = pa.phi[i];
      if (have_prev) pa.phi[i] = 2.0 * pv - pa.prev[i];
      pa.prev[i] = pv;
    }
    sq.add(pa.q[i]);
  }
  {
    const double v = block_sum_n(sq.get(), sh);
    if (threadIdx.x == 0) pa.part[blockIdx.x] = v;
  }
  if (!tm.sync()) return;
  const double qbar = sum_partials(pa.part, nb, sh) / double(N);
  const DF qbar_df = df_split(qbar);

  const double tol = st->tol;
  const int max_iter = st->max_iter;
  const bool carry = tol >= kTrustTol;
  int it = 0;
  double bn = 0.0, rr = 0.0, shift = 0.0;
  bool have_e = false, exact = true;
  for (int outer = 0;; ++outer) {
    // exact residual r = b - A phi (FP64 / double-float), |r|^2, |b|^2, sum phi
    double r2, b2, ps;
    if (!residual_pass<T, DFM>(pa, tm, L0, qbar, qbar_df, sh, r2, b2, ps)) return;
    if (outer == 0) bn = b2;
    rr = bn > 0.0 ? sqrt(r2 / bn) : 0.0;
    exact = true;
    shift = ps / double(N);
    have_e = false;
    if (rr < tol || it >= max_iter || !isfinite(rr)) break;
    const double rr_start = rr;
    // conjugate gradients on A e = r
    double rho_old = 1.0, alpha = 0.0, sum_e = 0.0;
    bool first = true;
    for (;;) {
      // U: update r and e, Hartley pass along x of r into w
      SumAcc<DFM> sr, se;
      const T al = T(alpha);
      const bool upd = !first, he = have_e;
      tile_pass<T>(
          a, 0, false, buf,
          [&](long long i) {
            T rv = a.r[i];
            if (upd) {
              rv -= al * a.q[i];
              a.r[i] = rv;
              const T ev = (he ? a.e[i] : T(0)) + al * a.p[i];
              a.e[i] = ev;
              se.add(ev);
            }
            sr.add(rv * rv);
            return rv;
          },
          [&](long long i, T v) { a.w[i] = v; });
      if (upd) have_e = true;
      {
        const double v0 = block_sum_n(sr.get(), sh);
        const double v1 = block_sum_n(se.get(), sh);
        if (threadIdx.x == 0) {
          pa.part[blockIdx.x] = v0;
          pa.part[nb + blockIdx.x] = v1;
        }
      }
      if (!tm.sync()) return;
      r2 = sum_partials(pa.part, nb, sh);
      if (have_e) sum_e = sum_partials(pa.part + nb, nb, sh);
      if (upd) {
        ++it;
        rr = bn > 0.0 ? sqrt(r2 / bn) : 0.0;
        exact = false;
        if (rr < tol || it >= max_iter || !isfinite(rr)) break;
      }
      // preconditioner: Y, Z (scale), Y, X passes on w
      tile_pass<T>(
          a, 1, false, buf, [&](long long i) { return a.w[i]; }, [&](long long i, T v) { a.w[i] = v; });
      if (!tm.sync()) return;
      tile_pass<T>(
          a, 2, true, buf, [&](long long i) { return a.w[i]; }, [&](long long i, T v) { a.w[i] = v; });
      if (!tm.sync()) return;
      tile_pass<T>(
          a, 1, false, buf, [&](long long i) { return a.w[i]; }, [&](long long i, T v) { a.w[i] = v; });
      if (!tm.sync()) return;
      SumAcc<DFM> srz;
      tile_pass<T>(
          a, 0, false, buf, [&](long long i) { return a.w[i]; },
          [&](long long i, T v) {
            a.w[i] = v;
            srz.add(a.r[i] * v);
          });
      {
        const double v = block_sum_n(srz.get(), sh);
        if (threadIdx.x == 0) pa.part[blockIdx.x] = v;
      }
      if (!tm.sync()) return;
      const double rho = sum_partials(pa.part, nb, sh);
      const double beta = first ? 0.0 : rho / rho_old;
      // F: search direction and its image
      {
        const double v = matvec_update<T, DFM>(a, a.w, T(beta), first, sh);
        if (threadIdx.x == 0) pa.part[blockIdx.x] = v;
      }
      if (!tm.sync()) return;
      const double pq = sum_partials(pa.part, nb, sh);
      alpha = pq != 0.0 ? rho / pq : 0.0;
      rho_old = rho;
      first = false;
    }
    shift += sum_e / double(N);
    if (it >= max_iter || !isfinite(rr) || (carry && rr + kEstErr * rr_start < tol)) break;
    // apply the correction and check it with an exact residual
    for (long long i = gt; i < N; i += G) {
      if constexpr (DFM) {
        const DF s = df_add(DF{pa.phi_hi[i], pa.phi_lo[i]}, DF{float(a.e[i]), 0.f});
        const DF v = df_sub(s, df_split(shift));
        pa.phi_hi[i] = v.hi;
        pa.phi_lo[i] = v.lo;
      } else {
        pa.phi[i] = pa.phi[i] + double(a.e[i]) - shift;
      }
    }
    have_e = false;
    if (!tm.sync()) return;
  }
  // phi += e (when pending), mean-free
  const bool zero = bn == 0.0;
  const DF shift_df = df_split(shift);
  for (long long i = gt; i < N; i += G) {
    if constexpr (DFM) {
      DF v{0.f, 0.f};
      if (!zero) {
        v = DF{pa.phi_hi[i], pa.phi_lo[i]};
        if (have_e) v = df_add(v, DF{float(a.e[i]), 0.f});
        v = df_sub(v, shift_df);
      }
      pa.phi_hi[i] = v.hi;
      pa.phi_lo[i] = v.lo;
    } else {
      pa.phi[i] = zero ? 0.0 : pa.phi[i] + (have_e ? double(a.e[i]) : 0.0) - shift;
    }
  }
  if (gt == 0) {
    st->mean_q = qbar;
    st->mean_phi = shift;
    st->bnorm2 = bn;
    st->relres = rr;
    st->iters = it;
    st->total_iters += it;
    const int fail = !(rr < tol);  // not converged, or not finite
    st->notconv = fail;
    st->cond = 0;
    st->zero = zero;
    st->have_prev = 1;
    if (fail) atomicOr(pa.status, ST_POISSON);
    if (!isfinite(rr)) atomicOr(pa.status, ST_NONFINITE);
  }
  (void)exact;
}

template <typename T> std::vector<C2<T>> roots_of(int n) {
  std::vector<C2<T>> w(n);
  for (int t = 0; t < n; ++t) {
    const double ang = -2.0 * M_PI * double(t) / double(n);
    w[t] = C2<T>{T(std::cos(ang)), T(std::sin(ang))};
  }
  return w;
}

}  // namespace

struct Spectral {
  int fp64 = 0;
  int grid = 0;
  size_t smem = 0;
  std::vector<void *> allocs;
  void *r = nullptr, *p = nullptr, *q = nullptr, *e = nullptr, *w = nullptr;
  void *tw[3] = {nullptr, nullptr, nullptr}, *sym[3] = {nullptr, nullptr, nullptr};
  int n[3] = {0, 0, 0}, W[3] = {0, 0, 0}, nrad[3] = {0, 0, 0};
  int rad[3][kMaxStages] = {};
  double eps_ref = 1.0;
};

bool spectral_supported(const Dims &d, int fp64) {
  int rad[kMaxStages];
  const int lim = fp64 ? 256 : kMaxN;
  for (int n : {d.nx, d.ny, d.nz})
    if (n < 2 || n > lim || !factorize(n, rad)) return false;
  return true;
}

template <typename T> static bool spectral_setup(Spectral *s, const Dims &d) {
  auto dal = [&](size_t bytes) -> void * {
    void *ptr = nullptr;
    if (cudaMalloc(&ptr, bytes) != cudaSuccess) return nullptr;
    s->allocs.push_back(ptr);
    return ptr;
  };
  const size_t nb = sizeof(T) * (size_t)d.N;
  if (!(s->r = dal(nb)) || !(s->p = dal(nb)) || !(s->q = dal(nb)) || !(s->e = dal(nb)) || !(s->w = dal(nb)))
    return false;
  const int ns[3] = {d.nx, d.ny, d.nz};
  size_t smem = 0;
  for (int A = 0; A < 3; ++A) {
    const int n = ns[A];
    s->n[A] = n;
    s->nrad[A] = factorize(n, s->rad[A]);
    int W = 32;  // lines per tile: the largest of 32, 16, 8 whose tile fits 40 KB
    while (W > 8 && 2 * (W / 2) * (n + 1) * sizeof(C2<T>) > 40 * 1024) W /= 2;
    s->W[A] = W;
    smem = std::max(smem, 2 * (size_t)(W / 2) * (n + 1) * sizeof(C2<T>));
    std::vector<C2<T>> w = roots_of<T>(n);
    std::vector<T> sy(n);
    for (int k = 0; k < n; ++k) sy[k] = T(2.0 * (1.0 - std::cos(2.0 * M_PI * double(k) / double(n))));
    if (!(s->tw[A] = dal(sizeof(C2<T>) * n)) || !(s->sym[A] = dal(sizeof(T) * n))) return false;
    if (cudaMemcpy(s->tw[A], w.data(), sizeof(C2<T>) * n, cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemcpy(s->sym[A], sy.data(), sizeof(T) * n, cudaMemcpyHostToDevice) != cudaSuccess)
      return false;
  }
  s->smem = smem;
  constexpr bool DFM = std::is_same<T, float>::value;
  if (!raise_smem_limit((const void *)k_spectral<T, DFM>, smem)) return false;
  int dev = 0, nsm = 0, coop = 0, per = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, dev);
  if (!coop || cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_spectral<T, DFM>, kSB, smem) != cudaSuccess ||
      per < 1) {
    cudaGetLastError();
    return false;
  }
  s->grid = nsm * std::min(per, 4);
  return true;
}

Spectral *spectral_create(const Ctx &c, int fp64, double eps_ref) {
  if (!spectral_supported(c.d, fp64)) return nullptr;
  Spectral *s = new Spectral;
  s->fp64 = fp64;
  s->eps_ref = eps_ref;
  const bool ok = fp64 ? spectral_setup<double>(s, c.d) : spectral_setup<float>(s, c.d);
  if (!ok) {
    spectral_destroy(s);
    return nullptr;
  }
  return s;
}

void spectral_destroy(Spectral *s) {
  if (!s) return;
  for (void *a : s->allocs) cudaFree(a);
  delete s;
}

template <typename T, bool DFM> static int launch(Spectral *s, const Ctx &c, const PArgs<T> &pa, cudaStream_t st) {
  SArgs<T> a{};
  a.pa = pa;
  Level<T> L0;
  L0.nx = c.d.nx;
  L0.ny = c.d.ny;
  L0.nz = c.d.nz;
  L0.N = c.d.N;
  L0.eps = (const T *)c.eps;
  L0.b = (T *)s->r;
  a.L0 = L0;
  for (int A = 0; A < 3; ++A) {
    AxisDev<T> &P = a.ax[A];
    P.n = s->n[A];
    P.nrad = s->nrad[A];
    P.W = s->W[A];
    P.ld = s->n[A] + 1;
    for (int k = 0; k < kMaxStages; ++k) P.rad[k] = s->rad[A][k];
    P.w = (const C2<T> *)s->tw[A];
    P.s = (const T *)s->sym[A];
  }
  a.g = Grid3{c.d.nx, c.d.ny, c.d.nz};
  a.r = (T *)s->r;
  a.p = (T *)s->p;
  a.q = (T *)s->q;
  a.e = (T *)s->e;
  a.w = (T *)s->w;
  a.inv_eref_n = T(1.0 / (s->eps_ref * double(c.d.N)));
  if (cudaMemsetAsync(pa.bar, 0, sizeof(Bar), st) != cudaSuccess) return -1;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(s->grid);
  cfg.blockDim = dim3(kSB);
  cfg.dynamicSmemBytes = s->smem;
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeCooperative;
  attr[0].val.cooperative = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  count_launch();
  return cudaLaunchKernelEx(&cfg, k_spectral<T, DFM>, a) == cudaSuccess ? 0 : -1;
}

int spectral_launch_f64(Spectral *s, const Ctx &c, const PArgs<double> &pa, cudaStream_t st) {
  return launch<double, false>(s, c, pa, st);
}
int spectral_launch_f32(Spectral *s, const Ctx &c, const PArgs<float> &pa, cudaStream_t st) {
  return launch<float, true>(s, c, pa, st);
}
int spectral_grid(const Spectral *s) { return s->grid; }

}  // namespace lbeh
