// Host driver of the spectral transform core (csrc/spectral.cuh) for the
// tests: the line transform, and the five lattice passes of the
// preconditioner with the same tile indexing, pairing of real lines into
// complex lines, Hartley split and symbol scaling as the device solver, run
// tile by tile.
#include <cmath>
#include <vector>

#include "spectral.cuh"
using namespace lbeh_spectral;

template <typename T> static std::vector<C2<T>> roots(int n) {
  std::vector<C2<T>> w(n);
  for (int t = 0; t < n; ++t) {
    const double a = -2.0 * M_PI * t / n;
    w[t] = C2<T>{T(std::cos(a)), T(std::sin(a))};
  }
  return w;
}
template <typename T> static std::vector<T> symb(int n) {
  std::vector<T> c(n);
  for (int k = 0; k < n; ++k) c[k] = T(2.0 * (1.0 - std::cos(2.0 * M_PI * k / n)));
  return c;
}

// the Stockham stages of a line plan (the device solver's transform)
template <typename T>
static C2<T> *fft_plan(C2<T> *b0, C2<T> *b1, const LinePlan &P, const std::vector<unsigned> &code,
                       const std::vector<C2<T>> &tw) {
  C2<T> *in = b0, *out = b1;
  for (int s = 0; s < P.nst; ++s) {
    for (int j = 0; j < P.nb[s]; ++j) plan_bfly(P, s, code.data(), tw.data(), in, out, j);
    C2<T> *t = in;
    in = out;
    out = t;
  }
  return in;
}

template <typename T>
static void pass_host(T *u, const Grid3 &g, int A, int W, const std::vector<C2<T>> &, bool fuse, T inv_n,
                      const T *sx, const T *sy, const T *sz) {
  const int N = line_len(g, A);
  LinePlan P;
  std::vector<unsigned> code;
  std::vector<C2<double>> twd;
  build_plan(N, P, code, twd);
  std::vector<C2<T>> tw(twd.size());
  for (size_t k = 0; k < twd.size(); ++k) tw[k] = C2<T>{T(twd[k].x), T(twd[k].y)};
  const int pairs = W / 2;
  std::vector<C2<T>> b0(N), b1(N), Z((size_t)pairs * N);
  const int nt = tile_count(g, A, W);
  for (int t = 0; t < nt; ++t) {
    for (int m = 0; m < pairs; ++m) {
      for (int p = 0; p < N; ++p) {
        bool oa, ob;
        const long long ia = tile_index(g, A, W, t, 2 * m, p, oa);
        const long long ib = tile_index(g, A, W, t, 2 * m + 1, p, ob);
        b0[p] = C2<T>{oa ? u[ia] : T(0), ob ? u[ib] : T(0)};
      }
      C2<T> *r = fft_plan(b0.data(), b1.data(), P, code, tw);
      if (fuse) {
        int kxa, kxb, ky;
        zline_k(g, W, t, 2 * m, kxa, ky);
        zline_k(g, W, t, 2 * m + 1, kxb, ky);
        std::vector<C2<T>> zz(N);
        for (int k = 0; k <= N / 2; ++k) {
          const Split<T> s = pair_split(r, N, k);
          const int kn = k == 0 ? 0 : N - k;
          const T sa = kxa < g.nx ? inv_symbol(kxa, ky, k, sx, sy, sz, inv_n) : T(0);
          const T sb = kxb < g.nx ? inv_symbol(kxb, ky, k, sx, sy, sz, inv_n) : T(0);
          const T sa2 = kxa < g.nx ? inv_symbol(kxa, ky, kn, sx, sy, sz, inv_n) : T(0);
          const T sb2 = kxb < g.nx ? inv_symbol(kxb, ky, kn, sx, sy, sz, inv_n) : T(0);
          zz[k] = C2<T>{s.ak * sa, s.bk * sb};
          zz[kn] = C2<T>{s.an * sa2, s.bn * sb2};
        }
        C2<T> *o = r == b0.data() ? b1.data() : b0.data();
        for (int k = 0; k < N; ++k) o[k] = zz[k];
        r = fft_plan(o, r, P, code, tw);
      }
      for (int p = 0; p < N; ++p) Z[(size_t)m * N + p] = r[p];
    }
    for (int m = 0; m < pairs; ++m)
      for (int p = 0; p < N; ++p) {
        const Split<T> s = pair_split(&Z[(size_t)m * N], N, p);
        bool oa, ob;
        const long long ia = tile_index(g, A, W, t, 2 * m, p, oa);
        const long long ib = tile_index(g, A, W, t, 2 * m + 1, p, ob);
        if (oa) u[ia] = s.ak;
        if (ob) u[ib] = s.bk;
      }
  }
}

template <typename T> static int precond(T *u, int nx, int ny, int nz, double eps_ref, int W) {
  int r[kMaxStages];
  if (!factorize(nx, r) || !factorize(ny, r) || !factorize(nz, r)) return -1;
  Grid3 g{nx, ny, nz};
  auto wx = roots<T>(nx), wy = roots<T>(ny), wz = roots<T>(nz);
  auto cx = symb<T>(nx), cy = symb<T>(ny), cz = symb<T>(nz);
  const T inv = T(1.0 / (eps_ref * double(nx) * ny * nz));
  pass_host<T>(u, g, 0, W, wx, false, T(0), nullptr, nullptr, nullptr);
  pass_host<T>(u, g, 1, W, wy, false, T(0), nullptr, nullptr, nullptr);
  pass_host<T>(u, g, 2, W, wz, true, inv, cx.data(), cy.data(), cz.data());
  pass_host<T>(u, g, 1, W, wy, false, T(0), nullptr, nullptr, nullptr);
  pass_host<T>(u, g, 0, W, wx, false, T(0), nullptr, nullptr, nullptr);
  return 0;
}

extern "C" int precond_host(float *u, int nx, int ny, int nz, double eps_ref, int W) {
  return precond<float>(u, nx, ny, nz, eps_ref, W);
}
extern "C" int precond_host_f64(double *u, int nx, int ny, int nz, double eps_ref, int W) {
  return precond<double>(u, nx, ny, nz, eps_ref, W);
}

extern "C" int dht_line(const float *x, float *h, int N) {
  int rad[kMaxStages];
  if (!factorize(N, rad)) return -1;
  std::vector<cf> w = roots<float>(N), b0(N), b1(N);
  dht_host(x, h, N, w.data(), b0.data(), b1.data());
  return 0;
}

// Hartley transforms of two real lines from one complex transform
extern "C" int dht_pair(const double *a, const double *b, double *ha, double *hb, int N) {
  int rad[kMaxStages];
  if (!factorize(N, rad)) return -1;
  std::vector<C2<double>> w = roots<double>(N), b0(N), b1(N);
  for (int i = 0; i < N; ++i) b0[i] = C2<double>{a[i], b[i]};
  const C2<double> *Z = fft_host(b0.data(), b1.data(), N, w.data());
  for (int k = 0; k < N; ++k) {
    const Split<double> s = pair_split(Z, N, k);
    ha[k] = s.ak;
    hb[k] = s.bk;
  }
  return 0;
}
