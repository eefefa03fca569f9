// Host driver of the spectral transform core (csrc/spectral.cuh) for the
// tests: the line transform, and the five lattice passes with the same tile
// staging and index helpers as the device kernels, run block by block.
#include <cmath>
#include <vector>

#include "spectral.cuh"
using namespace lbeh_spectral;

template <int A>
static void pass_host(float *u, const Grid3 &g, int N, const std::vector<cf> &w, bool fuse, float inv_eps0_n,
                      const float *cx, const float *cy, const float *cz) {
  std::vector<float> tile(kTileLines * N), line(N), out(N);
  std::vector<cf> b0(N), b1(N);
  const int nt = tile_count<A>(g);
  for (int t = 0; t < nt; ++t) {
    for (int l = 0; l < kTileLines; ++l)
      for (int p = 0; p < N; ++p) {
        bool ok;
        const long long gi = tile_index<A>(g, t, l, p, ok);
        tile[l * N + p] = ok ? u[gi] : 0.f;
      }
    for (int l = 0; l < kTileLines; ++l) {
      dht_host(&tile[l * N], out.data(), N, w.data(), b0.data(), b1.data());
      for (int p = 0; p < N; ++p) tile[l * N + p] = out[p];
      if (A == 2 && fuse) {
        const int xt = (g.nx + kTileLines - 1) / kTileLines;
        const int kx = (t % xt) * kTileLines + l, ky = t / xt;
        if (kx < g.nx)
          for (int p = 0; p < N; ++p) {
            const float lam = lap_symbol(g, kx, ky, p, cx, cy, cz);
            tile[l * N + p] = (kx == 0 && ky == 0 && p == 0) ? 0.f : tile[l * N + p] * inv_eps0_n / lam;
          }
        dht_host(&tile[l * N], out.data(), N, w.data(), b0.data(), b1.data());
        for (int p = 0; p < N; ++p) tile[l * N + p] = out[p];
      }
    }
    for (int l = 0; l < kTileLines; ++l)
      for (int p = 0; p < N; ++p) {
        bool ok;
        const long long gi = tile_index<A>(g, t, l, p, ok);
        if (ok) u[gi] = tile[l * N + p];
      }
  }
}

static std::vector<cf> roots(int n) {
  std::vector<cf> w(n);
  for (int t = 0; t < n; ++t) {
    const double a = -2.0 * M_PI * t / n;
    w[t] = cf{float(std::cos(a)), float(std::sin(a))};
  }
  return w;
}
static std::vector<float> symb(int n) {
  std::vector<float> c(n);
  for (int k = 0; k < n; ++k) c[k] = float(2.0 * (1.0 - std::cos(2.0 * M_PI * k / n)));
  return c;
}

extern "C" int precond_host(float *u, int nx, int ny, int nz, double eps0) {
  int r[kMaxStages];
  if (!factorize(nx, r) || !factorize(ny, r) || !factorize(nz, r)) return -1;
  Grid3 g{nx, ny, nz};
  auto wx = roots(nx), wy = roots(ny), wz = roots(nz);
  auto cx = symb(nx), cy = symb(ny), cz = symb(nz);
  const float inv = float(1.0 / (eps0 * double(nx) * ny * nz));
  pass_host<0>(u, g, nx, wx, false, 0.f, nullptr, nullptr, nullptr);
  pass_host<1>(u, g, ny, wy, false, 0.f, nullptr, nullptr, nullptr);
  pass_host<2>(u, g, nz, wz, true, inv, cx.data(), cy.data(), cz.data());
  pass_host<1>(u, g, ny, wy, false, 0.f, nullptr, nullptr, nullptr);
  pass_host<0>(u, g, nx, wx, false, 0.f, nullptr, nullptr, nullptr);
  return 0;
}

extern "C" int dht_line(const float *x, float *h, int N) {
  int rad[kMaxStages];
  if (!factorize(N, rad)) return -1;
  std::vector<cf> w = roots(N), b0(N), b1(N);
  dht_host(x, h, N, w.data(), b0.data(), b1.data());
  return 0;
}
