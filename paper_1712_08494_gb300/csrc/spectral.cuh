// Constant-coefficient inverse z = (eps0 L)^-1 r of the periodic seven-point
// Laplacian L by separable discrete Hartley transforms: the inner solve of
// the spectral split of Sec. II.D (eps0 L phi^{k+1} = b - div((eps - eps0)
// grad phi^k)) and the preconditioner of a conjugate-gradient solve of the
// variable-permittivity equation.  The discrete Hartley transform H[k] =
// Re F[k] - Im F[k] of a real line is real, is its own inverse up to 1/N and,
// applied along x, y and z, diagonalises L with the eigenvalues
// Lambda(k) = -sum_a 2 (1 - cos(2 pi k_a / n_a)).
//
// Line transform: mixed-radix Stockham FFT (radices 8, 4, 2 with explicit
// butterflies, 3, 5, 7 generic) of the real line.  Lattice passes: tiles of
// 32 lines of the pass axis staged in shared memory with coalesced global
// accesses; five passes H_x, H_y, [H_z, scale, H_z], H_y, H_x.
//
// Header only; the step does not call it yet (the multigrid solves Sec. II.B).
// The same line and tile functions run on the host in the tests.
#pragma once
#ifndef LBEH_SPEC_HD
#ifdef __CUDACC__
#define LBEH_SPEC_HD __host__ __device__ __forceinline__
#else
#define LBEH_SPEC_HD inline
#endif
#endif

namespace lbeh_spectral {

struct cf {
  float x, y;
};
LBEH_SPEC_HD cf cadd(cf a, cf b) { return cf{a.x + b.x, a.y + b.y}; }
LBEH_SPEC_HD cf cmul(cf a, cf b) { return cf{a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x}; }

constexpr int kMaxStages = 12;
constexpr int kMaxN = 512;

// radices of N (from {8, 4, 2, 3, 5, 7}); returns the count, 0 if N has
// another prime factor or exceeds kMaxN
LBEH_SPEC_HD int factorize(int N, int *rad) {
  if (N < 1 || N > kMaxN) return 0;
  int m = 0, n = N;
  const int order[6] = {8, 4, 2, 3, 5, 7};
  for (int t = 0; t < 6; ++t)
    while (n % order[t] == 0 && m < kMaxStages) {
      rad[m++] = order[t];
      n /= order[t];
    }
  return n == 1 ? m : 0;
}

// small DFTs (forward, exp(-2 pi i / R) convention); generic for 3, 5, 7
LBEH_SPEC_HD cf mul_mi(cf a) { return cf{a.y, -a.x}; }  // a * (-i)
template <int R> LBEH_SPEC_HD void dft_small(cf *v, const cf *w, int stride) {
  cf o[R];
  for (int a = 0; a < R; ++a) {
    cf s = v[0];
    for (int b = 1; b < R; ++b) s = cadd(s, cmul(v[b], w[((a * b) % R) * stride]));
    o[a] = s;
  }
  for (int a = 0; a < R; ++a) v[a] = o[a];
}
template <> LBEH_SPEC_HD void dft_small<2>(cf *v, const cf *, int) {
  const cf a = v[0], b = v[1];
  v[0] = cadd(a, b);
  v[1] = cf{a.x - b.x, a.y - b.y};
}
template <> LBEH_SPEC_HD void dft_small<4>(cf *v, const cf *, int) {
  const cf s02 = cadd(v[0], v[2]), d02 = cf{v[0].x - v[2].x, v[0].y - v[2].y};
  const cf s13 = cadd(v[1], v[3]), d13 = mul_mi(cf{v[1].x - v[3].x, v[1].y - v[3].y});
  v[0] = cadd(s02, s13);
  v[2] = cf{s02.x - s13.x, s02.y - s13.y};
  v[1] = cadd(d02, d13);
  v[3] = cf{d02.x - d13.x, d02.y - d13.y};
}
template <> LBEH_SPEC_HD void dft_small<8>(cf *v, const cf *, int) {
  // two radix-4 DFTs of the even and odd samples joined by the eighth roots
  cf e[4] = {v[0], v[2], v[4], v[6]}, o[4] = {v[1], v[3], v[5], v[7]};
  dft_small<4>(e, nullptr, 0);
  dft_small<4>(o, nullptr, 0);
  const float h = 0.70710678118654752f;
  const cf t1 = cf{h * (o[1].x + o[1].y), h * (o[1].y - o[1].x)};  // o1 * exp(-i pi/4)
  const cf t2 = mul_mi(o[2]);                                       // o2 * exp(-i pi/2)
  const cf t3 = cf{h * (o[3].y - o[3].x), -h * (o[3].x + o[3].y)};  // o3 * exp(-3 i pi/4)
  const cf t[4] = {o[0], t1, t2, t3};
  for (int k = 0; k < 4; ++k) {
    v[k] = cadd(e[k], t[k]);
    v[k + 4] = cf{e[k].x - t[k].x, e[k].y - t[k].y};
  }
}

// one butterfly j (0 <= j < N/R) of the Stockham stage with radix R after
// sub-transforms of size Ns; w[t] = exp(-2 pi i t / N)
template <int R> LBEH_SPEC_HD void stage_bfly_r(const cf *in, cf *out, const cf *w, int N, int Ns, int j) {
  cf v[R];
  const int stride = N / R;
  const int jn = j % Ns;
  const int tstep = N / (Ns * R);  // twiddle index unit of this stage
  v[0] = in[j];
  for (int r = 1; r < R; ++r) v[r] = cmul(in[j + r * stride], w[(jn * r * tstep) % N]);
  dft_small<R>(v, w, stride);
  const int idx = (j / Ns) * Ns * R + jn;
  for (int a = 0; a < R; ++a) out[idx + a * Ns] = v[a];
}
LBEH_SPEC_HD void stage_bfly(const cf *in, cf *out, const cf *w, int N, int R, int Ns, int j) {
  switch (R) {
    case 2: stage_bfly_r<2>(in, out, w, N, Ns, j); break;
    case 3: stage_bfly_r<3>(in, out, w, N, Ns, j); break;
    case 4: stage_bfly_r<4>(in, out, w, N, Ns, j); break;
    case 5: stage_bfly_r<5>(in, out, w, N, Ns, j); break;
    case 7: stage_bfly_r<7>(in, out, w, N, Ns, j); break;
    default: stage_bfly_r<8>(in, out, w, N, Ns, j); break;
  }
}

// whole transform on the host (reference driver of the same stages)
inline void dht_host(const float *x, float *h, int N, const cf *w, cf *b0, cf *b1) {
  int rad[kMaxStages];
  const int m = factorize(N, rad);
  for (int i = 0; i < N; ++i) b0[i] = cf{x[i], 0.f};
  cf *in = b0, *out = b1;
  int Ns = 1;
  for (int s = 0; s < m; ++s) {
    for (int j = 0; j < N / rad[s]; ++j) stage_bfly(in, out, w, N, rad[s], Ns, j);
    Ns *= rad[s];
    cf *t = in;
    in = out;
    out = t;
  }
  for (int k = 0; k < N; ++k) h[k] = in[k].x - in[k].y;
}

}  // namespace lbeh_spectral

namespace lbeh_spectral {

constexpr int kTileLines = 32;
constexpr int kWarps = 8;

struct AxisPlan {
  int n;                // line length
  int nrad;             // stages
  int rad[kMaxStages];  // radices
  const cf *w;          // n roots exp(-2 pi i t / n) in global memory
};

struct Grid3 {
  int nx, ny, nz;
};

// element (line l, position p) of tile t along axis A
template <int A> LBEH_SPEC_HD long long tile_index(const Grid3 &g, int t, int l, int p, bool &ok) {
  if (A == 0) {  // lines are rows: line = t*32 + l over (y, z), position = x
    const int line = t * kTileLines + l;
    ok = line < g.ny * g.nz;
    return (long long)line * g.nx + p;
  }
  // lines are columns x0 + l at fixed (z) for A = 1 (position y) or fixed (y) for A = 2 (position z)
  const int xt = (g.nx + kTileLines - 1) / kTileLines;
  const int x = (t % xt) * kTileLines + l;
  const int o = t / xt;  // z for A = 1, y for A = 2
  ok = x < g.nx;
  if (A == 1) return ((long long)o * g.ny + p) * g.nx + x;
  return ((long long)p * g.ny + o) * g.nx + x;
}

template <int A> LBEH_SPEC_HD int tile_count(const Grid3 &g) {
  if (A == 0) return (g.ny * g.nz + kTileLines - 1) / kTileLines;
  const int xt = (g.nx + kTileLines - 1) / kTileLines;
  return xt * (A == 1 ? g.nz : g.ny);
}

// Lambda(k) = -sum_a 2 (1 - cos(2 pi k_a / n_a)) of the seven-point Laplacian
LBEH_SPEC_HD float lap_symbol(const Grid3 &g, int kx, int ky, int kz, const float *cx, const float *cy, const float *cz) {
  return -(cx[kx] + cy[ky] + cz[kz]);
}

}  // namespace lbeh_spectral

#ifdef __CUDACC__
namespace lbeh_spectral {

// one warp transforms line l of the staged tile in place (real -> real)
__device__ __forceinline__ void warp_line_dht(float *tile_line, int stride, const AxisPlan &P, cf *b0, cf *b1,
                                              int lane) {
  const int N = P.n;
  for (int i = lane; i < N; i += 32) b0[i] = cf{tile_line[i * stride], 0.f};
  __syncwarp();
  cf *in = b0, *out = b1;
  int Ns = 1;
  for (int s = 0; s < P.nrad; ++s) {
    const int R = P.rad[s];
    for (int j = lane; j < N / R; j += 32) stage_bfly(in, out, P.w, N, R, Ns, j);
    __syncwarp();
    Ns *= R;
    cf *t = in;
    in = out;
    out = t;
  }
  for (int i = lane; i < N; i += 32) tile_line[i * stride] = in[i].x - in[i].y;
  __syncwarp();
}

// pass along axis A; for the z pass (A == 2) with fuse set, the forward
// transform, the scale and the inverse transform run on the staged tile
template <int A>
__global__ void __launch_bounds__(kWarps * 32) k_dht_pass(float *u, Grid3 g, AxisPlan P, bool fuse, float inv_eps0_n,
                                                          const float *cx, const float *cy, const float *cz) {
  extern __shared__ float smem[];
  const int N = P.n;
  float *tile = smem;                                    // [kTileLines][N] (line-major)
  cf *bufs = reinterpret_cast<cf *>(smem + kTileLines * N);  // per warp 2 N complex
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  cf *b0 = bufs + warp * 2 * N, *b1 = b0 + N;
  const int ntiles = tile_count<A>(g);
  for (int t = blockIdx.x; t < ntiles; t += gridDim.x) {
    // stage: consecutive threads read consecutive addresses
    for (int e = threadIdx.x; e < kTileLines * N; e += blockDim.x) {
      int l, p;
      if (A == 0) {
        l = e / N;
        p = e % N;
      } else {
        l = e % kTileLines;
        p = e / kTileLines;
      }
      bool ok;
      const long long gi = tile_index<A>(g, t, l, p, ok);
      tile[l * N + p] = ok ? u[gi] : 0.f;
    }
    __syncthreads();
    for (int l = warp; l < kTileLines; l += kWarps) {
      warp_line_dht(tile + l * N, 1, P, b0, b1, lane);
      if (A == 2 && fuse) {
        // position p is kz; (x, y) of the tile line are (kx, ky) after the x and y passes
        const int xt = (g.nx + kTileLines - 1) / kTileLines;
        const int kx = (t % xt) * kTileLines + l, ky = t / xt;
        if (kx < g.nx) {
          for (int p = lane; p < N; p += 32) {
            const float lam = lap_symbol(g, kx, ky, p, cx, cy, cz);
            tile[l * N + p] = (kx == 0 && ky == 0 && p == 0) ? 0.f : tile[l * N + p] * inv_eps0_n / lam;
          }
        }
        __syncwarp();
        warp_line_dht(tile + l * N, 1, P, b0, b1, lane);
      }
    }
    __syncthreads();
    for (int e = threadIdx.x; e < kTileLines * N; e += blockDim.x) {
      int l, p;
      if (A == 0) {
        l = e / N;
        p = e % N;
      } else {
        l = e % kTileLines;
        p = e / kTileLines;
      }
      bool ok;
      const long long gi = tile_index<A>(g, t, l, p, ok);
      if (ok) u[gi] = tile[l * N + p];
    }
    __syncthreads();
  }
}

}  // namespace lbeh_spectral
#endif
