// Constant-coefficient inverse z = (eps_ref L)^-1 r of the periodic seven-point
// Laplacian L by separable discrete Hartley transforms.  Sec. II.D solves the
// Poisson equation with a Fourier spectral method; at variable permittivity
// this library uses that constant-coefficient inverse as the preconditioner
// of a conjugate-gradient solve of the flux-form equation (eps_ref is a
// reference permittivity of the box, not the vacuum permittivity of
// Sec. II.B).  The discrete Hartley transform H[k] = Re F[k] - Im F[k] of a
// real line is real and is its own inverse up to 1/N; applied along x, y and z
// it diagonalises L with the eigenvalues
// Lambda(k) = -sum_a 2 (1 - cos(2 pi k_a / n_a)).
//
// Line transforms: mixed-radix Stockham FFT (radices 8, 4, 2 with explicit
// butterflies, 3, 5, 7 generic) of a complex line that packs two real lines
// (z = a + i b); the Hartley transforms of a and b follow from Z[k] and
// Z[N-k]:  H_a[k] = (P[k] + M[N-k]) / 2,  H_b[k] = (M[k] - P[N-k]) / 2 with
// P = Re Z - Im Z and M = Re Z + Im Z.
//
// Lattice passes: a tile of W lines of the pass axis is staged in shared
// memory (W consecutive rows for x; W consecutive x at fixed (z) or (y) for
// the y and z passes, so global accesses are coalesced along x), each warp
// transforms its pairs of lines, and the tile is written back in place.  The
// z pass can apply the symbol and transform again (forward, scale, inverse).
//
// The line and tile functions are __host__ __device__: the tests run them on
// the host with the same index arithmetic as the device solver.
#pragma once
#include <cmath>
#ifndef LBEH_SPEC_HD
#ifdef __CUDACC__
#define LBEH_SPEC_HD __host__ __device__ __forceinline__
#else
#define LBEH_SPEC_HD inline
#endif
#endif

namespace lbeh_spectral {

template <typename T> struct C2 {
  T x, y;
};
template <typename T> LBEH_SPEC_HD C2<T> cadd(C2<T> a, C2<T> b) { return C2<T>{a.x + b.x, a.y + b.y}; }
template <typename T> LBEH_SPEC_HD C2<T> csub(C2<T> a, C2<T> b) { return C2<T>{a.x - b.x, a.y - b.y}; }
template <typename T> LBEH_SPEC_HD C2<T> cmul(C2<T> a, C2<T> b) {
  return C2<T>{a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x};
}
template <typename T> LBEH_SPEC_HD C2<T> mul_mi(C2<T> a) { return C2<T>{a.y, -a.x}; }  // a * (-i)
using cf = C2<float>;

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

// small DFTs (forward, exp(-2 pi i / R) convention); generic for 3, 5, 7 with
// the R-th roots taken from the line's root table w (w[t] = exp(-2 pi i t / N))
template <typename T, int R> struct Dft {
  LBEH_SPEC_HD static void run(C2<T> *v, const C2<T> *w, int stride) {
    C2<T> o[R];
    for (int a = 0; a < R; ++a) {
      C2<T> s = v[0];
      for (int b = 1; b < R; ++b) s = cadd(s, cmul(v[b], w[((a * b) % R) * stride]));
      o[a] = s;
    }
    for (int a = 0; a < R; ++a) v[a] = o[a];
  }
};
template <typename T> struct Dft<T, 2> {
  LBEH_SPEC_HD static void run(C2<T> *v, const C2<T> *, int) {
    const C2<T> a = v[0], b = v[1];
    v[0] = cadd(a, b);
    v[1] = csub(a, b);
  }
};
template <typename T> struct Dft<T, 4> {
  LBEH_SPEC_HD static void run(C2<T> *v, const C2<T> *, int) {
    const C2<T> s02 = cadd(v[0], v[2]), d02 = csub(v[0], v[2]);
    const C2<T> s13 = cadd(v[1], v[3]), d13 = mul_mi(csub(v[1], v[3]));
    v[0] = cadd(s02, s13);
    v[2] = csub(s02, s13);
    v[1] = cadd(d02, d13);
    v[3] = csub(d02, d13);
  }
};
template <typename T> struct Dft<T, 8> {
  LBEH_SPEC_HD static void run(C2<T> *v, const C2<T> *, int) {
    // two radix-4 DFTs of the even and odd samples joined by the eighth roots
    C2<T> e[4] = {v[0], v[2], v[4], v[6]}, o[4] = {v[1], v[3], v[5], v[7]};
    Dft<T, 4>::run(e, nullptr, 0);
    Dft<T, 4>::run(o, nullptr, 0);
    const T h = T(0.70710678118654752440);
    const C2<T> t1{h * (o[1].x + o[1].y), h * (o[1].y - o[1].x)};  // o1 * exp(-i pi/4)
    const C2<T> t2 = mul_mi(o[2]);                                 // o2 * exp(-i pi/2)
    const C2<T> t3{h * (o[3].y - o[3].x), -h * (o[3].x + o[3].y)};  // o3 * exp(-3 i pi/4)
    const C2<T> t[4] = {o[0], t1, t2, t3};
    for (int k = 0; k < 4; ++k) {
      v[k] = cadd(e[k], t[k]);
      v[k + 4] = csub(e[k], t[k]);
    }
  }
};

// one butterfly j (0 <= j < N/R) of the Stockham stage with radix R after
// sub-transforms of size Ns; w[t] = exp(-2 pi i t / N)
template <typename T, int R>
LBEH_SPEC_HD void stage_bfly_r(const C2<T> *in, C2<T> *out, const C2<T> *w, int N, int Ns, int j) {
  C2<T> v[R];
  const int stride = N / R;
  const int jn = j % Ns;
  const int tstep = N / (Ns * R);  // twiddle index unit of this stage
  v[0] = in[j];
  for (int r = 1; r < R; ++r) v[r] = cmul(in[j + r * stride], w[(jn * r * tstep) % N]);
  Dft<T, R>::run(v, w, stride);
  const int idx = (j / Ns) * Ns * R + jn;
  for (int a = 0; a < R; ++a) out[idx + a * Ns] = v[a];
}
template <typename T>
LBEH_SPEC_HD void stage_bfly(const C2<T> *in, C2<T> *out, const C2<T> *w, int N, int R, int Ns, int j) {
  switch (R) {
    case 2: stage_bfly_r<T, 2>(in, out, w, N, Ns, j); break;
    case 3: stage_bfly_r<T, 3>(in, out, w, N, Ns, j); break;
    case 4: stage_bfly_r<T, 4>(in, out, w, N, Ns, j); break;
    case 5: stage_bfly_r<T, 5>(in, out, w, N, Ns, j); break;
    case 7: stage_bfly_r<T, 7>(in, out, w, N, Ns, j); break;
    default: stage_bfly_r<T, 8>(in, out, w, N, Ns, j); break;
  }
}

// ---------------------------------------------------------------- line plans
// Precomputed Stockham stages of one line length, so that a butterfly needs
// no integer division: for stage s with radix R after sub-transforms of size
// Ns, butterfly j (0 <= j < N/R) reads in[j + r N/R] and writes
// out[base_j + a Ns]; code[j] packs base_j (low 16 bits) and the offset of its
// R - 1 twiddles in the stage's twiddle table (high 16 bits).  After the
// twiddles of a stage with a generic radix (3, 5, 7) come its R roots of unity
// exp(-2 pi i t / R).  Radices: 8 while at least 32 butterflies remain per
// stage, then 4, 2, 3, 5, 7.
struct LinePlan {
  int n, nst, ncode, ntw;
  int R[kMaxStages], Ns[kMaxStages], nb[kMaxStages], code_off[kMaxStages], tw_off[kMaxStages];
};

LBEH_SPEC_HD int plan_radices(int N, int *rad) {
  if (N < 1 || N > kMaxN) return 0;
  int m = 0, n = N;
  while (n % 8 == 0 && N / 8 >= 32 && m < kMaxStages) {
    rad[m++] = 8;
    n /= 8;
  }
  const int order[5] = {4, 2, 3, 5, 7};
  for (int t = 0; t < 5; ++t)
    while (n % order[t] == 0 && m < kMaxStages) {
      rad[m++] = order[t];
      n /= order[t];
    }
  return n == 1 ? m : 0;
}

// host: the plan and its tables in FP64 (converted to the compute type by the caller)
template <class CodeVec, class TwVec> inline bool build_plan(int N, LinePlan &P, CodeVec &code, TwVec &tw) {
  int rad[kMaxStages];
  const int m = plan_radices(N, rad);
  if (!m) return false;
  P.n = N;
  P.nst = m;
  code.clear();
  tw.clear();
  const double two_pi = 6.283185307179586476925286766559;
  int Ns = 1;
  for (int s = 0; s < m; ++s) {
    const int R = rad[s], nb = N / R;
    P.R[s] = R;
    P.Ns[s] = Ns;
    P.nb[s] = nb;
    P.code_off[s] = (int)code.size();
    P.tw_off[s] = (int)tw.size();
    for (int jn = 0; jn < Ns; ++jn)
      for (int r = 1; r < R; ++r) {
        const double a = -two_pi * double(jn * r) / double(Ns * R);
        tw.push_back({std::cos(a), std::sin(a)});
      }
    if (R == 3 || R == 5 || R == 7)
      for (int t = 0; t < R; ++t) {
        const double a = -two_pi * double(t) / double(R);
        tw.push_back({std::cos(a), std::sin(a)});
      }
    for (int j = 0; j < nb; ++j) {
      const int jn = j % Ns;
      const unsigned base = unsigned((j / Ns) * Ns * R + jn);
      code.push_back(base | (unsigned(jn * (R - 1)) << 16));
    }
    Ns *= R;
  }
  P.ncode = (int)code.size();
  P.ntw = (int)tw.size();
  return true;
}

// butterfly j of stage s (tables of this stage: code + code_off, tw + tw_off)
template <typename T, int R>
LBEH_SPEC_HD void plan_bfly_r(const C2<T> *in, C2<T> *out, const C2<T> *tw, int Ns, int nb, int j, unsigned code) {
  C2<T> v[R];
  const unsigned base = code & 0xFFFFu, tb = code >> 16;
  v[0] = in[j];
  for (int r = 1; r < R; ++r) v[r] = cmul(in[j + r * nb], tw[tb + r - 1]);
  Dft<T, R>::run(v, tw + Ns * (R - 1), 1);
  for (int a = 0; a < R; ++a) out[base + a * Ns] = v[a];
}
template <typename T>
LBEH_SPEC_HD void plan_bfly(const LinePlan &P, int s, const unsigned *code, const C2<T> *tw, const C2<T> *in,
                            C2<T> *out, int j) {
  const int Ns = P.Ns[s], nb = P.nb[s];
  const unsigned c = code[P.code_off[s] + j];
  const C2<T> *t = tw + P.tw_off[s];
  switch (P.R[s]) {
    case 2: plan_bfly_r<T, 2>(in, out, t, Ns, nb, j, c); break;
    case 3: plan_bfly_r<T, 3>(in, out, t, Ns, nb, j, c); break;
    case 4: plan_bfly_r<T, 4>(in, out, t, Ns, nb, j, c); break;
    case 5: plan_bfly_r<T, 5>(in, out, t, Ns, nb, j, c); break;
    case 7: plan_bfly_r<T, 7>(in, out, t, Ns, nb, j, c); break;
    default: plan_bfly_r<T, 8>(in, out, t, Ns, nb, j, c); break;
  }
}

// Hartley values at positions k and N-k of the two real lines packed in the
// transformed complex line Z: (H_a[k], H_b[k], H_a[N-k], H_b[N-k])
template <typename T> struct Split {
  T ak, bk, an, bn;
};
template <typename T> LBEH_SPEC_HD Split<T> pair_split(const C2<T> *Z, int N, int k) {
  const int kn = k == 0 ? 0 : N - k;
  const C2<T> zk = Z[k], zn = Z[kn];
  const T Pk = zk.x - zk.y, Mk = zk.x + zk.y, Pn = zn.x - zn.y, Mn = zn.x + zn.y;
  return Split<T>{T(0.5) * (Pk + Mn), T(0.5) * (Mk - Pn), T(0.5) * (Pn + Mk), T(0.5) * (Mn - Pk)};
}

// whole transform of one complex line on the host (reference driver of the
// same stages); returns the buffer holding the result
template <typename T> inline C2<T> *fft_host(C2<T> *b0, C2<T> *b1, int N, const C2<T> *w) {
  int rad[kMaxStages];
  const int m = factorize(N, rad);
  C2<T> *in = b0, *out = b1;
  int Ns = 1;
  for (int s = 0; s < m; ++s) {
    for (int j = 0; j < N / rad[s]; ++j) stage_bfly(in, out, w, N, rad[s], Ns, j);
    Ns *= rad[s];
    C2<T> *t = in;
    in = out;
    out = t;
  }
  return in;
}

// Hartley transform of one real line on the host (imaginary part zero)
inline void dht_host(const float *x, float *h, int N, const cf *w, cf *b0, cf *b1) {
  for (int i = 0; i < N; ++i) b0[i] = cf{x[i], 0.f};
  const cf *Z = fft_host(b0, b1, N, w);
  for (int k = 0; k < N; ++k) h[k] = Z[k].x - Z[k].y;
}

// ---------------------------------------------------------------- tiles
struct Grid3 {
  int nx, ny, nz;
};

// Tiles of W lines along axis A.  A = 0: lines are the rows (y, z), tile t
// holds rows t*W .. t*W+W-1.  A = 1 / 2: lines are the columns at fixed z (A =
// 1) or fixed y (A = 2), tile t holds x = xb*W .. xb*W+W-1 with xb = t % xt.
LBEH_SPEC_HD int line_len(const Grid3 &g, int A) { return A == 0 ? g.nx : (A == 1 ? g.ny : g.nz); }
LBEH_SPEC_HD int tile_count(const Grid3 &g, int A, int W) {
  if (A == 0) return (g.ny * g.nz + W - 1) / W;
  const int xt = (g.nx + W - 1) / W;
  return xt * (A == 1 ? g.nz : g.ny);
}
// global index of element (line l, position p) of tile t; ok = line exists
LBEH_SPEC_HD long long tile_index(const Grid3 &g, int A, int W, int t, int l, int p, bool &ok) {
  if (A == 0) {
    const long long line = (long long)t * W + l;
    ok = line < (long long)g.ny * g.nz;
    return line * g.nx + p;
  }
  const int xt = (g.nx + W - 1) / W;
  const int x = (t % xt) * W + l;
  const int o = t / xt;  // z for A = 1, y for A = 2
  ok = x < g.nx;
  if (A == 1) return ((long long)o * g.ny + p) * g.nx + x;
  return ((long long)p * g.ny + o) * g.nx + x;
}
// wavenumbers (kx, ky) of line l of a z-pass tile (after the x and y passes)
LBEH_SPEC_HD void zline_k(const Grid3 &g, int W, int t, int l, int &kx, int &ky) {
  const int xt = (g.nx + W - 1) / W;
  kx = (t % xt) * W + l;
  ky = t / xt;
}

// scale of the symbol step: 1 / (eps_ref Lambda(k) N_sites), zero mode 0;
// s_a[k] = 2 (1 - cos(2 pi k / n_a))
template <typename T>
LBEH_SPEC_HD T inv_symbol(int kx, int ky, int kz, const T *sx, const T *sy, const T *sz, T inv_eref_n) {
  if (kx == 0 && ky == 0 && kz == 0) return T(0);
  return -inv_eref_n / (sx[kx] + sy[ky] + sz[kz]);
}

}  // namespace lbeh_spectral
