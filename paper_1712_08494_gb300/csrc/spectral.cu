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
//   F  p = z + beta p, q = A z + beta q (sums p.q, r.q, q.q).
// The sums of F give |r - alpha q|^2 before the update is made: when it is
// predicted below the target the next U is the update alone with its own
// sums (the x pass of the last iteration would be discarded), and a wrong
// prediction runs the x pass as a phase of its own.  Otherwise the sums of U
// (|r|^2, e) are reduced together with r.z after the X pass.
// Between the forward and the inverse pass along an axis whose lines are
// transformed in registers, the work array holds that axis's frequencies in
// the transform's own storage order; the symbols are stored in that order.
#include <algorithm>
#include <cmath>
#include <type_traits>
#include <vector>

#include "internal.h"
#include "poisson_dev.cuh"
#include "spectral.cuh"
#include "spectral_solve.h"

namespace lbeh {
using namespace lbeh_spectral;

namespace {

constexpr int kSB = 256;  // threads per block of the spectral solve
constexpr int kU = 8;     // elements per thread whose loads are in flight together
// reduction of the residual one conjugate-gradient run in the compute type may
// claim before the exact residual is formed again
template <typename T> constexpr double kInnerReduction = 1e-4;
template <> constexpr double kInnerReduction<double> = 0.0;

template <typename T> struct AxisDev {
  LinePlan P;          // Stockham stages of the line length
  int W, lgW, ld;      // lines per tile (power of two), its log2, padded line stride
  const unsigned *code;  // butterfly codes of the plan
  const C2<T> *tw;       // twiddles of the plan
  const T *s;            // symbol 2 (1 - cos(2 pi k / n))
  int code_at, tw_at, s_at;  // offsets of the three tables in the shared-memory table area
};

template <typename T> struct SArgs {
  PArgs<T> pa;  // potential, charge, field, solver state, barrier (residual_site)
  Level<T> L0;  // level-0 descriptor: faces from eps, residual into b (= r)
  AxisDev<T> ax[3];
  Grid3 g;
  T *r, *p, *q, *e, *w;
  T inv_eref_n;      // 1 / (eps_ref N)
  int ncode, ntw, ns;  // lengths of the shared-memory tables (all axes)
  int xrows;           // x passes on whole rows (x lines transformed in registers)
};

// Per-thread sums of the conjugate-gradient scalars (r.r, r.z, p.q, sum e):
// a thread adds a few dozen terms in the compute type, and blocks and the grid
// add the per-thread sums in FP64; the scalars steer the iteration, and the
// convergence it reports is confirmed by the exact residual.
template <typename T> struct CgAcc {
  T v = T(0);
  __device__ __forceinline__ void add(T x) { v += x; }
  __device__ __forceinline__ double get() const { return double(v); }
};

__device__ __forceinline__ float recip(float x) { return __frcp_rn(x); }
__device__ __forceinline__ double recip(double x) { return 1.0 / x; }
// c / x for the symbol scaling of the register passes: the preconditioner
// only has to be the same symmetric positive operator at every application,
// so FP32 takes the fast division intrinsic (about 2 ulp; x in (0, 12])
__device__ __forceinline__ float sym_div(float c, float x) { return __fdividef(c, x); }
__device__ __forceinline__ double sym_div(double c, double x) { return c / x; }

// Fixed-order sums of M values at once: a shared-memory tree over the block
// whose levels add all M values (the FP64 additions of M separate trees, but
// one set of barriers); only the active threads of a level add (the FP64 rate
// of the target is low).  sh holds M kSB doubles.
template <int M> __device__ __forceinline__ void block_sum_m(double (&v)[M], double *sh) {
#pragma unroll
  for (int m = 0; m < M; ++m) sh[m * kSB + threadIdx.x] = v[m];
  __syncthreads();
  for (int w = blockDim.x / 2; w > 0; w >>= 1) {
    if (threadIdx.x < w)
#pragma unroll
      for (int m = 0; m < M; ++m) sh[m * kSB + threadIdx.x] += sh[m * kSB + threadIdx.x + w];
    __syncthreads();
  }
#pragma unroll
  for (int m = 0; m < M; ++m) v[m] = sh[m * kSB];
  __syncthreads();
}
// The blocks' sums of M per-thread values into part[m nb + blockIdx.x], and
// after the grid barrier the M grid sums, added by every block in the same
// fixed order (every block holds bitwise the same scalars and takes the same
// branches).
template <int M> __device__ __forceinline__ void put_block_sums(double (&v)[M], double *part, int nb, double *sh) {
  block_sum_m<M>(v, sh);
  if (threadIdx.x == 0)
#pragma unroll
    for (int m = 0; m < M; ++m) part[m * nb + blockIdx.x] = v[m];
}
template <int M>
__device__ __forceinline__ bool sync_sums(const GridTeam &tm, double *part, int nb, double (&v)[M], double *sh) {
  if (!tm.sync()) return false;
#pragma unroll
  for (int m = 0; m < M; ++m) v[m] = 0.0;
  for (int b = threadIdx.x; b < nb; b += blockDim.x)
#pragma unroll
    for (int m = 0; m < M; ++m) v[m] += part[m * nb + b];
  block_sum_m<M>(v, sh);
  return true;
}

// Shared memory of a block, loaded once per launch: the three axes' plans,
// butterfly codes, twiddles and symbols; then the two tile buffers.
// Lines of N = 32 K points (K = 1, 2, 4, 8) are transformed in registers by
// one warp (dif_regs, dit_regs below); its per-lane twiddles live in shared
// memory: kLaneTw slots per lane and axis, K - 1 of W_N^(lane kappa), the five
// cross-lane twiddles of the decimation-in-frequency stages, then the five of
// the decimation-in-time stages (both 1 on a stage's top lanes, so a stage is
// two FMAs and one complex product on every lane, no select).
constexpr int kLaneTw = 17;
__host__ __device__ inline int reg_fft_k(int N) {
  return (N == 32 || N == 64 || N == 128 || N == 256) ? N / 32 : 0;
}
template <typename T> struct Smem {
  LinePlan *P;  // [3]
  unsigned *code;
  C2<T> *tw;
  T *sym;
  C2<T> *lanetw;  // [3][32][kLaneTw]
  C2<T> *bA;      // four tile buffers, one after the other
};
template <typename T> __device__ Smem<T> smem_layout(unsigned char *raw, const SArgs<T> &a) {
  Smem<T> m;
  m.P = reinterpret_cast<LinePlan *>(raw);
  size_t off = (3 * sizeof(LinePlan) + 15) & ~size_t(15);
  m.code = reinterpret_cast<unsigned *>(raw + off);
  off += ((size_t)a.ncode * 4 + 15) & ~size_t(15);
  m.tw = reinterpret_cast<C2<T> *>(raw + off);
  off += ((size_t)a.ntw * sizeof(C2<T>) + 15) & ~size_t(15);
  m.sym = reinterpret_cast<T *>(raw + off);
  off += ((size_t)a.ns * sizeof(T) + 15) & ~size_t(15);
  m.lanetw = reinterpret_cast<C2<T> *>(raw + off);
  off += (size_t)3 * 32 * kLaneTw * sizeof(C2<T>);
  m.bA = reinterpret_cast<C2<T> *>(raw + off);
  return m;
}

__device__ __forceinline__ void sincos_pi(float x, float *s, float *c) { sincospif(x, s, c); }
__device__ __forceinline__ void sincos_pi(double x, double *s, double *c) { sincospi(x, s, c); }
// exp(-2 pi i t / n)
template <typename T> __device__ __forceinline__ C2<T> root(int t, int n) {
  T sn, cs;
  sincos_pi(T(2) * T(t) / T(n), &sn, &cs);
  return C2<T>{cs, -sn};
}
template <typename T> __device__ void load_tables(const SArgs<T> &a, const Smem<T> &m) {
  for (int A = 0; A < 3; ++A) {
    const AxisDev<T> &X = a.ax[A];
    if (threadIdx.x == 0) m.P[A] = X.P;
    for (int k = threadIdx.x; k < X.P.ncode; k += blockDim.x) m.code[X.code_at + k] = X.code[k];
    for (int k = threadIdx.x; k < X.P.ntw; k += blockDim.x) m.tw[X.tw_at + k] = X.tw[k];
    for (int k = threadIdx.x; k < X.P.n; k += blockDim.x) m.sym[X.s_at + k] = X.s[k];
    const int K = reg_fft_k(X.P.n);
    if (K && threadIdx.x < 32) {
      const int lane = threadIdx.x;
      C2<T> *lt = m.lanetw + (A * 32 + lane) * kLaneTw;
      for (int kap = 1; kap < K; ++kap) lt[kap - 1] = root<T>(lane * kap, X.P.n);
      for (int st = 0; st < 5; ++st) {
        const int h = 16 >> st;
        lt[7 + st] = (lane & h) ? root<T>((lane & (h - 1)) * (16 / h), 32) : C2<T>{T(1), T(0)};
        const int h2 = 1 << st;
        lt[12 + st] = (lane & h2) ? root<T>((lane & (h2 - 1)) * (16 / h2), 32) : C2<T>{T(1), T(0)};
      }
    }
  }
  __syncthreads();
}

// Register transforms of one packed line pair z = a + i b of length
// N = 32 K by one warp.  Lane l holds elements l + 32 kappa (kappa < K).
//
// dif_regs (natural order in): K-point DFTs in registers, twiddles
// W_N^(l kappa), then the 32-point DFTs across the lanes by five radix-2
// decimation-in-frequency stages with shuffles.  Lane l, register kappa ends
// with frequency kappa + K bitrev5(l): the storage order of the forward
// passes, written back as it stands (no reordering, no bank conflicts).
//
// dit_regs (storage order in, natural order out): five radix-2
// decimation-in-time stages across the lanes (bit-reversed input; the bottom
// lane's value times W_2h^(l mod h) is exchanged), twiddles W_N^(l kappa),
// K-point DFTs in registers; lane l, register n2 ends with element l + 32 n2.
template <typename T, int K>
__device__ __forceinline__ void dif_regs(C2<T> (&v)[K], const C2<T> *lt, int lane) {
  if constexpr (K > 1) Dft<T, K>::run(v, nullptr, 0);
#pragma unroll
  for (int kap = 1; kap < K; ++kap) v[kap] = cmul(v[kap], lt[kap - 1]);
#pragma unroll
  for (int st = 0; st < 5; ++st) {
    const int h = 16 >> st;
    const T sg = (lane & h) ? T(-1) : T(1);  // bottom lanes take partner - own
    const C2<T> w = lt[7 + st];               // W_2h^(l mod h) on bottom lanes, 1 on top lanes
#pragma unroll
    for (int kap = 0; kap < K; ++kap) {
      C2<T> u;
      u.x = __shfl_xor_sync(0xffffffffu, v[kap].x, h);
      u.y = __shfl_xor_sync(0xffffffffu, v[kap].y, h);
      v[kap] = cmul(C2<T>{fma(sg, v[kap].x, u.x), fma(sg, v[kap].y, u.y)}, w);
    }
  }
}
template <typename T, int K>
__device__ __forceinline__ void dit_regs(C2<T> (&v)[K], const C2<T> *lt, int lane) {
#pragma unroll
  for (int st = 0; st < 5; ++st) {
    const int h = 1 << st;
    const T sg = (lane & h) ? T(-1) : T(1);  // top: own + partner's product, bottom: partner - own product
    const C2<T> w = lt[12 + st];              // W_2h^(l mod h) on bottom lanes, 1 on top lanes
#pragma unroll
    for (int kap = 0; kap < K; ++kap) {
      const C2<T> s = cmul(v[kap], w);
      C2<T> r;
      r.x = __shfl_xor_sync(0xffffffffu, s.x, h);
      r.y = __shfl_xor_sync(0xffffffffu, s.y, h);
      v[kap] = C2<T>{fma(sg, s.x, r.x), fma(sg, s.y, r.y)};
    }
  }
#pragma unroll
  for (int kap = 1; kap < K; ++kap) v[kap] = cmul(v[kap], lt[kap - 1]);
  if constexpr (K > 1) Dft<T, K>::run(v, nullptr, 0);
}

// Hartley values of the two real lines at one frequency from Z(k) and Z(N-k)
// of their packed transform (the arithmetic of pair_split)
template <typename T> __device__ __forceinline__ void split_one(C2<T> z, C2<T> zp, T &ha, T &hb) {
  const T P = z.x - z.y, M = z.x + z.y, Pn = zp.x - zp.y, Mn = zp.x + zp.y;
  ha = T(0.5) * (P + Mn);
  hb = T(0.5) * (M - Pn);
}
// split after dif_regs: the partner N - k of storage slot (l, kappa) sits in
// lane bitrev5(32 - bitrev5(l)), register 0 for kappa = 0, else in lane
// l ^ 31, register K - kappa
template <typename T, int K>
__device__ __forceinline__ void split_perm(const C2<T> (&v)[K], int lane, T (&ha)[K], T (&hb)[K]) {
  const int p0 = int(__brev(unsigned((32 - int(__brev(unsigned(lane)) >> 27)) & 31)) >> 27);
#pragma unroll
  for (int k = 0; k < K; ++k) {
    C2<T> zp;
    if (k == 0) {
      zp.x = __shfl_sync(0xffffffffu, v[0].x, p0);
      zp.y = __shfl_sync(0xffffffffu, v[0].y, p0);
    } else {
      zp.x = __shfl_xor_sync(0xffffffffu, v[K - k].x, 31);
      zp.y = __shfl_xor_sync(0xffffffffu, v[K - k].y, 31);
    }
    split_one(v[k], zp, ha[k], hb[k]);
  }
}
// split after dit_regs (natural order): the partner of l + 32 n2 is lane
// 32 - l, register K - 1 - n2, or for lane 0 its own register (K - n2) mod K
template <typename T, int K>
__device__ __forceinline__ void split_nat(const C2<T> (&v)[K], int lane, T (&ha)[K], T (&hb)[K]) {
  const int pl = (32 - lane) & 31;
#pragma unroll
  for (int k = 0; k < K; ++k) {
    C2<T> u;
    u.x = __shfl_sync(0xffffffffu, v[K - 1 - k].x, pl);
    u.y = __shfl_sync(0xffffffffu, v[K - 1 - k].y, pl);
    split_one(v[k], lane == 0 ? v[(K - k) % K] : u, ha[k], hb[k]);
  }
}

enum PassMode { kFwd = 0, kInv = 1, kFused = 2 };

// symbol scaling of one z line pair in the fused pass: -1 / (eps_ref N (s_x +
// s_y + s_z)), zero for the zero mode and a missing line
template <typename T> struct ScaleZ {
  const T *sz;
  T sa0, sb0, c;
  bool va, vb, nza;  // lines present; line a off the zero mode in x and y
};

// One line pair of the tile in place (X = its packed line in shared memory):
// forward (storage order out), inverse (storage order in, natural out) or
// forward, scaling and inverse; leaves (H_a, H_b) per slot.
template <typename T, int K>
__device__ __forceinline__ void reg_line_pair(C2<T> *X, int mode, const C2<T> *lt, int lane, const ScaleZ<T> &sc) {
  C2<T> v[K];
  T ha[K], hb[K];
#pragma unroll
  for (int k = 0; k < K; ++k) v[k] = X[lane + 32 * k];
  if (mode == kInv) {
    dit_regs<T, K>(v, lt, lane);
    split_nat<T, K>(v, lane, ha, hb);
  } else {
    dif_regs<T, K>(v, lt, lane);
    split_perm<T, K>(v, lane, ha, hb);
    if (mode == kFused) {
#pragma unroll
      for (int k = 0; k < K; ++k) {
        const int s = lane + 32 * k;
        const T z = sc.sz[s];
        const T ca = sc.va && (sc.nza || s != 0) ? sym_div(sc.c, sc.sa0 + z) : T(0);
        const T cb = sc.vb ? sym_div(sc.c, sc.sb0 + z) : T(0);
        v[k] = C2<T>{ha[k] * ca, hb[k] * cb};
      }
      dit_regs<T, K>(v, lt, lane);
      split_nat<T, K>(v, lane, ha, hb);
    }
  }
#pragma unroll
  for (int k = 0; k < K; ++k) X[lane + 32 * k] = C2<T>{ha[k], hb[k]};
}

// adjacent pair (p[i], p[i + 1]) as one aligned vector access (i even)
template <typename T> struct Vec2T;
template <> struct Vec2T<float> {
  using t = float2;
};
template <> struct Vec2T<double> {
  using t = double2;
};
template <typename T> __device__ __forceinline__ void st_pair(T *p, unsigned i, C2<T> v) {
  typename Vec2T<T>::t o;
  o.x = v.x;
  o.y = v.y;
  *reinterpret_cast<typename Vec2T<T>::t *>(p + i) = o;
}

// Asynchronous copies global -> shared (no registers held while in flight):
// one element, or an aligned adjacent pair into one packed slot.
template <typename T> __device__ __forceinline__ void cp_one(T *dst, const T *src) {
  const unsigned d = unsigned(__cvta_generic_to_shared(dst));
  if constexpr (sizeof(T) == 4)
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(d), "l"(src) : "memory");
  else
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(d), "l"(src) : "memory");
}
template <typename T> __device__ __forceinline__ void cp_pair(C2<T> *dst, const T *src) {
  const unsigned d = unsigned(__cvta_generic_to_shared(dst));
  if constexpr (sizeof(T) == 4)
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(d), "l"(src) : "memory");
  else
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(d), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_wait_all() { asm volatile("cp.async.wait_all;\n" ::: "memory"); }
__device__ __forceinline__ void cp_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
__device__ __forceinline__ void cp_wait_newest_pending() { asm volatile("cp.async.wait_group 1;\n" ::: "memory"); }
// line pair (a at ia, b at ib or missing) of array p into packed slot d
template <typename T>
__device__ __forceinline__ void cp_line_pair(C2<T> *d, const T *p, unsigned ia, unsigned ib, bool hb, bool adj) {
  if (adj) {
    cp_pair(d, p + ia);
    return;
  }
  cp_one(&d->x, p + ia);
  if (hb) cp_one(&d->y, p + ib);
  else d->y = T(0);
}

// Tile buffers of a pass: packed line pairs (a + i b) at slot m * ld + pos.
// bA receives the values to transform (and holds the result), bB is the
// aux / ping-pong buffer, bC and bD stage the update's e and p.
template <typename T> struct Bufs {
  C2<T> *A, *B, *C, *D;
  C2<T> *X;  // aux slots (bB) when the lines are transformed in place, else null
};

// Staging functors of one line-pair element: stage() issues the asynchronous
// copies into the tile buffers (line b may be missing: hb false; adj: b is
// the element after a and the pair is aligned, one vector copy); finish()
// runs after the copies have landed and forms the value to transform in bA.
// A pass that needs a second pair of values at its store keeps them in the
// aux slots (register transforms only: the plan stages use bB).
template <typename T> struct LoadW {
  static constexpr bool kFinish = false;
  static constexpr bool kDouble = true;  // no aux slots: tiles can be double-buffered
  const T *w;
  __device__ __forceinline__ void stage(unsigned ia, unsigned ib, bool hb, bool adj, const Bufs<T> &b, int s) const {
    cp_line_pair(b.A + s, w, ia, ib, hb, adj);
  }
  __device__ __forceinline__ void finish(unsigned, unsigned, bool, const Bufs<T> &, int) const {}
};
// stages w and keeps r in the aux slot (the last x pass: r.z at the store)
template <typename T> struct LoadWR {
  static constexpr bool kFinish = false;
  static constexpr bool kDouble = false;
  const T *w, *r;
  __device__ __forceinline__ void stage(unsigned ia, unsigned ib, bool hb, bool adj, const Bufs<T> &b, int s) const {
    cp_line_pair(b.A + s, w, ia, ib, hb, adj);
    if (b.X) cp_line_pair(b.X + s, r, ia, ib, hb, adj);
  }
  __device__ __forceinline__ void finish(unsigned, unsigned, bool, const Bufs<T> &, int) const {}
};
// r -= alpha q and e += alpha p (upd), sums of r^2 and e; stages r
template <typename T> struct LoadU {
  static constexpr bool kFinish = true;
  static constexpr bool kDouble = false;
  T *r, *e;
  const T *q, *p;
  T al;
  bool upd, he;
  CgAcc<T> *sr, *se;
  __device__ __forceinline__ void stage(unsigned ia, unsigned ib, bool hb, bool adj, const Bufs<T> &b, int s) const {
    cp_line_pair(b.A + s, (const T *)r, ia, ib, hb, adj);
    if (upd) {
      cp_line_pair(b.B + s, q, ia, ib, hb, adj);
      cp_line_pair(b.D + s, p, ia, ib, hb, adj);
      if (he) cp_line_pair(b.C + s, (const T *)e, ia, ib, hb, adj);
    }
  }
  __device__ __forceinline__ T fin(unsigned i, T rv, T qv, T ev, T pv) const {
    if (upd) {
      rv -= al * qv;
      r[i] = rv;
      const T en = ev + al * pv;
      e[i] = en;
      se->add(en);
    }
    sr->add(rv * rv);
    return rv;
  }
  __device__ __forceinline__ void finish(unsigned ia, unsigned ib, bool hb, const Bufs<T> &b, int s) const {
    const C2<T> rv = b.A[s];
    const C2<T> qv = upd ? b.B[s] : C2<T>{T(0), T(0)};
    const C2<T> pv = upd ? b.D[s] : C2<T>{T(0), T(0)};
    const C2<T> ev = upd && he ? b.C[s] : C2<T>{T(0), T(0)};
    const T ra = fin(ia, rv.x, qv.x, ev.x, pv.x);
    const T rb = hb ? fin(ib, rv.y, qv.y, ev.y, pv.y) : T(0);
    b.A[s] = C2<T>{ra, rb};
  }
};
template <typename T> struct StoreW {
  T *w;
  __device__ __forceinline__ void operator()(unsigned ia, unsigned ib, bool hb, bool adj, C2<T> v,
                                             const C2<T> *) const {
    if (adj) {
      st_pair(w, ia, v);
      return;
    }
    w[ia] = v.x;
    if (hb) w[ib] = v.y;
  }
};
// stores z and adds r.z (r from the aux slot, else from memory)
template <typename T> struct StoreRZ {
  T *w;
  const T *r;
  CgAcc<T> *acc;
  __device__ __forceinline__ void operator()(unsigned ia, unsigned ib, bool hb, bool, C2<T> v,
                                             const C2<T> *aux) const {
    w[ia] = v.x;
    acc->add((aux ? aux->x : r[ia]) * v.x);
    if (hb) {
      w[ib] = v.y;
      acc->add((aux ? aux->y : r[ib]) * v.y);
    }
  }
};

// One lattice pass along axis A over every tile owned by this block: stage
// the tile's line pairs through `ldr` (asynchronous copies, all in flight
// together), transform them (mode: forward, inverse,
// or forward + symbol scaling + inverse), write through `store`.  Each thread
// stages and stores whole line pairs (a, b): the packed value a + i b is one
// shared-memory word.  Axes of length 32 K (K = 1, 2, 4, 8) are transformed
// in registers (reg_line_pair; the forward passes leave the storage order of
// dif_regs along the axis, the inverse passes read it and restore the natural
// order); other lengths by the Stockham stages of the plan in natural order,
// Hartley values split out at the store.  Element positions advance without
// integer division: for the x pass a thread's (pair, position) steps by the
// block size decomposed once; for the y and z passes the number of pairs
// divides the block size, so each thread keeps its pair and steps its
// position.
template <typename T, class Load, class Store>
__device__ void tile_pass(const SArgs<T> &a, const Smem<T> &sm, int A, int mode, const Load &ldr, Store store) {
  const AxisDev<T> &X = a.ax[A];
  const Grid3 g = a.g;
  const int W = X.W, lgW = X.lgW, pairs = W >> 1, lgP = lgW - 1, ld = X.ld;
  const LinePlan &P = sm.P[A];
  const unsigned *code = sm.code + X.code_at;
  const C2<T> *tw = sm.tw + X.tw_at;
  C2<T> *bA = sm.bA, *bB = sm.bA + pairs * ld;
  const int N = P.n;
  const int regK = reg_fft_k(N);  // register transform of the lines, or the plan's stages
  const int nt = tile_count(g, A, W);
  const int xt = (g.nx + W - 1) >> lgW;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
  const int nm = warp < pairs ? (pairs - warp + nw - 1) / nw : 0;  // line pairs of this warp
  const int B = blockDim.x;
  const int E = pairs * N;  // line-pair elements of a tile
  // x pass: (pair, position) of element tid and the block stride, decomposed once
  const int m0 = threadIdx.x / N, q0 = threadIdx.x - (threadIdx.x / N) * N;
  const int dm = B / N, dq = B - (B / N) * N;
  const unsigned nlines = unsigned(g.ny) * unsigned(g.nz);
  const unsigned sy = unsigned(g.nx), sz = unsigned(g.nx) * unsigned(g.ny);
  // y and z passes: the thread's pair, its first position and position step
  const int myp = threadIdx.x & (pairs - 1), myq = threadIdx.x >> lgP, qstep = B >> lgP;
  const unsigned step = A == 1 ? sy : sz;
  if constexpr (Load::kDouble) {
    if (regK && A != 0) {
      // y and z passes with register transforms: tile t + grid is copied into
      // the other buffer while tile t is transformed and stored
      C2<T> *const slot0 = bA, *const slot1 = bB + pairs * ld;
      const bool adj = (g.nx & 1) == 0;  // even rows: every pair (x, x + 1) is aligned
      auto stage = [&](int t, C2<T> *buf) {
        const int o = t / xt, x = ((t - o * xt) << lgW) + 2 * myp;
        const bool va = x < g.nx, vb = x + 1 < g.nx;
        const unsigned base = (A == 1 ? unsigned(o) * sz : unsigned(o) * sy) + unsigned(x);
        const Bufs<T> bf{buf, nullptr, nullptr, nullptr, nullptr};
        for (int pos = myq; pos < N; pos += qstep) {
          const unsigned i = base + unsigned(pos) * step;
          if (va) ldr.stage(i, i + 1u, vb, adj, bf, myp * ld + pos);
          else buf[myp * ld + pos] = C2<T>{T(0), T(0)};
        }
      };
      if (int(blockIdx.x) < nt) stage(blockIdx.x, slot0);
      cp_commit();
      int k = 0;
      for (int t = blockIdx.x; t < nt; t += gridDim.x, ++k) {
        const int tn = t + gridDim.x;
        if (tn < nt) stage(tn, (k & 1) ? slot0 : slot1);
        cp_commit();
        cp_wait_newest_pending();  // tile t has landed
        __syncthreads();
        C2<T> *cur = (k & 1) ? slot1 : slot0;
        const int o = t / xt, x0 = (t - o * xt) << lgW;
        const C2<T> *lt = sm.lanetw + (A * 32 + lane) * kLaneTw;
        ScaleZ<T> sc{};
        const T *sx = sm.sym + a.ax[0].s_at, *sy_ = sm.sym + a.ax[1].s_at;
        sc.sz = sm.sym + a.ax[2].s_at;
        sc.c = -a.inv_eref_n;
        for (int mi = 0; mi < nm; ++mi) {
          const int m = warp + mi * nw;
          if (mode == kFused) {
            const int kxa = x0 + 2 * m, kxb = kxa + 1, ky = o;
            sc.va = kxa < g.nx;
            sc.vb = kxb < g.nx;
            sc.sa0 = sc.va ? sx[kxa] + sy_[ky] : T(1);
            sc.sb0 = sc.vb ? sx[kxb] + sy_[ky] : T(1);
            sc.nza = (kxa | ky) != 0;
          }
          C2<T> *line = cur + m * ld;
          switch (regK) {
            case 1: reg_line_pair<T, 1>(line, mode, lt, lane, sc); break;
            case 2: reg_line_pair<T, 2>(line, mode, lt, lane, sc); break;
            case 4: reg_line_pair<T, 4>(line, mode, lt, lane, sc); break;
            default: reg_line_pair<T, 8>(line, mode, lt, lane, sc); break;
          }
        }
        __syncthreads();
        const int x = x0 + 2 * myp;
        if (x < g.nx) {
          const unsigned base = (A == 1 ? unsigned(o) * sz : unsigned(o) * sy) + unsigned(x);
          const bool vb = x + 1 < g.nx;
          for (int pos = myq; pos < N; pos += qstep) {
            const unsigned i = base + unsigned(pos) * step;
            store(i, i + 1u, vb, adj, cur[myp * ld + pos], nullptr);
          }
        }
        __syncthreads();  // the buffer is staged again two tiles on
      }
      cp_wait_all();
      return;
    }
  }
  for (int t = blockIdx.x; t < nt; t += gridDim.x) {
    // tile origin: first row (x pass) or (x0, o) with o = z (y pass) or y (z pass)
    const int o = A == 0 ? 0 : t / xt;
    const int x0 = A == 0 ? 0 : (t - o * xt) << lgW;
    const unsigned row0 = unsigned(t) << lgW;
    // staging: every copy of the tile in flight at once (asynchronous copies
    // into the packed slots), then the functor's arithmetic on the tile
    const Bufs<T> bufs{bA, bB, bB + pairs * ld, bB + 2 * pairs * ld, regK ? bB : nullptr};
    if (A == 0) {
      int m = m0, pos = q0;
      for (int e = threadIdx.x; e < E; e += B) {
        const unsigned ra = row0 + 2u * unsigned(m);
        if (ra < nlines)
          ldr.stage(ra * sy + unsigned(pos), (ra + 1u) * sy + unsigned(pos), ra + 1u < nlines, false, bufs,
                    m * ld + pos);
        else
          bA[m * ld + pos] = C2<T>{T(0), T(0)};
        pos += dq;
        m += dm;
        if (pos >= N) {
          pos -= N;
          ++m;
        }
      }
    } else {
      const int x = x0 + 2 * myp;
      const bool va = x < g.nx, vb = x + 1 < g.nx;
      const bool adj = (g.nx & 1) == 0;  // even rows: every pair (x, x + 1) is aligned
      const unsigned base = (A == 1 ? unsigned(o) * sz : unsigned(o) * sy) + unsigned(x);
      for (int pos = myq; pos < N; pos += qstep) {
        const unsigned i = base + unsigned(pos) * step;
        if (va) ldr.stage(i, i + 1u, vb, adj, bufs, myp * ld + pos);
        else bA[myp * ld + pos] = C2<T>{T(0), T(0)};
      }
    }
    cp_wait_all();
    __syncthreads();
    if (Load::kFinish) {
      if (A == 0) {
        int m = m0, pos = q0;
        for (int e = threadIdx.x; e < E; e += B) {
          const unsigned ra = row0 + 2u * unsigned(m);
          if (ra < nlines)
            ldr.finish(ra * sy + unsigned(pos), (ra + 1u) * sy + unsigned(pos), ra + 1u < nlines, bufs, m * ld + pos);
          pos += dq;
          m += dm;
          if (pos >= N) {
            pos -= N;
            ++m;
          }
        }
      } else {
        const int x = x0 + 2 * myp;
        if (x < g.nx) {
          const unsigned base = (A == 1 ? unsigned(o) * sz : unsigned(o) * sy) + unsigned(x);
          for (int pos = myq; pos < N; pos += qstep) {
            const unsigned i = base + unsigned(pos) * step;
            ldr.finish(i, i + 1u, x + 1 < g.nx, bufs, myp * ld + pos);
          }
        }
      }
      __syncthreads();
    }
    const C2<T> *res = bA;  // the transformed line pairs
    if (regK) {
      const C2<T> *lt = sm.lanetw + (A * 32 + lane) * kLaneTw;
      ScaleZ<T> sc{};
      const T *sx = sm.sym + a.ax[0].s_at, *sy_ = sm.sym + a.ax[1].s_at;
      sc.sz = sm.sym + a.ax[2].s_at;
      sc.c = -a.inv_eref_n;
      for (int mi = 0; mi < nm; ++mi) {
        const int m = warp + mi * nw;
        if (mode == kFused) {
          const int kxa = x0 + 2 * m, kxb = kxa + 1, ky = o;
          sc.va = kxa < g.nx;
          sc.vb = kxb < g.nx;
          sc.sa0 = sc.va ? sx[kxa] + sy_[ky] : T(1);
          sc.sb0 = sc.vb ? sx[kxb] + sy_[ky] : T(1);
          sc.nza = (kxa | ky) != 0;
        }
        C2<T> *line = bA + m * ld;
        switch (regK) {
          case 1: reg_line_pair<T, 1>(line, mode, lt, lane, sc); break;
          case 2: reg_line_pair<T, 2>(line, mode, lt, lane, sc); break;
          case 4: reg_line_pair<T, 4>(line, mode, lt, lane, sc); break;
          default: reg_line_pair<T, 8>(line, mode, lt, lane, sc); break;
        }
      }
    } else {
      C2<T> *in = bA, *out = bB;
      for (int rep = 0; rep < (mode == kFused ? 2 : 1); ++rep) {
        for (int s = 0; s < P.nst; ++s) {
          const int nb = P.nb[s];
          for (int mi = 0; mi < nm; ++mi) {
            const int m = warp + mi * nw;
            for (int j = lane; j < nb; j += 32) plan_bfly(P, s, code, tw, in + m * ld, out + m * ld, j);
          }
          __syncwarp();
          C2<T> *tp = in;
          in = out;
          out = tp;
        }
        if (mode == kFused && rep == 0) {
          // scale -1 / (eps_ref N sum_a s_a(k_a)); the zero mode and missing lines get 0
          const T *sx = sm.sym + a.ax[0].s_at, *sy_ = sm.sym + a.ax[1].s_at, *sz_ = sm.sym + a.ax[2].s_at;
          for (int mi = 0; mi < nm; ++mi) {
            const int m = warp + mi * nw;
            const int kxa = x0 + 2 * m, kxb = kxa + 1, ky = o;
            const bool va = kxa < g.nx, vb = kxb < g.nx;
            const T sxa = va ? sx[kxa] + sy_[ky] : T(1), sxb = vb ? sx[kxb] + sy_[ky] : T(1);
            const T c = -a.inv_eref_n;
            for (int k = lane; k <= N / 2; k += 32) {
              const Split<T> sp = pair_split(in + m * ld, N, k);
              const int kn = k == 0 ? 0 : N - k;
              const T szk = sz_[k], szn = sz_[kn];
              const T sa = va && (kxa | ky | k) ? c * recip(sxa + szk) : T(0);
              const T sb = vb ? c * recip(sxb + szk) : T(0);
              const T sa2 = va && (kxa | ky | kn) ? c * recip(sxa + szn) : T(0);
              const T sb2 = vb ? c * recip(sxb + szn) : T(0);
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
      res = in;
    }
    __syncthreads();
    // (H_a, H_b) of slot pos: as it stands after the register transform, else
    // split from the packed transform Z(pos), Z(N - pos)
    auto value = [&](int m, int pos) -> C2<T> {
      if (regK) return res[m * ld + pos];
      const Split<T> sp = pair_split(res + m * ld, N, pos);
      return C2<T>{sp.ak, sp.bk};
    };
    if (A == 0) {
      int m = m0, pos = q0;
      for (int e = threadIdx.x; e < E; e += B) {
        const unsigned ra = row0 + 2u * unsigned(m);
        if (ra < nlines)
          store(ra * sy + unsigned(pos), (ra + 1u) * sy + unsigned(pos), ra + 1u < nlines, false, value(m, pos),
                regK ? bB + m * ld + pos : nullptr);
        pos += dq;
        m += dm;
        if (pos >= N) {
          pos -= N;
          ++m;
        }
      }
    } else {
      const int x = x0 + 2 * myp;
      if (x < g.nx) {
        const unsigned base = (A == 1 ? unsigned(o) * sz : unsigned(o) * sy) + unsigned(x);
        const bool vb = x + 1 < g.nx, adj = (g.nx & 1) == 0;
        for (int pos = myq; pos < N; pos += qstep) {
          const unsigned i = base + unsigned(pos) * step;
          store(i, i + 1u, vb, adj, value(myp, pos), regK ? bB + myp * ld + pos : nullptr);
        }
      }
    }
    __syncthreads();
  }
}

// ---- x passes on whole rows -----------------------------------------------
// A tile of the x pass is W consecutive rows: one contiguous block of W nx
// words of every array.  When the x lines are transformed in registers the
// tile is copied row-major into the tile buffers by 16-byte asynchronous
// copies (every copy of the tile in flight at once), the arithmetic runs on
// 16-byte packs, and the results leave by 16-byte stores.  All of it stays in
// the generic proxy: no proxy fence is needed between the phases.
template <typename T> struct alignas(16) Pack {
  static constexpr int n = 16 / sizeof(T);
  T v[n];
};
template <typename T> __device__ __forceinline__ void cp16(T *dst, const T *src) {
  const unsigned d = unsigned(__cvta_generic_to_shared(dst));
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(d), "l"(src) : "memory");
}
// rows of nw words (nw * sizeof(T) a multiple of 16), global -> shared
template <typename T> __device__ __forceinline__ void cp_rows(T *dst, const T *src, int nw) {
  constexpr int P = Pack<T>::n;
  for (int i = threadIdx.x; i < nw / P; i += blockDim.x) cp16(dst + i * P, src + i * P);
}

enum XKind { kXUpdate = 0, kXForward = 1, kXInverse = 2 };

// One x pass over this block's tiles (K = nx / 32):
//   kXUpdate   r -= alpha q, e += alpha p (upd), sums of r^2 (s1) and e (s2),
//              forward transform of r into w;
//   kXForward  forward transform of r into w;
//   kXInverse  inverse transform of w (z = M^-1 r) and the sum r.z (s1).
// Buffers: B0 r (or w), B1 q (then the transform's output) or r, B2 e, B3 p.
template <typename T, int K>
__device__ void x_pass_rows(const SArgs<T> &a, const Smem<T> &sm, int kind, T al, bool upd, bool he, CgAcc<T> &s1,
                            CgAcc<T> &s2) {
  constexpr int P = Pack<T>::n;
  const Grid3 g = a.g;
  const int W = a.ax[0].W, lgW = a.ax[0].lgW, N = g.nx;
  const unsigned nlines = unsigned(g.ny) * unsigned(g.nz);
  const int nt = int((nlines + unsigned(W) - 1u) >> lgW);
  const int tile = W * N, B = blockDim.x;
  T *B0 = reinterpret_cast<T *>(sm.bA), *B1 = B0 + tile, *B2 = B1 + tile, *B3 = B2 + tile;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
  const C2<T> *lt = sm.lanetw + lane * kLaneTw;
  for (int t = blockIdx.x; t < nt; t += gridDim.x) {
    const unsigned row0 = unsigned(t) << lgW;
    const int rows = min(W, int(nlines - row0));
    const int nwd = rows * N;  // words of the tile's rows
    const size_t off = size_t(row0) * size_t(N);
    const bool lq = kind == kXUpdate && upd;
    cp_rows(B0, (kind == kXInverse ? a.w : a.r) + off, nwd);
    if (kind == kXInverse) cp_rows(B1, a.r + off, nwd);
    if (lq) {
      cp_rows(B1, a.q + off, nwd);
      cp_rows(B3, a.p + off, nwd);
      if (he) cp_rows(B2, a.e + off, nwd);
    }
    for (int e = nwd + threadIdx.x; e < tile; e += B) B0[e] = T(0);  // line b past the last row
    cp_wait_all();
    __syncthreads();
    if (kind == kXUpdate) {
      for (int i = threadIdx.x; i < nwd / P; i += B) {
        Pack<T> rv = reinterpret_cast<const Pack<T> *>(B0)[i];
        if (upd) {
          const Pack<T> qv = reinterpret_cast<const Pack<T> *>(B1)[i];
          const Pack<T> pv = reinterpret_cast<const Pack<T> *>(B3)[i];
          Pack<T> ev{};
          if (he) ev = reinterpret_cast<const Pack<T> *>(B2)[i];
#pragma unroll
          for (int j = 0; j < P; ++j) {
            rv.v[j] -= al * qv.v[j];
            ev.v[j] += al * pv.v[j];
            s2.add(ev.v[j]);
          }
          reinterpret_cast<Pack<T> *>(B0)[i] = rv;
          reinterpret_cast<Pack<T> *>(a.r + off)[i] = rv;
          reinterpret_cast<Pack<T> *>(a.e + off)[i] = ev;
        }
#pragma unroll
        for (int j = 0; j < P; ++j) s1.add(rv.v[j] * rv.v[j]);
      }
      __syncthreads();
    }
    // the line pairs (rows 2m, 2m + 1) in registers, one warp per pair
    T *dst = kind == kXInverse ? B0 : B1;
    for (int m = warp; m < (W >> 1); m += nw) {
      const T *ra = B0 + 2 * m * N, *rb = ra + N;
      C2<T> v[K];
      T ha[K], hb[K];
#pragma unroll
      for (int k = 0; k < K; ++k) v[k] = C2<T>{ra[lane + 32 * k], rb[lane + 32 * k]};
      if (kind == kXInverse) {
        dit_regs<T, K>(v, lt, lane);
        split_nat<T, K>(v, lane, ha, hb);
      } else {
        dif_regs<T, K>(v, lt, lane);
        split_perm<T, K>(v, lane, ha, hb);
      }
      T *da = dst + 2 * m * N, *db = da + N;
#pragma unroll
      for (int k = 0; k < K; ++k) {
        da[lane + 32 * k] = ha[k];
        db[lane + 32 * k] = hb[k];
      }
    }
    __syncthreads();
    for (int i = threadIdx.x; i < nwd / P; i += B) {
      const Pack<T> zv = reinterpret_cast<const Pack<T> *>(dst)[i];
      reinterpret_cast<Pack<T> *>(a.w + off)[i] = zv;
      if (kind == kXInverse) {
        const Pack<T> rv = reinterpret_cast<const Pack<T> *>(B1)[i];
#pragma unroll
        for (int j = 0; j < P; ++j) s1.add(rv.v[j] * zv.v[j]);
      }
    }
    __syncthreads();
  }
}
template <typename T>
__device__ void x_pass_rows_k(const SArgs<T> &a, const Smem<T> &sm, int kind, T al, bool upd, bool he, CgAcc<T> &s1,
                              CgAcc<T> &s2) {
  switch (reg_fft_k(a.g.nx)) {
    case 1: x_pass_rows<T, 1>(a, sm, kind, al, upd, he, s1, s2); break;
    case 2: x_pass_rows<T, 2>(a, sm, kind, al, upd, he, s1, s2); break;
    case 4: x_pass_rows<T, 4>(a, sm, kind, al, upd, he, s1, s2); break;
    default: x_pass_rows<T, 8>(a, sm, kind, al, upd, he, s1, s2); break;
  }
}

// q = A z + beta q, p = z + beta p over the team's cells; the thread's shares
// of p.q and, for the prediction of the next residual, r.q and q.q
template <typename T, bool DFM>
__device__ void matvec_update(const SArgs<T> &a, const T *z, T beta, bool first, double *sh, double &pq, double &rq,
                              double &qq) {
  const Level<T> L0 = a.L0;
  const Dims d = L0.dims();
  const long long G = (long long)gridDim.x * blockDim.x;
  constexpr int U = 4;  // cells per thread with their loads in flight together
  CgAcc<T> apq, arq, aqq;
  Walk wk(blockIdx.x * (long long)blockDim.x + threadIdx.x, G, d.nx, d.ny);
  while (wk.z < d.nz) {
    Nbr c[U];
    bool v[U];
#pragma unroll
    for (int u = 0; u < U; ++u) {
      v[u] = wk.z < d.nz;
      c[u] = nbr(d, v[u] ? wk.u : 0, v[u] ? wk.y : 0, v[u] ? wk.z : 0);
      if (v[u]) wk.next();
    }
    T zc[U], zn[U][6], ec[U], en[U][6], pv[U], qv[U], rv[U];
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const unsigned nb6[6] = {c[u].xp, c[u].xm, c[u].yp, c[u].ym, c[u].zp, c[u].zm};
      zc[u] = z[c[u].i];
      ec[u] = L0.eps[c[u].i];
#pragma unroll
      for (int k = 0; k < 6; ++k) {
        zn[u][k] = z[nb6[k]];
        en[u][k] = L0.eps[nb6[k]];
      }
      pv[u] = first ? T(0) : a.p[c[u].i];
      qv[u] = first ? T(0) : a.q[c[u].i];
      rv[u] = a.r[c[u].i];
    }
#pragma unroll
    for (int u = 0; u < U; ++u) {
      if (!v[u]) continue;
      T Az = T(0);
#pragma unroll
      for (int k = 0; k < 6; ++k) Az += T(0.5) * (ec[u] + en[u][k]) * (zn[u][k] - zc[u]);
      const T pn = zc[u] + beta * pv[u];
      const T qn = Az + beta * qv[u];
      a.p[c[u].i] = pn;
      a.q[c[u].i] = qn;
      apq.add(pn * qn);
      arq.add(rv[u] * qn);
      aqq.add(qn * qn);
    }
  }
  pq = apq.get();
  rq = arq.get();
  qq = aqq.get();
}

// r -= alpha q, e += alpha p over the team's cells with the sums of r^2 and e
// (the update of an iteration predicted to be the last: no x pass follows)
template <typename T>
__device__ void update_cells(const SArgs<T> &a, T al, bool he, CgAcc<T> &sr, CgAcc<T> &se) {
  const long long N = a.L0.N;
  const long long G = (long long)gridDim.x * blockDim.x;
  constexpr int U = kU / 2;
  for (long long i0 = blockIdx.x * (long long)blockDim.x + threadIdx.x; i0 < N; i0 += U * G) {
    T rv[U], qv[U], ev[U], pv[U];
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const long long i = i0 + u * G;
      const bool in = i < N;
      rv[u] = in ? a.r[i] : T(0);
      qv[u] = in ? a.q[i] : T(0);
      ev[u] = in && he ? a.e[i] : T(0);
      pv[u] = in ? a.p[i] : T(0);
    }
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const long long i = i0 + u * G;
      if (i >= N) continue;
      const T r = rv[u] - al * qv[u];
      const T e = ev[u] + al * pv[u];
      a.r[i] = r;
      a.e[i] = e;
      sr.add(r * r);
      se.add(e);
    }
  }
}

// Exact residual r = b - A phi with b = -(q - qbar) + sum_d k (E_ext . c_d)
// (FP64, or double-float words in the FP32 modes: the arithmetic of
// residual_site in poisson_dev.cuh), two cells per thread with all their
// loads in flight together; the thread's shares of |r|^2, |b|^2 and sum phi.
template <typename T, bool DFM>
__device__ void residual_cells(const SArgs<T> &a, double qbar, DF qbar_df, double *sh, double &ar, double &ab,
                               double &ap) {
  const PArgs<T> &pa = a.pa;
  const Level<T> &L0 = a.L0;
  const Dims d = L0.dims();
  const long long G = (long long)gridDim.x * blockDim.x;
  constexpr int U = 2;
  // per-thread sums of a few dozen cells: FP32 in the FP32 modes (relative
  // error ~1e-6 of |r|^2 and |b|^2, far inside the margins of the tests they
  // steer; the sum of phi only sets the mean shift, ~1e-10 of phi per site),
  // FP64 in the FP64 mode
  using Acc = typename std::conditional<DFM, CgAcc<float>, SumAcc<false>>::type;
  Acc sr, sb, sp;
  Walk wk(blockIdx.x * (long long)blockDim.x + threadIdx.x, G, d.nx, d.ny);
  while (wk.z < d.nz) {
    Nbr c[U];
    bool v[U];
#pragma unroll
    for (int u = 0; u < U; ++u) {
      v[u] = wk.z < d.nz;
      c[u] = nbr(d, v[u] ? wk.u : 0, v[u] ? wk.y : 0, v[u] ? wk.z : 0);
      if (v[u]) wk.next();
    }
    using P = typename std::conditional<DFM, float, double>::type;
    P ph[U][7], pl[U][7];
    T ev[U][7], qv[U];
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const unsigned idx[7] = {c[u].i, c[u].xp, c[u].xm, c[u].yp, c[u].ym, c[u].zp, c[u].zm};
#pragma unroll
      for (int k = 0; k < 7; ++k) {
        if constexpr (DFM) {
          ph[u][k] = pa.phi_hi[idx[k]];
          pl[u][k] = pa.phi_lo[idx[k]];
        } else {
          ph[u][k] = pa.phi[idx[k]];
          pl[u][k] = 0.0;
        }
        ev[u][k] = L0.eps[idx[k]];
      }
      qv[u] = pa.q[c[u].i];
    }
#pragma unroll
    for (int u = 0; u < U; ++u) {
      if (!v[u]) continue;
      T kf[6];
#pragma unroll
      for (int k = 0; k < 6; ++k) kf[k] = T(0.5) * (ev[u][0] + ev[u][k + 1]);
      if constexpr (DFM) {
        // sum_k kf_k (phi_k - phi_0): each difference is the exact difference
        // of the high words (two_sum) plus the difference of the low words;
        // the high part of kf_k d_k is exact with its FMA error term, the high
        // parts are summed with compensation and the low parts in FP32
        // (error about 2^-46 of the largest flux term, as in double-float
        // arithmetic)
        float ahi = 0.f, alo = 0.f;
#pragma unroll
        for (int k = 0; k < 6; ++k) {
          const DF d = two_sum(ph[u][k + 1], -ph[u][0]);
          const float dlo = __fadd_rn(d.lo, __fsub_rn(pl[u][k + 1], pl[u][0]));
          const float prod = __fmul_rn(d.hi, kf[k]);
          const float plo = __fmaf_rn(dlo, kf[k], __fmaf_rn(d.hi, kf[k], -prod));
          const DF t = two_sum(ahi, prod);
          ahi = t.hi;
          alo = __fadd_rn(alo, __fadd_rn(t.lo, plo));
        }
        DF b = two_sum(qbar_df.hi, -float(qv[u]));
        b.lo = __fadd_rn(b.lo, qbar_df.lo);
        if (pa.edf[0].hi != 0.f) b = df_add(b, df_mul(pa.edf[0], two_sum(kf[0], -kf[1])));
        if (pa.edf[1].hi != 0.f) b = df_add(b, df_mul(pa.edf[1], two_sum(kf[2], -kf[3])));
        if (pa.edf[2].hi != 0.f) b = df_add(b, df_mul(pa.edf[2], two_sum(kf[4], -kf[5])));
        const DF r = two_sum(b.hi, -ahi);
        const float rf = __fadd_rn(r.hi, __fadd_rn(r.lo, __fsub_rn(b.lo, alo)));
        L0.b[c[u].i] = T(rf);
        sr.add(rf * rf);
        sb.add(b.hi * b.hi);
        sp.add(ph[u][0]);
      } else {
        const double p = ph[u][0];
        double b = -(double(qv[u]) - qbar);
        if (pa.ex != 0.0) b += pa.ex * (double(kf[0]) - double(kf[1]));
        if (pa.ey != 0.0) b += pa.ey * (double(kf[2]) - double(kf[3]));
        if (pa.ez != 0.0) b += pa.ez * (double(kf[4]) - double(kf[5]));
        const double Ap = double(kf[0]) * (ph[u][1] - p) - double(kf[1]) * (p - ph[u][2]) +
                          double(kf[2]) * (ph[u][3] - p) - double(kf[3]) * (p - ph[u][4]) +
                          double(kf[4]) * (ph[u][5] - p) - double(kf[5]) * (p - ph[u][6]);
        const double r = b - Ap;
        L0.b[c[u].i] = T(r);
        sr.add(r * r);
        sb.add(b * b);
        sp.add(p);
      }
    }
  }
  ar = sr.get();
  ab = sb.get();
  ap = sp.get();
}

// Scalar arithmetic of the iteration (divisions, square roots in FP64) by
// thread 0 alone, broadcast through shared memory: the FP64 rate of the
// target is a small fraction of its FP32 rate, and 256 threads repeating a
// division or a square root cost about a microsecond per phase.  Each call
// site has its own cell, so a cell is rewritten only after the barriers of
// the passes in between.
__device__ __forceinline__ double bcast0(double v, double *cell) {
  if (threadIdx.x == 0) *cell = v;
  __syncthreads();
  return *cell;
}

template <typename T, bool DFM>
__global__ void __launch_bounds__(kSB, 2) k_spectral(SArgs<T> a) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ double sh[3 * kSB];  // block sums of up to three values
  __shared__ double bc[8];  // broadcast cells of the scalar arithmetic
  const bool t0 = threadIdx.x == 0;
  const Smem<T> sm = smem_layout<T>(smem_raw, a);
  load_tables(a, sm);
  const PArgs<T> &pa = a.pa;
  const GridTeam tm{pa.bar, pa.status, pa.spin_limit};
  const Level<T> L0 = a.L0;
  const Dims d = L0.dims();
  const long long N = d.N;
  const long long G = tm.size(), gt = tm.rank();
  const int nb = tm.nblocks();
  PDev *st = pa.st;
  const int have_prev = st->have_prev;

  // initial guess 2 phi(t-1) - phi(t-2), sum of q (kU cells per thread in flight)
  SumAcc<DFM> sq;
  for (long long i0 = gt; i0 < N; i0 += kU * G) {
    if constexpr (DFM) {
      float h[kU], l[kU], ph[kU], pl[kU], qq[kU];
#pragma unroll
      for (int u = 0; u < kU; ++u) {
        const long long i = i0 + u * G;
        const bool in = i < N;
        h[u] = in ? pa.phi_hi[i] : 0.f;
        l[u] = in ? pa.phi_lo[i] : 0.f;
        ph[u] = in && have_prev ? pa.prev_hi[i] : 0.f;
        pl[u] = in && have_prev ? pa.prev_lo[i] : 0.f;
        qq[u] = in ? float(pa.q[i]) : 0.f;
      }
#pragma unroll
      for (int u = 0; u < kU; ++u) {
        const long long i = i0 + u * G;
        if (i >= N) continue;
        if (have_prev) {
          const DF gv = df_sub(DF{2.f * h[u], 2.f * l[u]}, DF{ph[u], pl[u]});
          pa.phi_hi[i] = gv.hi;
          pa.phi_lo[i] = gv.lo;
        }
        pa.prev_hi[i] = h[u];
        pa.prev_lo[i] = l[u];
        sq.add(qq[u]);
      }
    } else {
      double pv[kU], pr[kU], qq[kU];
#pragma unroll
      for (int u = 0; u < kU; ++u) {
        const long long i = i0 + u * G;
        const bool in = i < N;
        pv[u] = in ? pa.phi[i] : 0.0;
        pr[u] = in && have_prev ? pa.prev[i] : 0.0;
        qq[u] = in ? double(pa.q[i]) : 0.0;
      }
#pragma unroll
      for (int u = 0; u < kU; ++u) {
        const long long i = i0 + u * G;
        if (i >= N) continue;
        if (have_prev) pa.phi[i] = 2.0 * pv[u] - pr[u];
        pa.prev[i] = pv[u];
        sq.add(qq[u]);
      }
    }
  }
  {
    double v[1] = {sq.get()};
    put_block_sums<1>(v, pa.part, nb, sh);
  }
  double qs[1];
  if (!sync_sums<1>(tm, pa.part, nb, qs, sh)) return;
  const double qbar = bcast0(t0 ? qs[0] / double(N) : 0.0, &bc[0]);
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
    {
      double v[3];
      residual_cells<T, DFM>(a, qbar, qbar_df, sh, v[0], v[1], v[2]);
      put_block_sums<3>(v, pa.part, nb, sh);
      if (!sync_sums<3>(tm, pa.part, nb, v, sh)) return;
      r2 = v[0];
      b2 = v[1];
      ps = v[2];
    }
    if (outer == 0) bn = b2;
    rr = bcast0(t0 ? rel_res(r2, bn) : 0.0, &bc[1]);
    exact = true;
    shift = bcast0(t0 ? ps / double(N) : 0.0, &bc[2]);
    have_e = false;
    if (rr < tol || it >= max_iter || !isfinite(rr)) break;
    const double rr_start = rr;
    // the compute-type recursion tracks the residual to a fraction of its
    // start; below that the exact residual restarts the iteration
    const double target = fmax(tol, rr_start * kInnerReduction<T>);
    // conjugate gradients on A e = r
    double rho_old = 1.0, alpha = 0.0, sum_e = 0.0;
    bool first = true;
    bool last = false;  // the coming update is predicted to end the iteration
    for (;;) {
      // U: update r and e, Hartley pass along x of r into w.  Its sums of
      // |r|^2 and e join the reduction of r.z one phase later; only the
      // update predicted to be the last runs alone with its own reduction.
      CgAcc<T> sr, se;
      const T al = T(alpha);
      const bool upd = !first, he = have_e;
      if (last) {
        update_cells<T>(a, al, he, sr, se);
        have_e = true;
        double v[2] = {sr.get(), se.get()};
        put_block_sums<2>(v, pa.part, nb, sh);
        if (!sync_sums<2>(tm, pa.part, nb, v, sh)) return;
        r2 = v[0];
        sum_e = v[1];
        ++it;
        rr = bcast0(t0 ? rel_res(r2, bn) : 0.0, &bc[3]);
        exact = false;
        if (rr < target || it >= max_iter || !isfinite(rr)) break;
        // mispredicted: the x pass of the updated r
        if (a.xrows) {
          CgAcc<T> d0, d1;
          x_pass_rows_k<T>(a, sm, kXForward, T(0), false, false, d0, d1);
        } else {
          tile_pass<T>(a, sm, 0, kFwd, LoadW<T>{a.r}, StoreW<T>{a.w});
        }
      } else {
        if (a.xrows) {
          x_pass_rows_k<T>(a, sm, kXUpdate, al, upd, he, sr, se);
        } else {
          LoadU<T> lu{a.r, a.e, a.q, a.p, al, upd, he, &sr, &se};
          tile_pass<T>(a, sm, 0, kFwd, lu, StoreW<T>{a.w});
        }
        if (upd) {
          have_e = true;
          ++it;
        }
      }
      if (!tm.sync()) return;
      // preconditioner: Y, Z (scale), Y, X passes on w
      const LoadW<T> lw{a.w};
      tile_pass<T>(a, sm, 1, kFwd, lw, StoreW<T>{a.w});
      if (!tm.sync()) return;
      tile_pass<T>(a, sm, 2, kFused, lw, StoreW<T>{a.w});
      if (!tm.sync()) return;
      tile_pass<T>(a, sm, 1, kInv, lw, StoreW<T>{a.w});
      if (!tm.sync()) return;
      CgAcc<T> srz;
      if (a.xrows) {
        CgAcc<T> d1;
        x_pass_rows_k<T>(a, sm, kXInverse, T(0), false, false, srz, d1);
      } else {
        tile_pass<T>(a, sm, 0, kInv, LoadWR<T>{a.w, a.r}, StoreRZ<T>{a.w, a.r, &srz});
      }
      double rz[3] = {srz.get(), sr.get(), se.get()};
      put_block_sums<3>(rz, pa.part, nb, sh);
      if (!sync_sums<3>(tm, pa.part, nb, rz, sh)) return;
      const double rho = rz[0];
      if (upd) {
        // the residual and the correction after this iteration's update: a
        // convergence the prediction missed ends the iteration here
        r2 = rz[1];
        sum_e = rz[2];
        rr = bcast0(t0 ? rel_res(r2, bn) : 0.0, &bc[3]);
        exact = false;
        if (rr < target || it >= max_iter || !isfinite(rr)) break;
      }
      const double beta = bcast0(t0 && !first ? rho / rho_old : 0.0, &bc[4]);
      // F: search direction and its image
      {
        double v[3];
        matvec_update<T, DFM>(a, a.w, T(beta), first, sh, v[0], v[1], v[2]);
        put_block_sums<3>(v, pa.part, nb, sh);
      }
      double fs[3];
      if (!sync_sums<3>(tm, pa.part, nb, fs, sh)) return;
      const double pq = fs[0], rq = fs[1], qq = fs[2];
      alpha = bcast0(t0 && pq != 0.0 ? rho / pq : 0.0, &bc[5]);
      rho_old = rho;
      first = false;
      // |r - alpha q|^2 from the sums (the same in every block)
      last = it + 1 >= max_iter ||
             bcast0(t0 ? rel_res(fmax(r2 - 2.0 * alpha * rq + alpha * alpha * qq, 0.0), bn) : 0.0, &bc[6]) < target;
    }
    shift += bcast0(t0 ? sum_e / double(N) : 0.0, &bc[7]);
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
  // FP32 modes, N a multiple of 4: four cells per 16-byte access (the
  // arrays start 256-byte aligned), two groups in flight per thread
  const long long N4 = DFM && (N & 3) == 0 ? N / 4 : 0;
  if constexpr (DFM) {
    for (long long j0 = gt; j0 < N4; j0 += 2 * G) {
      float4 h[2], l[2], ev[2];
#pragma unroll
      for (int u = 0; u < 2; ++u) {
        const long long j = j0 + u * G;
        const bool in = j < N4 && !zero;
        const float4 z4 = make_float4(0.f, 0.f, 0.f, 0.f);
        h[u] = in ? reinterpret_cast<const float4 *>(pa.phi_hi)[j] : z4;
        l[u] = in ? reinterpret_cast<const float4 *>(pa.phi_lo)[j] : z4;
        ev[u] = in && have_e ? reinterpret_cast<const float4 *>(a.e)[j] : z4;
      }
#pragma unroll
      for (int u = 0; u < 2; ++u) {
        const long long j = j0 + u * G;
        if (j >= N4) continue;
        const float hh[4] = {h[u].x, h[u].y, h[u].z, h[u].w}, ll[4] = {l[u].x, l[u].y, l[u].z, l[u].w};
        const float ee[4] = {ev[u].x, ev[u].y, ev[u].z, ev[u].w};
        float oh[4], ol[4];
#pragma unroll
        for (int c = 0; c < 4; ++c) {
          DF v{0.f, 0.f};
          if (!zero) v = df_sub(df_add(DF{hh[c], ll[c]}, DF{ee[c], 0.f}), shift_df);
          oh[c] = v.hi;
          ol[c] = v.lo;
        }
        reinterpret_cast<float4 *>(pa.phi_hi)[j] = make_float4(oh[0], oh[1], oh[2], oh[3]);
        reinterpret_cast<float4 *>(pa.phi_lo)[j] = make_float4(ol[0], ol[1], ol[2], ol[3]);
      }
    }
  }
  for (long long i0 = gt + 4 * N4; i0 < N; i0 += kU * G) {
    if constexpr (DFM) {
      float h[kU], l[kU], ev[kU];
#pragma unroll
      for (int u = 0; u < kU; ++u) {
        const long long i = i0 + u * G;
        const bool in = i < N && !zero;
        h[u] = in ? pa.phi_hi[i] : 0.f;
        l[u] = in ? pa.phi_lo[i] : 0.f;
        ev[u] = in && have_e ? float(a.e[i]) : 0.f;
      }
#pragma unroll
      for (int u = 0; u < kU; ++u) {
        const long long i = i0 + u * G;
        if (i >= N) continue;
        DF v{0.f, 0.f};
        if (!zero) v = df_sub(df_add(DF{h[u], l[u]}, DF{ev[u], 0.f}), shift_df);
        pa.phi_hi[i] = v.hi;
        pa.phi_lo[i] = v.lo;
      }
    } else {
      double pv[kU], ev[kU];
#pragma unroll
      for (int u = 0; u < kU; ++u) {
        const long long i = i0 + u * G;
        const bool in = i < N && !zero;
        pv[u] = in ? pa.phi[i] : 0.0;
        ev[u] = in && have_e ? double(a.e[i]) : 0.0;
      }
#pragma unroll
      for (int u = 0; u < kU; ++u) {
        const long long i = i0 + u * G;
        if (i < N) pa.phi[i] = zero ? 0.0 : pv[u] + ev[u] - shift;
      }
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

}  // namespace

struct Spectral {
  int fp64 = 0;
  int grid = 0;
  size_t smem = 0;
  std::vector<void *> allocs;
  void *r = nullptr, *p = nullptr, *q = nullptr, *e = nullptr, *w = nullptr;
  void *code[3] = {nullptr, nullptr, nullptr}, *tw[3] = {nullptr, nullptr, nullptr};
  void *sym[3] = {nullptr, nullptr, nullptr};
  LinePlan plan[3];
  int W[3] = {0, 0, 0}, lgW[3] = {0, 0, 0};
  int code_at[3] = {0, 0, 0}, tw_at[3] = {0, 0, 0}, s_at[3] = {0, 0, 0};
  int ncode = 0, ntw = 0, ns = 0;
  double eps_ref = 1.0;
};

bool spectral_supported(const Dims &d, int fp64) {
  int rad[kMaxStages];
  const int lim = fp64 ? 256 : kMaxN;
  for (int n : {d.nx, d.ny, d.nz})
    if (n < 2 || n > lim || !plan_radices(n, rad)) return false;
  return true;
}

template <typename T> static bool spectral_setup(Spectral *s, const Dims &d) {
  auto dal = [&](size_t bytes) -> void * {
    void *ptr = nullptr;
    if (cudaMalloc(&ptr, bytes) != cudaSuccess) return nullptr;
    s->allocs.push_back(ptr);
    return ptr;
  };
  // the five work arrays in one allocation, each start skewed by an odd
  // number of 256-byte lines from the power-of-two strides of the lattice, so
  // that the same site of the five arrays (read and written together by the
  // passes) does not fall into the same L2 sets
  const size_t nb = sizeof(T) * (size_t)d.N;
  const size_t stride = ((nb + 255) & ~size_t(255)) + 97 * 256;
  unsigned char *base = (unsigned char *)dal(5 * stride);
  if (!base) return false;
  s->r = base;
  s->p = base + stride;
  s->q = base + 2 * stride;
  s->e = base + 3 * stride;
  s->w = base + 4 * stride;
  const int ns[3] = {d.nx, d.ny, d.nz};
  size_t tiles = 0;
  for (int A = 0; A < 3; ++A) {
    const int n = ns[A];
    std::vector<unsigned> code;
    std::vector<C2<double>> twd;
    if (!build_plan(n, s->plan[A], code, twd)) return false;
    std::vector<C2<T>> tw(twd.size());
    for (size_t k = 0; k < twd.size(); ++k) tw[k] = C2<T>{T(twd[k].x), T(twd[k].y)};
    s->code_at[A] = s->ncode;
    s->tw_at[A] = s->ntw;
    s->s_at[A] = s->ns;
    s->ncode += (int)code.size();
    s->ntw += (int)tw.size();
    s->ns += n;
    int W = 32, lg = 5;  // lines per tile: the largest of 32, 16, 8 whose tile fits 40 KB
    while (W > 8 && 2 * (W / 2) * (n + 1) * sizeof(C2<T>) > 40 * 1024) {
      W /= 2;
      --lg;
    }
    s->W[A] = W;
    s->lgW[A] = lg;
    tiles = std::max(tiles, 4 * (size_t)(W / 2) * (n + 1) * sizeof(C2<T>));
    // symbols 2 (1 - cos(2 pi k / n)) in the axis's storage order: slot
    // l + 32 kappa of a register-transformed axis holds frequency
    // kappa + K bitrev5(l)
    std::vector<T> sy(n);
    const int K = reg_fft_k(n);
    for (int j = 0; j < n; ++j) {
      int k = j;
      if (K) {
        int br = 0;
        for (int b = 0; b < 5; ++b) br |= ((j & 31) >> b & 1) << (4 - b);
        k = (j >> 5) + K * br;
      }
      sy[j] = T(2.0 * (1.0 - std::cos(2.0 * M_PI * double(k) / double(n))));
    }
    if (!(s->code[A] = dal(4 * code.size())) || !(s->tw[A] = dal(sizeof(C2<T>) * tw.size())) ||
        !(s->sym[A] = dal(sizeof(T) * n)))
      return false;
    if (cudaMemcpy(s->code[A], code.data(), 4 * code.size(), cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemcpy(s->tw[A], tw.data(), sizeof(C2<T>) * tw.size(), cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemcpy(s->sym[A], sy.data(), sizeof(T) * n, cudaMemcpyHostToDevice) != cudaSuccess)
      return false;
  }
  // layout of smem_layout(): plans, codes, twiddles, symbols, tile buffers (16-byte aligned parts)
  auto al = [](size_t b) { return (b + 15) & ~size_t(15); };
  const size_t smem = al(3 * sizeof(LinePlan)) + al((size_t)s->ncode * 4) + al((size_t)s->ntw * sizeof(C2<T>)) +
                      al((size_t)s->ns * sizeof(T)) + (size_t)3 * 32 * kLaneTw * sizeof(C2<T>) + tiles;
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
    AxisDev<T> &X = a.ax[A];
    X.P = s->plan[A];
    X.W = s->W[A];
    X.lgW = s->lgW[A];
    X.ld = s->plan[A].n + 1;
    X.code = (const unsigned *)s->code[A];
    X.tw = (const C2<T> *)s->tw[A];
    X.s = (const T *)s->sym[A];
    X.code_at = s->code_at[A];
    X.tw_at = s->tw_at[A];
    X.s_at = s->s_at[A];
  }
  a.ncode = s->ncode;
  a.ntw = s->ntw;
  a.ns = s->ns;
  a.g = Grid3{c.d.nx, c.d.ny, c.d.nz};
  a.r = (T *)s->r;
  a.p = (T *)s->p;
  a.q = (T *)s->q;
  a.e = (T *)s->e;
  a.w = (T *)s->w;
  a.inv_eref_n = T(1.0 / (s->eps_ref * double(c.d.N)));
  // rows of nx words start on 16-byte boundaries (arrays 256-byte aligned)
  a.xrows = reg_fft_k(c.d.nx) != 0 && (c.d.nx * sizeof(T)) % 16 == 0;
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
