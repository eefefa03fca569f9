// Projection of spherical colloids onto the lattice (Sec. II.E).
//
// A node is solid when its centre is strictly inside a sphere (minimum-image
// squared distance < r^2).  The solid fraction psi_s = nu/(h+1)^3 counts the
// sub-cube centres (h+1 per axis) strictly inside.  Surface nodes are solid
// nodes with a fluid D3Q19 neighbour; the colloid's charge Q is split equally
// over them.  Distances are evaluated with explicitly rounded FP64 operations
// (no fused multiply-add) in a fixed order, so the masks are bit-identical to
// any IEEE FP64 evaluation of ((dx*dx + dy*dy) + dz*dz) < r*r.
#include "internal.h"

namespace lbeh {

__device__ __forceinline__ double min_image(double dd, int n) {
  const double half = 0.5 * double(n);
  if (dd > half) return __dsub_rn(dd, double(n));
  if (dd < -half) return __dadd_rn(dd, double(n));
  return dd;
}

__device__ __forceinline__ double dist2(double px, double py, double pz, const double *X, const Dims &d) {
  const double dx = min_image(__dsub_rn(px, X[0]), d.nx);
  const double dy = min_image(__dsub_rn(py, X[1]), d.ny);
  const double dz = min_image(__dsub_rn(pz, X[2]), d.nz);
  return __dadd_rn(__dadd_rn(__dmul_rn(dx, dx), __dmul_rn(dy, dy)), __dmul_rn(dz, dz));
}

struct Box {
  int lo[3], cnt[3];
};

__device__ __forceinline__ Box bbox(const Dims &d, const double *X, double r, double margin) {
  Box b;
  const int dims[3] = {d.nx, d.ny, d.nz};
  for (int a = 0; a < 3; ++a) {
    b.lo[a] = int(ceil(X[a] - r - margin));
    const int hi = int(floor(X[a] + r + margin));
    b.cnt[a] = min(dims[a], hi - b.lo[a] + 1);
  }
  return b;
}

__device__ __forceinline__ void box_site(const Dims &d, const Box &b, long long t, int &x, int &y, int &z) {
  x = ((b.lo[0] + int(t % b.cnt[0])) % d.nx + d.nx) % d.nx;
  y = ((b.lo[1] + int((t / b.cnt[0]) % b.cnt[1])) % d.ny + d.ny) % d.ny;
  z = ((b.lo[2] + int(t / ((long long)b.cnt[0] * b.cnt[1]))) % d.nz + d.nz) % d.nz;
}

// Position of a node or sample relative to the sphere centre, split into
// the integer part of the centre (exact) and a fractional remainder: in FP32
// the offset d = (x - floor(X)) + o - frac(X) is then within 1e-6 of the exact
// value times 2^-23 |d|, so |d^2 - r^2| > 1e-3 + 1e-5 r^2 decides "inside"
// exactly as the rounded FP64 test does; closer cases use the FP64 test itself.
constexpr float kCertain = 1e-3f;

__device__ __forceinline__ int wrap_rel(int dx, int n) {
  // minimum-image integer offset in (-n/2, n/2]
  if (dx > n / 2) dx -= n;
  if (dx <= -((n + 1) / 2)) dx += n;
  return dx;
}

template <typename T>
__global__ void k_project(Dims d, int h, const double *__restrict__ cx, const double *__restrict__ cr,
                          uint8_t *__restrict__ solid, int *__restrict__ owner, T *__restrict__ psi_s, int slabs) {
  const int j = blockIdx.x / slabs, sl = blockIdx.x - j * slabs;
  const double X[3] = {cx[3 * j], cx[3 * j + 1], cx[3 * j + 2]};
  const double r = cr[j];
  const double r2 = __dmul_rn(r, r);
  const float r2f = float(r2);
  const float certain = kCertain + 1e-5f * r2f;
  const Box b = bbox(d, X, r, 1.0);
  const long long tot = (long long)b.cnt[0] * b.cnt[1] * b.cnt[2];
  const int hp = h + 1;
  const double inv = double(hp) * hp * hp;
  const int dims[3] = {d.nx, d.ny, d.nz};
  int Xi[3];
  float Xf[3];
  for (int a = 0; a < 3; ++a) {
    const double fl = floor(X[a]);
    Xi[a] = int(fl);
    Xf[a] = float(X[a] - fl);  // exact difference, rounded once to FP32
  }
  // sub-cube centre offsets (k + 1/2)/(h+1) - 1/2, once per block
  __shared__ double off[16];
  __shared__ float offf[16];
  if (threadIdx.x < hp) {
    off[threadIdx.x] = __dsub_rn(__ddiv_rn(threadIdx.x + 0.5, double(hp)), 0.5);
    offf[threadIdx.x] = float(off[threadIdx.x]);  // dyadic: exact in FP32
  }
  __syncthreads();
  // Every sub-cube centre lies within sqrt(3) (1/2 - 1/(2(h+1))) of its node;
  // a node farther than that (plus 1e-3) from the sphere surface has all its
  // samples on one side.  Used only where every sample and the node share one
  // periodic image.
  const double reach = 1.7320508075688772 * (0.5 - 0.5 / double(hp)) + 1e-3;
  const double r_in = r - reach, r_out = r + reach;
  const bool shortcut = 2.0 * (r_out + 1.0) < double(min(d.nx, min(d.ny, d.nz)));
  for (long long t = (long long)sl * blockDim.x + threadIdx.x; t < tot; t += (long long)slabs * blockDim.x) {
    int x, y, z;
    box_site(d, b, t, x, y, z);
    const long long i = site(d, x, y, z);
    const int p[3] = {x, y, z};
    float rel[3];
    for (int a = 0; a < 3; ++a) rel[a] = float(wrap_rel(p[a] - Xi[a], dims[a])) - Xf[a];
    const float d2f = rel[0] * rel[0] + rel[1] * rel[1] + rel[2] * rel[2];
    // (the FP32 offsets pick the nearest periodic image; the FP64 test may pick
    // the other one only for samples about half a box away, which are outside
    // whenever the shortcut condition holds, so the fast path is used only then)
    bool in_node;
    if (shortcut && fabsf(d2f - r2f) > certain) in_node = d2f < r2f;
    else in_node = dist2(double(x), double(y), double(z), X, d) < r2;
    if (in_node) {
      solid[i] = 1;
      atomicMax(owner + i, j);
    }
    int nu = 0;
    const float rinf = float(r_in), routf = float(r_out);
    if (shortcut && r_in > 0.0 && d2f < rinf * rinf - certain) {
      nu = hp * hp * hp;
    } else if (shortcut && d2f > routf * routf + certain) {
      nu = 0;
    } else {
      for (int kz = 0; kz < hp; ++kz) {
        const float qz = rel[2] + offf[kz];
        for (int ky = 0; ky < hp; ++ky) {
          const float qy = rel[1] + offf[ky];
          const float s2 = qy * qy + qz * qz;
          for (int kx = 0; kx < hp; ++kx) {
            const float qx = rel[0] + offf[kx];
            const float e2 = qx * qx + s2;
            bool in;
            if (shortcut && fabsf(e2 - r2f) > certain)
              in = e2 < r2f;
            else
              in = dist2(__dadd_rn(double(x), off[kx]), __dadd_rn(double(y), off[ky]), __dadd_rn(double(z), off[kz]),
                         X, d) < r2;
            nu += in ? 1 : 0;
          }
        }
      }
    }
    if (nu) atomicAdd(psi_s + i, T(double(nu) / inv));  // dyadic values: exact in any order
  }
}

template <typename T>
__global__ void k_surface(Dims d, const double *__restrict__ cx, const double *__restrict__ cr,
                          const uint8_t *__restrict__ solid, const int *__restrict__ owner,
                          uint8_t *__restrict__ surface, int *__restrict__ count, T *__restrict__ psi_s,
                          int slabs) {
  const int j = blockIdx.x / slabs, sl = blockIdx.x - j * slabs;
  const double X[3] = {cx[3 * j], cx[3 * j + 1], cx[3 * j + 2]};
  const Box b = bbox(d, X, cr[j], 1.0);
  const long long tot = (long long)b.cnt[0] * b.cnt[1] * b.cnt[2];
  int mine = 0;
  for (long long t = (long long)sl * blockDim.x + threadIdx.x; t < tot; t += (long long)slabs * blockDim.x) {
    int x, y, z;
    box_site(d, b, t, x, y, z);
    const long long i = site(d, x, y, z);
    if (psi_s[i] > T(1)) psi_s[i] = T(1);
    if (!solid[i] || owner[i] != j) continue;
    long long nb[19];
    neighbours19(d, x, y, z, nb);
    bool any = false;
    for (int q = 1; q < 19; ++q) any |= !solid[nb[q]];
    if (any) {
      surface[i] = 1;
      ++mine;
    }
  }
  atomicAdd(count + j, mine);  // integer: exact in any order
}

template <typename T>
__global__ void k_charge(Dims d, const double *__restrict__ cx, const double *__restrict__ cr,
                         const double *__restrict__ cq, const uint8_t *__restrict__ surface,
                         const int *__restrict__ owner, const int *__restrict__ count, T *__restrict__ qc,
                         int slabs) {
  const int j = blockIdx.x / slabs, sl = blockIdx.x - j * slabs;
  const double X[3] = {cx[3 * j], cx[3 * j + 1], cx[3 * j + 2]};
  const Box b = bbox(d, X, cr[j], 1.0);
  const long long tot = (long long)b.cnt[0] * b.cnt[1] * b.cnt[2];
  const double val = count[j] > 0 ? __ddiv_rn(cq[j], double(count[j])) : 0.0;
  for (long long t = (long long)sl * blockDim.x + threadIdx.x; t < tot; t += (long long)slabs * blockDim.x) {
    int x, y, z;
    box_site(d, b, t, x, y, z);
    const long long i = site(d, x, y, z);
    if (surface[i] && owner[i] == j) qc[i] = T(val);
  }
}

template <typename T>
__global__ void k_psi_f(long long N, const uint8_t *__restrict__ solid, const T *__restrict__ psi_s,
                        T *__restrict__ psi_f) {
  long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (i >= N) return;
  psi_f[i] = solid[i] ? T(0) : T(1) - psi_s[i];
}

template <typename T> static void build(Ctx &c) {
  const long long N = c.d.N;
  cudaMemsetAsync(c.solid, 0, N, c.s);
  cudaMemsetAsync(c.surface, 0, N, c.s);
  cudaMemsetAsync(c.owner, 0xff, N * sizeof(int), c.s);  // -1
  cudaMemsetAsync(c.psi_s, 0, N * sizeof(T), c.s);
  cudaMemsetAsync(c.qc, 0, N * sizeof(T), c.s);
  if (c.ncoll > 0) {
    cudaMemsetAsync(c.ccount, 0, c.ncoll * sizeof(int), c.s);
    const int sl = colloid_slabs(c.ncoll);
    count_launch(), k_project<T><<<c.ncoll * sl, 256, 0, c.s>>>(c.d, c.h, c.cx, c.cr, c.solid, c.owner, (T *)c.psi_s, sl);
    count_launch(), k_surface<T><<<c.ncoll * sl, 256, 0, c.s>>>(c.d, c.cx, c.cr, c.solid, c.owner, c.surface, c.ccount,
                                                                 (T *)c.psi_s, sl);
    count_launch(), k_charge<T><<<c.ncoll * sl, 256, 0, c.s>>>(c.d, c.cx, c.cr, c.cq, c.surface, c.owner, c.ccount,
                                                                (T *)c.qc, sl);
  }
  count_launch(), k_psi_f<T><<<grid_for(N, 256), 256, 0, c.s>>>(N, c.solid, (const T *)c.psi_s, (T *)c.psi_f);
  c.geom_empty = c.ncoll == 0;
}

void geometry_build(Ctx &c) {
  if (c.prec == LBEH_FP64)
    build<double>(c);
  else
    build<float>(c);
}

}  // namespace lbeh
