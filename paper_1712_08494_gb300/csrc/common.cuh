// Device-side helpers shared by the kernels of the coupled lattice step.
//
// D3Q19 velocity set and weights of Sec. II.A (weights 1/3, 1/18, 1/36),
// periodic indexing, and the storage conversions of the reduced-precision
// population formats (populations kept as f - w_q rho0 in bf16 / fp16).
#pragma once

#include <cuda_runtime.h>
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <stdint.h>

#include "../../include/lbeh.h"

namespace lbeh {

// ------------------------------------------------------------------ lattice
// Order: 0 rest; 1..6 = +x -x +y -y +z -z; 7..18 face diagonals.
__host__ __device__ constexpr int cx(int q) {
  return (q == 1 || q == 7 || q == 9 || q == 11 || q == 13) ? 1
       : (q == 2 || q == 8 || q == 10 || q == 12 || q == 14) ? -1 : 0;
}
__host__ __device__ constexpr int cy(int q) {
  return (q == 3 || q == 7 || q == 10 || q == 15 || q == 17) ? 1
       : (q == 4 || q == 8 || q == 9 || q == 16 || q == 18) ? -1 : 0;
}
__host__ __device__ constexpr int cz(int q) {
  return (q == 5 || q == 11 || q == 14 || q == 15 || q == 18) ? 1
       : (q == 6 || q == 12 || q == 13 || q == 16 || q == 17) ? -1 : 0;
}
__host__ __device__ constexpr int opp(int q) { return q == 0 ? 0 : ((q & 1) ? q + 1 : q - 1); }
template <typename T>
__host__ __device__ constexpr T wq(int q) {
  return q == 0 ? T(1.0 / 3.0) : (q <= 6 ? T(1.0 / 18.0) : T(1.0 / 36.0));
}

// ------------------------------------------------------------------ storage
template <typename S, typename T> struct Store;
template <typename T> struct Store<double, T> {
  __device__ static T ld(const double *p, size_t i, T) { return T(p[i]); }
  __device__ static T ldc(const double *p, size_t i, T) { return T(p[i]); }
  __device__ static void st(double *p, size_t i, T v, T) { p[i] = double(v); }
};
template <typename T> struct Store<float, T> {
  __device__ static T ld(const float *p, size_t i, T) { return T(__ldg(p + i)); }
  __device__ static T ldc(const float *p, size_t i, T) { return T(p[i]); }
  __device__ static void st(float *p, size_t i, T v, T) { p[i] = float(v); }
};
template <typename T> struct Store<__nv_bfloat16, T> {
  __device__ static T ld(const __nv_bfloat16 *p, size_t i, T shift) {
    return T(__bfloat162float(p[i])) + shift;
  }
  __device__ static T ldc(const __nv_bfloat16 *p, size_t i, T shift) { return ld(p, i, shift); }
  __device__ static void st(__nv_bfloat16 *p, size_t i, T v, T shift) {
    p[i] = __float2bfloat16_rn(float(v - shift));
  }
};
template <typename T> struct Store<__half, T> {
  __device__ static T ld(const __half *p, size_t i, T shift) { return T(__half2float(p[i])) + shift; }
  __device__ static T ldc(const __half *p, size_t i, T shift) { return ld(p, i, shift); }
  __device__ static void st(__half *p, size_t i, T v, T shift) { p[i] = __float2half_rn(float(v - shift)); }
};

// ------------------------------------------------------------------ grid
struct Dims {
  int nx, ny, nz;
  long long N;
};

__device__ __forceinline__ int wrapp(int a, int n) { return a + 1 == n ? 0 : a + 1; }
__device__ __forceinline__ int wrapm(int a, int n) { return a == 0 ? n - 1 : a - 1; }
__device__ __forceinline__ int wrap(int a, int n) { return a < 0 ? a + n : (a >= n ? a - n : a); }

// Neighbour indices of site (x, y, z) for the 19 velocities.
__device__ __forceinline__ void neighbours19(const Dims &d, int x, int y, int z, long long nb[19]) {
  const int xs[3] = {wrapm(x, d.nx), x, wrapp(x, d.nx)};
  const int ys[3] = {wrapm(y, d.ny), y, wrapp(y, d.ny)};
  const int zs[3] = {wrapm(z, d.nz), z, wrapp(z, d.nz)};
#pragma unroll
  for (int q = 0; q < 19; ++q)
    nb[q] = ((long long)zs[cz(q) + 1] * d.ny + ys[cy(q) + 1]) * d.nx + xs[cx(q) + 1];
}

__device__ __forceinline__ long long site(const Dims &d, int x, int y, int z) {
  return ((long long)z * d.ny + y) * d.nx + x;
}

// Decomposition of a linear site index (boxes hold fewer than 2^31 sites, so
// 32-bit unsigned division suffices; 64-bit division is emulated and slow).
__device__ __forceinline__ void coords(const Dims &d, long long i, int &x, int &y, int &z) {
  const unsigned ii = unsigned(i);
  const unsigned r = ii / unsigned(d.nx);
  x = int(ii - r * unsigned(d.nx));
  const unsigned zz = r / unsigned(d.ny);
  z = int(zz);
  y = int(r - zz * unsigned(d.ny));
}

// Device status word bits (sticky until lbeh_set_fields).
enum : int { ST_POISSON = 1, ST_NONFINITE = 2, ST_TIMEOUT = 4 };

}  // namespace lbeh
