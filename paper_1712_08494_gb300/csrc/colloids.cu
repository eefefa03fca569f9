// Colloid dynamics (Sec. II.E): pair forces and velocity-Verlet motion.
//
// Total force on colloid i: the momentum exchanged on its bounce-back links
// plus the electric force on its surface charge (both summed by k_colloid_bb),
// plus Hertz contact k_H delta^{3/2} along the line of centres (repulsive) and
// the lubrication force -(3 pi/2) eta r_i r_j n (n.(v_i - v_j)) (1/h - 1) for
// surface gaps 0 < h < 2/3, eta = c_s^2 (tau - 1/2) (eqs. colloid_interaction,
// lubrication).  Motion: x += v + F/(2m), v += F/m, m = rho_p (4/3) pi r^3,
// positions wrapped into the periodic box.  After the lattice remap the
// colloid's velocity takes the momentum of covered and uncovered nodes.
#include <cmath>

#include "internal.h"

namespace lbeh {

__device__ __forceinline__ double min_image_d(double d, int n) {
  if (d > 0.5 * n) return d - n;
  if (d < -0.5 * n) return d + n;
  return d;
}

// Pair forces on colloid i (block i, partners strided over the threads,
// fixed-order block sum), added to the force of the step.
__global__ void __launch_bounds__(128) k_colloid_pairs(Dims dm, int nc, const double *__restrict__ cx,
                                                       const double *__restrict__ cv, const double *__restrict__ cr,
                                                       double *__restrict__ cforce, double k_hertz, double eta) {
  const int i = blockIdx.x;
  const int dims[3] = {dm.nx, dm.ny, dm.nz};
  double F[3] = {0.0, 0.0, 0.0};
  for (int j = threadIdx.x; j < nc; j += blockDim.x) {
    if (j == i) continue;
    double dd[3];
    for (int a = 0; a < 3; ++a) dd[a] = min_image_d(cx[3 * i + a] - cx[3 * j + a], dims[a]);
    const double dist = sqrt(dd[0] * dd[0] + dd[1] * dd[1] + dd[2] * dd[2]);
    if (dist == 0.0) continue;
    const double nh[3] = {dd[0] / dist, dd[1] / dist, dd[2] / dist};
    const double overlap = cr[i] + cr[j] - dist;
    if (overlap > 0.0) {
      const double fh = k_hertz * overlap * sqrt(overlap);
      for (int a = 0; a < 3; ++a) F[a] += fh * nh[a];
    }
    const double gap = dist - (cr[i] + cr[j]);
    if (gap > 0.0 && gap < 2.0 / 3.0) {
      double vrel = 0.0;
      for (int a = 0; a < 3; ++a) vrel += nh[a] * (cv[3 * i + a] - cv[3 * j + a]);
      const double fl = -1.5 * M_PI * eta * cr[i] * cr[j] * vrel * (1.0 / gap - 1.0);
      for (int a = 0; a < 3; ++a) F[a] += fl * nh[a];
    }
  }
  __shared__ double sh[3][128];
  for (int a = 0; a < 3; ++a) sh[a][threadIdx.x] = F[a];
  __syncthreads();
  for (int w = blockDim.x / 2; w > 0; w >>= 1) {
    if (threadIdx.x < w)
      for (int a = 0; a < 3; ++a) sh[a][threadIdx.x] += sh[a][threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x < 3) cforce[3 * i + threadIdx.x] += sh[threadIdx.x][0];
}

// velocity-Verlet with the step's force held over the step
__global__ void k_colloid_move(Dims dm, int nc, double *__restrict__ cx, double *__restrict__ cv,
                               const double *__restrict__ cr, const double *__restrict__ cforce, double rho_p) {
  const int dims[3] = {dm.nx, dm.ny, dm.nz};
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < nc; i += gridDim.x * blockDim.x) {
    const double m = rho_p * (4.0 / 3.0) * M_PI * cr[i] * cr[i] * cr[i];
    for (int a = 0; a < 3; ++a) {
      const double acc = cforce[3 * i + a] / m;
      double x = cx[3 * i + a] + cv[3 * i + a] + 0.5 * acc;
      if (x < 0.0) x += dims[a];
      if (x >= dims[a]) x -= dims[a];
      cx[3 * i + a] = x;
      cv[3 * i + a] += acc;
    }
  }
}

__global__ void k_colloid_apply_dp(int nc, double *__restrict__ cv, const double *__restrict__ cr,
                                   const double *__restrict__ dp, double rho_p) {
  for (int i = threadIdx.x; i < nc; i += blockDim.x) {
    const double m = rho_p * (4.0 / 3.0) * M_PI * cr[i] * cr[i] * cr[i];
    for (int a = 0; a < 3; ++a) cv[3 * i + a] += dp[3 * i + a] / m;
  }
}

void colloid_forces_move(Ctx &c) {
  if (c.ncoll == 0) return;
  const double eta = (c.tau - 0.5) / 3.0;
  count_launch(), k_colloid_pairs<<<c.ncoll, 128, 0, c.s>>>(c.d, c.ncoll, c.cx, c.cv, c.cr, c.cforce, c.k_hertz, eta);
  if (c.moving)
    count_launch(), k_colloid_move<<<grid_for(c.ncoll, 128), 128, 0, c.s>>>(c.d, c.ncoll, c.cx, c.cv, c.cr, c.cforce,
                                                                          c.rho_p);
}

void colloid_apply_dp(Ctx &c) {
  if (c.ncoll == 0) return;
  count_launch(), k_colloid_apply_dp<<<1, 256, 0, c.s>>>(c.ncoll, c.cv, c.cr, c.cdp, c.rho_p);
}

}  // namespace lbeh
