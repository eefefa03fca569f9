// Host-side interfaces between the translation units of the library.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <atomic>
#include <utility>
#include <vector>

#include "common.cuh"

namespace lbeh {

// Kernel launches made by the library (process-wide, read as differences).
extern std::atomic<long long> g_launches;
inline void count_launch() { g_launches.fetch_add(1, std::memory_order_relaxed); }

// Everything a launch needs: sizes, model constants and device pointers.
// Field pointers are of the compute type T (double for FP64, float otherwise)
// unless noted; populations are of the storage type of the precision mode.
struct Ctx {
  Dims d;
  int ncomp = 1, nions = 0, prec = LBEH_FP32;
  bool solids = false;      // colloids present
  bool geom_empty = false;  // geometry arrays hold the empty geometry (no colloids)
  bool has_field = false;   // potential or applied field present
  bool solvation = false;   // dmu != 0
  double tau = 1, G = 0, D = 0;
  double gas[2] = {0, 0};   // G_{a+-} = dmu / (drho_a c_s^2)
  double dmd[2] = {0, 0};   // dmu / drho_a
  double eps_a = 0, eps_b = 0, eps_p = 0, eps_bar = 0;
  double Eext[3] = {0, 0, 0};
  double shift[2] = {0, 0};
  int h = 3;                // solid-fraction subdivision
  int psolver = 0;          // Poisson solver: LBEH_POISSON_AUTO, _MULTIGRID or _SPECTRAL

  void *f[2] = {nullptr, nullptr};  // populations ping-pong [ncomp][19][N]
  int cur = 0;
  void *rho = nullptr;     // [ncomp][N] incl. virtual densities
  void *psi = nullptr;     // [ncomp][N]
  void *eps = nullptr;     // [N]
  void *q = nullptr;       // [N]
  void *n[2] = {nullptr, nullptr};  // ions ping-pong [2][N]
  int ncur = 0;
  void *u = nullptr;       // [3][N]
  void *flux = nullptr;    // [2][3][N]
  void *psi_s = nullptr;   // [N]
  void *psi_f = nullptr;   // [N]
  void *qc = nullptr;      // [N]
  double *phi = nullptr;   // [N] FP64 potential (FP64 mode)
  void *phit = nullptr;    // [N] potential in the compute type: aliases phi in FP64 mode; in the
                           // FP32 modes the high words of the double-float potential phit + phi_lo
  float *phi_lo = nullptr; // [N] low words of the double-float potential (FP32 modes)
  void *J = nullptr;       // [3][N] momentum sum_sigma sum_q f c_q
  uint8_t *solid = nullptr, *surface = nullptr;
  int *owner = nullptr;
  uint8_t *solid_old = nullptr;  // geometry before the colloid move (moving colloids)
  int *owner_old = nullptr;

  int ncoll = 0, ncoll_max = 0;
  double *cx = nullptr, *cv = nullptr, *cq = nullptr, *cr = nullptr;  // device colloid table
  double *cforce = nullptr;  // [ncoll][3] total force of the step
  double *cdp = nullptr;     // [ncoll][3] momentum change of the remap
  void *remap_share = nullptr;    // [2][N] ion share of each covered node (moving colloids with ions)
  uint8_t *remap_flag = nullptr;  // [N] receives a share this remap (kept zero between remaps)
  bool moving = false;
  double rho_p = 5.0, k_hertz = 1.0;
  int *ccount = nullptr;     // [ncoll] surface node counts
  int *status = nullptr;     // device status word

  long long launches = 0;    // kernels launched (all launch sites count here)
  double *red = nullptr;     // reduction scratch (FP64)
  size_t red_len = 0;
  cudaStream_t s = nullptr;
};

// Per-storage-type kernels (defined in step_<prec>.cu).
struct PrecOps {
  // rho [ncomp][N], u [3][N] or null: device arrays, FP32 if f32 else FP64
  void (*init_eq)(Ctx &, const void *rho, const void *u, int f32);
  void (*init_f)(Ctx &, const double *f);                      // [ncomp][19][N] FP64 device
  void (*get_f)(Ctx &, double *f);                             // [ncomp][19][N] FP64 device
  void (*get_rho)(Ctx &, double *rho);                         // [ncomp][N] FP64 device
  void (*macro)(Ctx &);
  void (*virt)(Ctx &);
  void (*collide)(Ctx &);
  void (*np)(Ctx &);
  int (*obs_partials)(Ctx &, double *partials, int max_blocks);  // kObsLen doubles per block; returns the blocks
  void (*colloid_bb)(Ctx &);                                    // momentum exchange + electric force into cforce
  void (*remap)(Ctx &);                                         // node covering / uncovering after a move
};
PrecOps ops_f64();
PrecOps ops_f32();
PrecOps ops_bf16();
PrecOps ops_f16();

// The projection kernels spread each colloid's bounding box over several
// blocks (slabs of its cells), about 1024 blocks in all and at most
// kColloidSlabsMax per colloid; what they accumulate (solid fractions of
// dyadic values, owner maxima, surface counts) is exact in any order.
constexpr int kColloidSlabsMax = 16;
inline int colloid_slabs(int ncoll) {
  if (ncoll < 1) return 1;
  const int s = (1024 + ncoll - 1) / ncoll;
  return s > kColloidSlabsMax ? kColloidSlabsMax : (s < 1 ? 1 : s);
}
constexpr int kObsLen = 16;  // see step_kernels.cuh obs layout
constexpr int kRedBlocks = 512;

// Colloid dynamics (colloids.cu): pair forces added to cforce, velocity-Verlet
// when moving; velocity update by the remap momentum.
void colloid_forces_move(Ctx &c);
void colloid_apply_dp(Ctx &c);

// Geometry (geometry.cu).
void geometry_build(Ctx &c);  // solid, owner, psi_s, psi_f, surface, ccount, qc

// Poisson (poisson.cu).
struct Poisson;
struct PoissonStats {
  int iters = 0;             // cycles of the last solve
  double relres = 0.0;       // relative residual of the last solve
  long long total_iters = 0; // cycles since creation
  int notconv = 0;           // last solve hit the cycle cap
  int body_launches = 0;     // kernels per cycle inside a captured graph
};
// Solver of the box: the spectral solve (spectral.cu) when c.psolver asks for
// it, or, by default, for boxes without colloid capacity whose permittivity contrast
// is at most kSpectralMaxContrast and whose axes the transforms support; the
// multigrid otherwise.  Null on failure.
constexpr double kSpectralMaxContrast = 4.0;
bool poisson_spectral_choice(const Ctx &c, int fp64);
Poisson *poisson_create(const Ctx &c, int fp64);
bool poisson_is_spectral(const Poisson *p);
// Polls of a grid-barrier wait before the solve gives up (LBEH_ERR_BARRIER_TIMEOUT).
void poisson_set_wait_limit(Poisson *p, long long polls);
void poisson_destroy(Poisson *p);
int poisson_configure(Poisson *p, double tol, int max_iter, cudaStream_t s);
int poisson_reset(Poisson *p, cudaStream_t s);  // new state: no previous solution to extrapolate from
// Eager solve for c.phi from c.eps and c.q: returns the cycle count, -(count+2)
// if the cap was reached before the tolerance, -1 on a CUDA error.
int poisson_solve(Poisson *p, Ctx &c, double *relres);
// Records the solve into the graph being captured on c.s, its cycles under a
// conditional WHILE node driven by `handle`.  Returns 0 or -1.
int poisson_capture(Poisson *p, Ctx &c, cudaGraphConditionalHandle handle);
int poisson_read(Poisson *p, cudaStream_t s, PoissonStats *out);
// false when the whole solve is one cooperative launch (no conditional node)
bool poisson_needs_conditional(const Poisson *p);
// Arguments of the whole solve of this system by one team of blocks (the
// batched step): writes PArgs<double> (FP64) or PArgs<float> (double-float
// potential) into `out` (out_bytes must match) and returns the dynamic shared
// memory of the tail cycle, or -1 when the level structure needs the
// multi-kernel solve.
long long poisson_team_args(Poisson *p, const Ctx &c, void *out, size_t out_bytes);
// Device buffers the solve carries from step to step (previous solution,
// solver state): (pointer, bytes) pairs.
void poisson_state_buffers(Poisson *p, const Ctx &c, std::vector<std::pair<void *, size_t>> &out);
void phi_to_double(Ctx &c, double *out);       // FP64 values of the potential
void phi_from_double(Ctx &c, const double *in);

// Batched step (batch.cu; kernels in batch_<prec>.cu).
struct BatchBox {
  Ctx *c;
  Poisson *pois;  // null: no potential
};
struct BatchKernels {
  size_t rec_bytes = 0;                                // device record of one system
  long long (*fill)(const BatchBox &, void *rec) = nullptr;  // tail shared memory, or -1
  const void *(*kernel)(int ncomp, int nions) = nullptr;
};
BatchKernels batch_kernels_f64();
BatchKernels batch_kernels_f32();
struct Batch;
// Boxes share precision (FP64 or FP32), ncomp, nions and stream; their status
// words are moved into one array owned by the batch.  rc receives the error.
Batch *batch_create(const std::vector<BatchBox> &boxes, cudaStream_t s, int *rc);
void batch_destroy(Batch *b);
// nsteps steps of every box: one graph-launched kernel (sequential = false) or
// one launch per box in box order.  Flips the boxes' parities; returns the
// first non-zero device status word over the boxes (0 when all are clear).
int batch_step(Batch *b, int nsteps, bool sequential, int *first_status);
int batch_set_shape(Batch *b, int cluster_blocks);  // LBEH_OK or LBEH_ERR_UNSUPPORTED
int batch_shape(const Batch *b);
int batch_box_status(const Batch *b, int box);  // status word of a box read by the last batch_step
// Times each feasible cluster size on probe_steps steps (state restored after
// each) and keeps the fastest.
int batch_tune(Batch *b, int probe_steps, int *best_blocks, double *best_ms_per_step);

// Discrete adjoint of the coupled step (adjoint_<prec>.cu): kernel passes of
// one reversed step on plain device arrays in the compute type.
struct AdjArgs {
  const void *f, *n;                                     // forward state at t
  const void *rho, *J, *psi, *eps, *phi, *u, *flux;      // forward fields of step t
  const void *fbo, *nbo;                                 // adjoint state at t+1
  void *fbn, *nbn;                                       // adjoint state at t
  void *rb, *Jb, *Felb, *KC, *Sb, *psib, *epsb, *Fb, *Efb, *Eb, *qadj;  // work arrays
  const void *lam;                                       // adjoint potential (compute type)
};
constexpr int kAdjBlocks = 1024;  // fixed grid of the passes with parameter sums
constexpr int kAdjPar = 4;        // dJ/dE_x, dJ/dE_y, dJ/dE_z, dJ/dG per block
struct AdjOps {
  // passes before the adjoint Poisson solve (its right-hand side lands in qadj)
  void (*before_solve)(const Ctx &, const AdjArgs &, double *part) = nullptr;
  // passes after it (lam holds the solution); completes fbn and nbn
  void (*after_solve)(const Ctx &, const AdjArgs &, double *part) = nullptr;
  // adds scale * dD/df of the drop deformation to fb; mom = {X, Z, sqrt(Mxx), sqrt(Mzz)}
  void (*seed)(const Ctx &, const void *f, void *fb, const double mom[4], double scale) = nullptr;
  size_t elem = 0;
};
AdjOps adj_ops_f64();
AdjOps adj_ops_f32();

// Deterministic FP64 reductions (reduce.cu).
void reduce_partials_final(const double *partials, int nblocks, int len, double *out, cudaStream_t s);
double dot_f64(const double *a, const double *b, long long n, double *scratch, cudaStream_t s);
double sum_f64(const double *a, long long n, double *scratch, cudaStream_t s);

inline int grid_for(long long n, int block) { return int((n + block - 1) / block); }

// Raise (never lower) a kernel's dynamic shared-memory limit: the limit is a
// property of the kernel shared by every system in the process, so a smaller
// system created later must not shrink what an earlier one launches with.
inline bool raise_smem_limit(const void *fn, size_t bytes) {
  cudaFuncAttributes a{};
  if (cudaFuncGetAttributes(&a, fn) != cudaSuccess) return false;
  if ((size_t)a.maxDynamicSharedSizeBytes >= bytes) return true;
  return cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes) == cudaSuccess;
}

}  // namespace lbeh
