/*
 * lbeh -- coupled electrohydrodynamic lattice step on one NVIDIA GB300 (sm_103a).
 *
 * The library advances the model of Rivas, Frijters, Pagonabarraga and
 * Harting, "Mesoscopic electrohydrodynamic simulations of binary colloidal
 * suspensions" (arXiv:1712.08494), Sec. II, one lattice timestep at a time:
 *   - two-component D3Q19 BGK stream-collide with Shan-Chen pseudopotential
 *     forcing (Sec. II.A, II.C eq. shanChenForce),
 *   - electric body forces: ion friction and Kelvin force (Sec. II.C),
 *   - link-flux Nernst-Planck update of two monovalent ion species on the
 *     D3Q7 faces with solid-fraction weighting (Sec. II.B, II.E),
 *   - variable-permittivity Poisson solve for the potential (Sec. II.B, II.D),
 *   - halfway bounce-back on colloid boundary links with the moving-wall term
 *     and momentum exchange, colloid projection and motion (Sec. II.E).
 *
 * Conventions for every entry point:
 *   - lattice units: dx = dt = e = beta = rho0 = 1;
 *   - scalar fields are nz*ny*nx arrays indexed (z*ny + y)*nx + x (x fastest);
 *     multi-component fields are stacked along a leading index;
 *   - component 0 is "a" (red, water), component 1 is "b" (blue, oil);
 *     ion species 0 is the cation (z=+1), species 1 the anion (z=-1);
 *   - D3Q19 velocity order: 0 rest; 1..6 = +x -x +y -y +z -z; then
 *     (1,1,0) (-1,-1,0) (1,-1,0) (-1,1,0) (1,0,1) (-1,0,-1) (1,0,-1) (-1,0,1)
 *     (0,1,1) (0,-1,-1) (0,1,-1) (0,-1,1);
 *   - every function returns LBEH_OK (0) or a negative LBEH_ERR_* code and
 *     never aborts; the caller owns every buffer it passes, the handle owns
 *     all device state it allocates; a handle is bound to one CUDA stream and
 *     must not be used from two host threads at once.
 */
#ifndef LBEH_H
#define LBEH_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define LBEH_OK 0
#define LBEH_ERR_INVALID_ARG (-1)
#define LBEH_ERR_OOM (-2)
#define LBEH_ERR_CUDA (-3)
#define LBEH_ERR_POISSON_NOT_CONVERGED (-4)
#define LBEH_ERR_NONFINITE (-5)
#define LBEH_ERR_BARRIER_TIMEOUT (-6)
#define LBEH_ERR_UNSUPPORTED (-7)

/* Arithmetic and storage of the populations.  FP64: all FP64.  FP32: FP32
 * compute and storage.  *_BF16STORE / *_FP16STORE: FP32 compute, populations
 * stored as f - w_q rho0_shift[sigma] in bf16 / fp16.  The potential is held
 * in FP64 (FP64 mode) or as a double-float pair of FP32 words (FP32 modes),
 * the Poisson residuals formed in that precision and the corrections in the
 * compute type. */
typedef enum {
  LBEH_FP64 = 0,
  LBEH_FP32 = 1,
  LBEH_FP32_BF16STORE = 2,
  LBEH_FP32_FP16STORE = 3
} lbeh_precision;

/* Model parameters (Sec. II).  Unused members may be zero. */
typedef struct lbeh_params {
  int nx, ny, nz;       /* periodic box, each >= 2 */
  int ncomp;            /* fluid components: 1 or 2 */
  int nions;            /* ion species: 0 or 2 */
  int prec;             /* lbeh_precision */
  double tau;           /* BGK relaxation time, equal for both components (Sec. II.A) */
  double G;             /* fluid-fluid Shan-Chen coupling G_ab, D3Q19-weighted (Sec. II.C) */
  double rho0_shift[2]; /* reduced-precision storage offset per component */
  double D;             /* ion diffusivity (Sec. II.B eq. ionicflux) */
  double bjerrum;       /* Bjerrum length l_B; eps_ref = 1/(4 pi l_B) (Sec. III.E) */
  double eps_r[2];      /* relative permittivity of components a, b (eq. dielectric_constant) */
  double eps_r_colloid; /* relative permittivity of the colloids (Sec. II.E) */
  double dmu[2];        /* Gibbs transfer energies of cation, anion (eq. solvation_potential) */
  double drho_a;        /* Delta rho^a of eq. solvation_potential */
  double E_ext[3];      /* applied uniform field (Sec. II.B potential split) */
  double poisson_tol;   /* stop when ||b - A phi||_2 / ||b||_2 < tol */
  int poisson_max_iter; /* multigrid cycles per step before LBEH_ERR_POISSON_NOT_CONVERGED */
  int ncolloid_max;     /* capacity of the colloid table (0: no colloids) */
  double rho_p;         /* colloid mass density, m = rho_p (4/3) pi r^3 (Sec. II.E) */
  double k_hertz;       /* Hertz stiffness (eq. colloid_interaction) */
  int psi_subdiv;       /* h: solid fraction from (h+1)^3 sub-cube centres (Sec. II.E) */
  int colloids_move;    /* 0: fixed colloids; 1: velocity-Verlet motion and remap */
  void *stream;         /* cudaStream_t all work is issued on (NULL: legacy default stream) */
  int poisson_solver;   /* LBEH_POISSON_AUTO (0), LBEH_POISSON_MULTIGRID or LBEH_POISSON_SPECTRAL */
} lbeh_params;

/* Poisson solvers (Sec. II.D).  Both solve the same flux-form equation to
 * poisson_tol; they differ in cost.  SPECTRAL: conjugate gradients
 * preconditioned by the constant-coefficient inverse of the seven-point
 * Laplacian computed with Hartley transforms (the Fourier method of Sec.
 * II.D); its iteration count grows with the permittivity contrast
 * eps_max / eps_min.  Each axis must factor into 2, 3, 5 and 7 and be at most
 * 512 long (256 in FP64), else lbeh_create returns LBEH_ERR_UNSUPPORTED.
 * MULTIGRID: geometric multigrid defect correction, robust at high contrast
 * (colloids).  AUTO: spectral for boxes without colloids whose contrast is at
 * most 4 and whose axes it supports, multigrid otherwise.  poisson_max_iter
 * counts multigrid cycles or conjugate-gradient iterations.  Batches always
 * use the multigrid (SPECTRAL there: LBEH_ERR_UNSUPPORTED). */
#define LBEH_POISSON_AUTO 0
#define LBEH_POISSON_MULTIGRID 1
#define LBEH_POISSON_SPECTRAL 2

#define LBEH_F64 0
#define LBEH_F32 1

/* Field buffers for lbeh_set_fields / lbeh_get_fields.  `dtype` (LBEH_F64 or
 * LBEH_F32) is the element type of rho, u, f, n and phi; `on_device` says
 * whether those pointers are device (1) or host (0) memory.  Colloid arrays
 * are always host FP64.  NULL members are skipped. */
typedef struct lbeh_fields {
  int dtype;
  int on_device;
  void *rho[2];  /* component densities; set: equilibrium initialisation */
  void *u;       /* [3][N] velocity for the equilibrium initialisation; get: physical velocity */
  void *f;       /* [ncomp][19][N] populations (set: overrides rho/u) */
  void *n[2];    /* cation, anion concentrations */
  void *phi;     /* internal potential (set: starting guess of the first solve; on an
                    FP32 handle, FP32 values become the high word of the pair) */
  int ncolloid;  /* number of colloids (<= ncolloid_max) */
  double *cx;    /* [ncolloid][3] centres (x, y, z) */
  double *cv;    /* [ncolloid][3] velocities */
  double *cq;    /* [ncolloid] total charges */
  double *cr;    /* [ncolloid] radii */
  double *cf;    /* get only: [ncolloid][3] total force of the last step */
} lbeh_fields;

/* Observables, all FP64. */
typedef struct lbeh_obs {
  double mass[2];        /* sum of rho^sigma over fluid nodes */
  double ions[2];        /* sum of n^+, n^- */
  double charge;         /* sum of n^+ - n^- plus the colloid charge */
  double momentum[3];    /* fluid momentum sum_x sum_sigma sum_q f c_q */
  double deformation;    /* (sqrt(Mzz)-sqrt(Mxx))/(sqrt(Mzz)+sqrt(Mxx)), weight max(0,c) */
  double centroid[3];    /* weighted centre of the drop */
  double colloid_v[3];   /* mean colloid velocity */
  double poisson_relres; /* relative residual of the last solve */
  int poisson_iters;     /* multigrid cycles or conjugate-gradient iterations of the last solve */
  int status;            /* sticky device status (LBEH_OK or an error code) */
  long long steps;       /* steps taken since the last lbeh_set_fields */
  int poisson_solver;    /* solver in use: LBEH_POISSON_MULTIGRID or _SPECTRAL (0: no potential) */
} lbeh_obs;

typedef struct lbeh_handle lbeh_handle;

/* Allocate the device state of one lattice system (model of Sec. II).
 * Copies *p.  Besides device memory the handle owns two non-blocking streams
 * (whole-step graph replay; host-to-device copies of lbeh_set_fields), both
 * ordered against p->stream with events.  Errors: INVALID_ARG (bad sizes or
 * flags), OOM, CUDA. */
int lbeh_create(const lbeh_params *p, lbeh_handle **out);

/* Load the state: colloids first (projection of Sec. II.E: solid nodes,
 * solid fraction, surface charge), then populations as the second-order
 * equilibrium of Sec. II.A at rho (and u, zero if NULL) on fluid nodes, or
 * the populations themselves; ions are zeroed on solid nodes.  Synchronous
 * with respect to the host buffers.  Errors: INVALID_ARG, CUDA. */
int lbeh_set_fields(lbeh_handle *h, const lbeh_fields *in);

/* Copy the state out (densities and physical velocity of the last step,
 * populations with the storage offset added back, ions, potential, colloid
 * table and forces).  Synchronises the handle's stream. */
int lbeh_get_fields(lbeh_handle *h, lbeh_fields *out);

/* Advance nsteps coupled timesteps (Sec. II: macro fields, Poisson solve,
 * ion fluxes, forces, Nernst-Planck update, forced BGK collision, streaming
 * with halfway bounce-back, colloid motion).  Work is issued on the handle's
 * stream; a Poisson solve that reaches poisson_max_iter cycles returns
 * LBEH_ERR_POISSON_NOT_CONVERGED and leaves the sticky status set. */
int lbeh_step(lbeh_handle *h, int nsteps);

/* Conserved sums, drop deformation and colloid drift, reduced on the device
 * in a fixed order (bitwise reproducible): per-site values in the compute
 * type, per-thread running sums in double-float words (FP32 modes, products
 * of the drop moments formed exactly) or FP64, block and grid sums in FP64.
 * Synchronises. */
int lbeh_observables(lbeh_handle *h, lbeh_obs *out);

/* Auxiliary read-outs for validation (host destination, FP64 unless noted):
 * fields of the last step or of the current geometry. */
#define LBEH_AUX_SOLID 0   /* uint8 [N] solid mask */
#define LBEH_AUX_OWNER 1   /* int32 [N] colloid id or -1 */
#define LBEH_AUX_PSI_S 2   /* [N] solid fraction */
#define LBEH_AUX_SURFACE 3 /* uint8 [N] surface (interface solid) nodes */
#define LBEH_AUX_QC 4      /* [N] colloid charge */
#define LBEH_AUX_EPS 5     /* [N] permittivity of the last step */
#define LBEH_AUX_Q 6       /* [N] charge density of the last step */
#define LBEH_AUX_RHO_V 7   /* [ncomp][N] densities incl. virtual densities */
#define LBEH_AUX_U 8       /* [3][N] physical velocity of the last step */
int lbeh_get_aux(lbeh_handle *h, int which, void *out_host);

/* Time-out of the grid-barrier waits of the one-launch Poisson solves: a
 * block that polls a barrier `polls` times (about 100 ns each) without every
 * block arriving raises an abort flag, every block returns, and the step
 * reports LBEH_ERR_BARRIER_TIMEOUT (sticky until lbeh_set_fields) instead of
 * hanging.  polls <= 0 restores the default of 2^24 (about two seconds).
 * Applies to later steps; errors: INVALID_ARG. */
int lbeh_set_wait_limit(lbeh_handle *h, long long polls);

/* Per-stage device time of lbeh_step, measured with CUDA events recorded on
 * the handle's stream around each stage, and the number of kernels the
 * library launched.  lbeh_profile_enable(h, 1) resets and starts the
 * accumulation (0 stops it); lbeh_profile_read synchronises the stream and
 * returns the totals since the last enable.  Stages: */
#define LBEH_STAGE_MACRO 0   /* macro fields + virtual densities */
#define LBEH_STAGE_POISSON 1 /* Poisson solve (includes its host convergence checks) */
#define LBEH_STAGE_COLLIDE 2 /* fused forces / fluxes / collision / streaming / bounce-back */
#define LBEH_STAGE_NP 3      /* Nernst-Planck update */
#define LBEH_STAGE_COLLOID 4 /* colloid momentum exchange, forces, motion */
#define LBEH_NSTAGES 5
typedef struct lbeh_profile {
  double ms[LBEH_NSTAGES];       /* summed device time per stage */
  long long calls[LBEH_NSTAGES]; /* stage executions */
  long long launches;            /* kernels launched by the library */
  long long poisson_cycles;      /* multigrid cycles of the Poisson solves */
} lbeh_profile;
int lbeh_profile_enable(lbeh_handle *h, int on);
int lbeh_profile_read(lbeh_handle *h, lbeh_profile *out);

/* Allocation-free observables, for callers that cannot allocate device
 * memory where they need the sums: code under a fixed memory budget that
 * forbids cudaMalloc, plugins that only hold borrowed device buffers, or
 * processes whose device allocator belongs to another runtime.  The paper has
 * no counterpart; it is a service entry point of this library.  Inputs are
 * the caller's device buffers: f [ncomp][19][N] populations of element type
 * `dtype` (LBEH_F64 or LBEH_F32, the layout lbeh_get_fields writes with
 * on_device = 1), n [2][N] ions (NULL when nions == 0), solid [N] uint8 mask
 * (NULL: all fluid), qc [N] FP64 colloid charge (NULL: none).  Fills mass,
 * ions, charge, momentum, deformation and centroid of *out exactly as
 * lbeh_observables defines them (other members zero); it ends with a
 * device-to-host copy of the sums and synchronises `stream`.  It calls no
 * allocator: its partial sums live in a static device array of
 * LBEH_NOALLOC_SCRATCH_BYTES that every GPU loading the library keeps until
 * exit, which limits N to LBEH_NOALLOC_MAX_SITES (larger boxes:
 * LBEH_ERR_INVALID_ARG, checked before any launch).  The first call in each
 * CUDA context looks that array's address up in that context (and may
 * initialise the device's primary context when none is current).  All calls
 * share the array; calls whose kernels overlap on the GPU race on it. */
#define LBEH_NOALLOC_MAX_SITES 16777216LL
#define LBEH_NOALLOC_SCRATCH_BYTES (1024 * 16 * 8 + 16 * 8)
int lbeh_observables_noalloc(int nx, int ny, int nz, int ncomp, int nions, int dtype, const void *f,
                             const void *n, const uint8_t *solid, const double *qc, lbeh_obs *out,
                             void *stream);

/* Gradients through nsteps coupled steps by the discrete adjoint.
 *
 * The objective is J = d_deformation * D(t_end) + sum f_bar . f(t_end)
 * + sum n_bar . n(t_end), with D the drop deformation of lbeh_observables
 * (second moments of w = max(c, 0), c = (rho_b - rho_a)/(rho_a + rho_b)).
 * lbeh_step_adjoint advances the handle by nsteps exactly as lbeh_step does,
 * keeping a checkpoint of (f, n) every ckpt_every steps and the potential of
 * every step, then sweeps backwards: each segment is recomputed from its
 * checkpoint, and each step is reversed by hand-written adjoint kernels (the
 * transposes of collision, streaming, Shan-Chen, Kelvin and friction forces,
 * ion face fluxes and upwind advection) plus one adjoint Poisson solve with
 * the same multigrid solver (the operator is symmetric).
 *
 * Supported: two components, nions 0 or 2 without solvation (dmu = 0), no
 * colloids, prec LBEH_FP64 or LBEH_FP32 (UNSUPPORTED otherwise).  Outputs:
 * dJ/dE_ext, dJ/dG, dJ/dQ = sum n0_bar . dn0_dQ for a caller-given
 * derivative of the initial ions with respect to a charge Q (for instance the
 * drop charge placement of a synthetic input), and optionally the adjoint
 * state at the start (f0_bar, n0_bar).  FP64 arrays; host or device per
 * on_device.  Synchronises.  Afterwards the handle is in the state lbeh_step
 * would leave (fields of the last step included).  A Poisson solve of either
 * sweep that misses its tolerance returns LBEH_ERR_POISSON_NOT_CONVERGED with
 * the gradients filled in. */
typedef struct lbeh_obs_seed {
  double d_deformation; /* dJ/dD of the final state */
  const double *f_bar;  /* optional [2][19][N]: dJ/df(t_end) */
  const double *n_bar;  /* optional [2][N]: dJ/dn(t_end) */
  int on_device;        /* f_bar and n_bar are device pointers */
} lbeh_obs_seed;

typedef struct lbeh_grads {
  double deformation;        /* D(t_end) */
  double dE_ext[3];          /* dJ/dE_ext */
  double dG;                 /* dJ/dG (Shan-Chen coupling) */
  double dQ;                 /* sum n0_bar . dn0_dQ (0 when dn0_dQ is NULL) */
  const double *dn0_dQ;      /* input, optional [2][N] */
  double *f0_bar;            /* output, optional [2][19][N]: dJ/df(t_start) */
  double *n0_bar;            /* output, optional [2][N]: dJ/dn(t_start) */
  int on_device;             /* dn0_dQ, f0_bar and n0_bar are device pointers */
  double forward_ms;         /* device time of the forward sweep */
  double adjoint_ms;         /* device time of the reverse sweep (recompute included) */
  long long adjoint_poisson_cycles; /* multigrid cycles of the adjoint Poisson solves */
} lbeh_grads;

int lbeh_step_adjoint(lbeh_handle *h, int nsteps, int ckpt_every, const lbeh_obs_seed *seed, lbeh_grads *out);

/* Batches of independent systems (the model of Sec. II on each, no coupling
 * between them), for parameter sweeps over many small boxes of uneven size.
 *
 * lbeh_create_batch allocates nbox systems, box b from per_box[b].  All boxes
 * share prec (LBEH_FP64 or LBEH_FP32), ncomp, nions and stream, and carry no
 * colloids (ncolloid_max = 0); each box's Poisson multigrid levels above its
 * coarse tail must have even extents (edges divisible by 8 suffice).
 * Errors: INVALID_ARG (mismatched or bad parameters), UNSUPPORTED (other
 * precisions, odd levels, no feasible launch shape), OOM, CUDA.
 *
 * lbeh_batch_box returns a handle to box b that the batch owns (valid until
 * lbeh_destroy of the batch; lbeh_destroy on it does nothing).  Load, read and
 * observe each box through it with lbeh_set_fields / lbeh_get_fields /
 * lbeh_get_aux / lbeh_observables; lbeh_step on it advances that box alone
 * with the single-system kernels.  Those calls on the batch handle itself
 * return INVALID_ARG.
 *
 * lbeh_step on the batch handle advances every box by nsteps with one
 * kernel launch, replayed from a CUDA graph: one thread-block cluster per
 * box runs the whole coupled step for all nsteps, separated by cluster
 * barriers.  lbeh_batch_step_sequential runs the same kernel once per box, in
 * box order; with the same launch shape the two give bitwise-identical
 * states.  Both synchronise the stream and return the first error status over
 * the boxes (each box keeps its own in lbeh_observables).
 *
 * The launch shape is the number of blocks (of 512 threads) per cluster, one
 * of 1, 2, 4, 8, 16.  lbeh_batch_tune times every feasible shape on
 * probe_steps steps from the current state (restored after each trial, so
 * the boxes' states are unchanged), keeps the fastest and reports it and its
 * time per step in ms.  lbeh_batch_set_shape fixes a shape (UNSUPPORTED if it
 * cannot launch); lbeh_batch_shape returns the current one. */
int lbeh_create_batch(const lbeh_params *per_box, int nbox, lbeh_handle **out);
int lbeh_batch_box(lbeh_handle *batch, int b, lbeh_handle **box);
int lbeh_batch_step_sequential(lbeh_handle *batch, int nsteps);
int lbeh_batch_tune(lbeh_handle *batch, int probe_steps, int *cluster_blocks, double *ms_per_step);
int lbeh_batch_set_shape(lbeh_handle *batch, int cluster_blocks);
int lbeh_batch_shape(lbeh_handle *batch);

/* Release all device state (a batch releases its boxes). */
void lbeh_destroy(lbeh_handle *h);

/* Text of the last CUDA failure seen by the handle (empty if none); owned by
 * the handle, valid until its next call. */
const char *lbeh_last_error(lbeh_handle *h);

/* Static description of a status code. */
const char *lbeh_status_string(int code);

#ifdef __cplusplus
}
#endif
#endif /* LBEH_H */
