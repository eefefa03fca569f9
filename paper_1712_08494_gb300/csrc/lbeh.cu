// C-ABI of the coupled electrohydrodynamic lattice step (include/lbeh.h).
//
// The handle owns the device state of one periodic lattice system and issues
// all work on the caller's stream.  One step (Sec. II): macro fields and
// virtual densities, Poisson solve, fused forces/fluxes/collision/streaming
// with bounce-back, Nernst-Planck update, colloid momentum exchange.
#include <cmath>
#include <cstdlib>
#include <cstdio>
#include <cstring>
#include <new>
#include <vector>

#include "internal.h"

using namespace lbeh;

struct lbeh_handle {
  lbeh_params p;
  Ctx c;
  PrecOps ops;
  Poisson *pois = nullptr;
  std::vector<void *> allocs;
  int status = LBEH_OK;
  long long steps = 0;
  int last_iters = 0;
  double last_relres = 0.0;
  bool loaded = false;
  std::vector<double> hx, hv, hq, hr, hf;  // host copy of the colloid table
  // staging buffers of set/get calls, kept between calls (device memory is
  // not allocated and freed per call; a cudaFree synchronises the device)
  struct Stage {
    void *p;
    size_t bytes;
    bool busy;
  };
  std::vector<Stage> stage;
  // profiling: event pairs per executed stage, accumulated on read
  struct Mark {
    int stage;
    cudaEvent_t a, b;
  };
  bool prof = false;
  std::vector<Mark> marks;
  std::vector<cudaEvent_t> pool;
  double prof_ms[LBEH_NSTAGES] = {0};
  long long prof_calls[LBEH_NSTAGES] = {0};
  long long launches0 = 0;
  long long cycles0 = 0;
  char last_error[256] = {0};  // text of the last CUDA failure
  // whole-step CUDA graphs, one per ping-pong parity
  cudaStream_t gs = nullptr;           // capture / replay stream
  cudaEvent_t ev_in = nullptr, ev_out = nullptr;
  // host-to-device copies run on their own stream; work issued on the
  // handle's stream after a copy waits for it (ev_cp), so conversions of the
  // first inputs overlap the copies of the later ones
  cudaStream_t cs = nullptr;
  cudaEvent_t ev_fence = nullptr, ev_cp = nullptr;
  bool fenced = false;  // cs already ordered after the work issued on the handle's stream
  bool copied = false;  // ev_cp marks copies the host has not yet waited for
  cudaGraphExec_t exec[2] = {nullptr, nullptr};
  bool graphs_ready = false;
  bool eager = false;                  // LBEH_EAGER=1 disables graphs
  int graph_launches = 0;              // kernels per replay outside the Poisson cycles
  long long total_iters_seen = 0;      // Poisson cycles already accounted
  // batches: the batch handle owns its boxes; a box points back to its batch
  Batch *batch = nullptr;
  std::vector<lbeh_handle *> boxes;
  lbeh_handle *parent = nullptr;
  bool stats_stale = false;  // Poisson statistics not read back since a batched step
  Poisson *adj_pois = nullptr;  // solver of the adjoint Poisson problems (created on first use)
  long long wait_limit = 0;     // barrier-wait polls of the Poisson solves (0: default)
};

std::atomic<long long> lbeh::g_launches{0};

namespace {

template <typename A, typename B> __global__ void k_cvt(const A *__restrict__ a, B *__restrict__ b, long long n) {
  long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (i < n) b[i] = B(a[i]);
}

template <typename T>
__global__ void k_mask_fluid(T *__restrict__ a, const uint8_t *__restrict__ solid, long long N, int ncomp) {
  long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (i >= N || !solid[i]) return;
  for (int s = 0; s < ncomp; ++s) a[s * N + i] = T(0);
}

__global__ void k_add(double *__restrict__ acc, const double *__restrict__ v, int n) {
  if (threadIdx.x < n) acc[threadIdx.x] += v[threadIdx.x];
}

inline bool cuda_ok(cudaError_t e) { return e == cudaSuccess; }

cudaEvent_t take_event(lbeh_handle *h) {
  if (!h->pool.empty()) {
    cudaEvent_t e = h->pool.back();
    h->pool.pop_back();
    return e;
  }
  cudaEvent_t e = nullptr;
  cudaEventCreate(&e);
  return e;
}

void flush_marks(lbeh_handle *h) {
  if (h->marks.empty()) return;
  cudaStreamSynchronize(h->c.s);
  for (auto &m : h->marks) {
    float ms = 0.f;
    if (cudaEventElapsedTime(&ms, m.a, m.b) == cudaSuccess) {
      h->prof_ms[m.stage] += ms;
      h->prof_calls[m.stage] += 1;
    }
    h->pool.push_back(m.a);
    h->pool.push_back(m.b);
  }
  h->marks.clear();
}

struct StageTimer {
  lbeh_handle *h;
  lbeh_handle::Mark m;
  StageTimer(lbeh_handle *hh, int stage) : h(hh) {
    if (!h->prof) return;
    m.stage = stage;
    m.a = take_event(h);
    m.b = take_event(h);
    cudaEventRecord(m.a, h->c.s);
  }
  ~StageTimer() {
    if (!h->prof) return;
    cudaEventRecord(m.b, h->c.s);
    h->marks.push_back(m);
    if (h->marks.size() > 8192) flush_marks(h);
  }
};

void *dalloc(lbeh_handle *h, size_t bytes) {
  void *p = nullptr;
  if (cudaMalloc(&p, bytes) != cudaSuccess) return nullptr;
  h->allocs.push_back(p);
  return p;
}

size_t pop_bytes(int prec) { return prec == LBEH_FP64 ? 8 : (prec == LBEH_FP32 ? 4 : 2); }

// Stage `count` elements of the caller's buffer as FP64 on the device.
// Returns a device pointer (the caller's own if it already is FP64 device
// memory) and records temporaries in `tmp`.
// A staging buffer of at least `bytes` for the current call, taken from the
// handle's kept buffers (or allocated and kept); released by free_tmp.
// Buffers above kStageKeep are freed after the call instead of kept.
constexpr size_t kStageKeep = size_t(256) << 20;
void *stage_buf(lbeh_handle *h, size_t bytes, std::vector<void *> &tmp) {
  for (auto &b : h->stage)
    if (!b.busy && b.bytes >= bytes) {
      b.busy = true;
      tmp.push_back(b.p);
      return b.p;
    }
  void *p = nullptr;
  if (cudaMalloc(&p, bytes) != cudaSuccess) return nullptr;
  h->stage.push_back({p, bytes, true});
  tmp.push_back(p);
  return p;
}

// Host-to-device copy on the copy stream, ordered after the work already
// issued on the handle's stream (once per set call, else before each copy);
// work issued on the handle's stream afterwards waits for the copy.
void h2d(lbeh_handle *h, void *dst, const void *src, size_t bytes) {
  if (!h->cs) {  // handle without a copy stream: in order on its own stream
    cudaMemcpyAsync(dst, src, bytes, cudaMemcpyHostToDevice, h->c.s);
    return;
  }
  if (!h->fenced) {
    cudaEventRecord(h->ev_fence, h->c.s);
    cudaStreamWaitEvent(h->cs, h->ev_fence, 0);
  }
  cudaMemcpyAsync(dst, src, bytes, cudaMemcpyHostToDevice, h->cs);
  cudaEventRecord(h->ev_cp, h->cs);
  cudaStreamWaitEvent(h->c.s, h->ev_cp, 0);
  h->copied = true;
}

// host or device source into device memory
void copy_in(lbeh_handle *h, void *dst, const void *src, size_t bytes, int on_device) {
  if (on_device)
    cudaMemcpyAsync(dst, src, bytes, cudaMemcpyDeviceToDevice, h->c.s);
  else
    h2d(h, dst, src, bytes);
}

const double *stage_in(lbeh_handle *h, const void *src, int dtype, int on_device, long long count,
                       std::vector<void *> &tmp, double *dst = nullptr) {
  cudaStream_t s = h->c.s;
  if (on_device && dtype == LBEH_F64 && !dst) return (const double *)src;
  double *out = dst ? dst : (double *)stage_buf(h, count * 8, tmp);
  if (!out) return nullptr;
  if (dtype == LBEH_F64) {
    copy_in(h, out, src, count * 8, on_device);
    return out;
  }
  const float *fsrc = (const float *)src;
  if (!on_device) {
    float *fd = (float *)stage_buf(h, count * 4, tmp);
    if (!fd) return nullptr;
    h2d(h, fd, src, count * 4);
    fsrc = fd;
  }
  count_launch(), k_cvt<float, double><<<grid_for(count, 256), 256, 0, s>>>(fsrc, out, count);
  return out;
}

// Copy `count` FP64 device values to the caller's buffer in its dtype.
bool stage_out(lbeh_handle *h, const double *dsrc, void *dst, int dtype, int on_device, long long count,
               std::vector<void *> &tmp) {
  cudaStream_t s = h->c.s;
  if (dtype == LBEH_F64) {
    return cuda_ok(cudaMemcpyAsync(dst, dsrc, count * 8,
                                   on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, s));
  }
  float *fd = (float *)dst;
  if (!on_device) {
    fd = (float *)stage_buf(h, count * 4, tmp);
    if (!fd) return false;
  }
  count_launch(), k_cvt<double, float><<<grid_for(count, 256), 256, 0, s>>>(dsrc, fd, count);
  if (!on_device) return cuda_ok(cudaMemcpyAsync(dst, fd, count * 4, cudaMemcpyDeviceToHost, s));
  return true;
}

// FP64 device copy of a compute-type field.
const double *as_f64(lbeh_handle *h, const void *src, long long count, std::vector<void *> &tmp) {
  if (h->c.prec == LBEH_FP64) return (const double *)src;
  double *out = (double *)stage_buf(h, count * 8, tmp);
  if (!out) return nullptr;
  count_launch(), k_cvt<float, double><<<grid_for(count, 256), 256, 0, h->c.s>>>((const float *)src, out, count);
  return out;
}

void to_compute(lbeh_handle *h, const double *src, void *dst, long long count) {
  if (h->c.prec == LBEH_FP64)
    cudaMemcpyAsync(dst, src, count * 8, cudaMemcpyDeviceToDevice, h->c.s);
  else
    count_launch(), k_cvt<double, float><<<grid_for(count, 256), 256, 0, h->c.s>>>(src, (float *)dst, count);
}

// Load `count` values of the caller's array into a field held in the compute
// type; FP32 input to an FP32 field is copied as it is, without an FP64 stage.
bool load_compute(lbeh_handle *h, const void *src, int dtype, int on_device, long long count, void *dst,
                  std::vector<void *> &tmp) {
  if (h->c.prec != LBEH_FP64 && dtype == LBEH_F32) {
    copy_in(h, dst, src, count * 4, on_device);
    return true;
  }
  const double *d = stage_in(h, src, dtype, on_device, count, tmp);
  if (!d) return false;
  to_compute(h, d, dst, count);
  return true;
}

// Return staged buffers to the pool.  Without wait, the work still queued on
// the handle's stream may read them: every later use is ordered after it
// (same stream, or the copy stream behind a fence), and cudaFree of the
// large ones synchronises the device.
void free_tmp(lbeh_handle *h, std::vector<void *> &tmp, bool wait = true) {
  if (wait) cudaStreamSynchronize(h->c.s);
  for (void *t : tmp)
    for (size_t k = 0; k < h->stage.size(); ++k)
      if (h->stage[k].p == t) {
        if (h->stage[k].bytes > kStageKeep) {
          cudaFree(t);
          h->stage.erase(h->stage.begin() + (long)k);
        } else {
          h->stage[k].busy = false;
        }
        break;
      }
  tmp.clear();
}

int check_params(const lbeh_params *p) {
  if (!p) return LBEH_ERR_INVALID_ARG;
  if (p->nx < 2 || p->ny < 2 || p->nz < 2) return LBEH_ERR_INVALID_ARG;
  if ((long long)p->nx * p->ny * p->nz >= (1LL << 31)) return LBEH_ERR_INVALID_ARG;  // 32-bit site indices
  if (p->ncomp != 1 && p->ncomp != 2) return LBEH_ERR_INVALID_ARG;
  if (p->nions != 0 && p->nions != 2) return LBEH_ERR_INVALID_ARG;
  if (p->prec < LBEH_FP64 || p->prec > LBEH_FP32_FP16STORE) return LBEH_ERR_INVALID_ARG;
  if (!(p->tau > 0.5)) return LBEH_ERR_INVALID_ARG;
  if (p->nions && !(p->D > 0.0)) return LBEH_ERR_INVALID_ARG;
  if ((p->nions || p->ncolloid_max > 0) && !(p->bjerrum > 0.0)) return LBEH_ERR_INVALID_ARG;
  if (p->nions && (p->dmu[0] != 0.0 || p->dmu[1] != 0.0) && p->drho_a == 0.0) return LBEH_ERR_INVALID_ARG;
  if (p->ncolloid_max < 0 || p->psi_subdiv < 0 || p->psi_subdiv > 15) return LBEH_ERR_INVALID_ARG;
  if (p->poisson_max_iter < 0) return LBEH_ERR_INVALID_ARG;
  if (p->poisson_solver < LBEH_POISSON_AUTO || p->poisson_solver > LBEH_POISSON_SPECTRAL) return LBEH_ERR_INVALID_ARG;
  return LBEH_OK;
}

// Record the pending CUDA error (if any) in the handle and return LBEH_ERR_CUDA.
int cuda_fail(lbeh_handle *h, const char *where) {
  const cudaError_t e = cudaGetLastError();
  snprintf(h->last_error, sizeof(h->last_error), "%s: %s", where,
           e == cudaSuccess ? "failure reported by a CUDA call" : cudaGetErrorString(e));
  return LBEH_ERR_CUDA;
}

void drop_graphs(lbeh_handle *h) {
  for (int k = 0; k < 2; ++k)
    if (h->exec[k]) {
      cudaGraphExecDestroy(h->exec[k]);
      h->exec[k] = nullptr;
    }
  h->graphs_ready = false;
}

// Kernels of one coupled step on the context's stream (eager or captured).
// `handle` != 0: the Poisson cycles go under a conditional WHILE node.
int enqueue_step(lbeh_handle *h, Ctx &c, bool capture, cudaGraphConditionalHandle handle) {
  {
    StageTimer st(h, LBEH_STAGE_MACRO);
    h->ops.macro(c);
    h->ops.virt(c);
  }
  if (h->pois) {
    StageTimer st(h, LBEH_STAGE_POISSON);
    if (capture) {
      if (poisson_capture(h->pois, c, handle) != 0) return cuda_fail(h, "Poisson capture");
    } else {
      double rr = 0.0;
      const int it = poisson_solve(h->pois, c, &rr);
      if (it == -1) return cuda_fail(h, "Poisson solve");
      h->last_relres = rr;
      if (it < -1) {
        h->last_iters = -it - 2;
        h->status = LBEH_ERR_POISSON_NOT_CONVERGED;
      } else {
        h->last_iters = it;
      }
    }
  }
  {
    StageTimer st(h, LBEH_STAGE_COLLIDE);
    h->ops.collide(c);
    c.cur ^= 1;
  }
  if (c.nions) {
    StageTimer st(h, LBEH_STAGE_NP);
    h->ops.np(c);
    c.ncur ^= 1;
  }
  if (c.solids) {
    // colloid forces and motion, then the lattice remap (Sec. II.E)
    StageTimer st(h, LBEH_STAGE_COLLOID);
    h->ops.colloid_bb(c);
    colloid_forces_move(c);
    if (c.moving) {
      cudaMemcpyAsync(c.solid_old, c.solid, c.d.N, cudaMemcpyDeviceToDevice, c.s);
      cudaMemcpyAsync(c.owner_old, c.owner, 4 * c.d.N, cudaMemcpyDeviceToDevice, c.s);
      geometry_build(c);
      h->ops.remap(c);
      colloid_apply_dp(c);
    }
  }
  return LBEH_OK;
}

// Capture the step for both ping-pong parities into graphs on h->gs.
int build_graphs(lbeh_handle *h) {
  drop_graphs(h);
  const bool prof = h->prof;
  h->prof = false;
  int rc = LBEH_OK;
  for (int par = 0; par < 2 && rc == LBEH_OK; ++par) {
    Ctx cc = h->c;
    cc.s = h->gs;
    cc.cur = par;
    cc.ncur = cc.nions ? par : 0;
    const long long before = g_launches.load();
    if (cudaStreamBeginCapture(h->gs, cudaStreamCaptureModeThreadLocal) != cudaSuccess) {
      rc = cuda_fail(h, "begin capture");
      break;
    }
    cudaGraphConditionalHandle handle = 0;
    if (h->pois && poisson_needs_conditional(h->pois)) {
      cudaStreamCaptureStatus cs;
      cudaGraph_t g = nullptr;
      if (cudaStreamGetCaptureInfo(h->gs, &cs, nullptr, &g, nullptr, nullptr, nullptr) != cudaSuccess ||
          cudaGraphConditionalHandleCreate(&handle, g, 0, 0) != cudaSuccess)
        rc = LBEH_ERR_CUDA;
    }
    if (rc == LBEH_OK) rc = enqueue_step(h, cc, true, handle);
    cudaGraph_t graph = nullptr;
    const cudaError_t e = cudaStreamEndCapture(h->gs, &graph);
    h->graph_launches = int(g_launches.load() - before);
    g_launches.fetch_sub(h->graph_launches);  // captured, not launched
    if (rc == LBEH_OK && e != cudaSuccess) rc = cuda_fail(h, "end capture");
    if (rc == LBEH_OK && cudaGraphInstantiate(&h->exec[par], graph, 0) != cudaSuccess)
      rc = cuda_fail(h, "graph instantiate");
    if (graph) cudaGraphDestroy(graph);
  }
  h->prof = prof;
  if (rc != LBEH_OK) {
    drop_graphs(h);
    cudaGetLastError();
    return rc;
  }
  h->graphs_ready = true;
  return LBEH_OK;
}

}  // namespace

extern "C" {

const char *lbeh_status_string(int code) {
  switch (code) {
    case LBEH_OK: return "ok";
    case LBEH_ERR_INVALID_ARG: return "invalid argument";
    case LBEH_ERR_OOM: return "out of device memory";
    case LBEH_ERR_CUDA: return "CUDA error";
    case LBEH_ERR_POISSON_NOT_CONVERGED: return "Poisson solve did not reach its tolerance";
    case LBEH_ERR_NONFINITE: return "non-finite value in the state";
    case LBEH_ERR_BARRIER_TIMEOUT: return "device wait timed out";
    case LBEH_ERR_UNSUPPORTED: return "unsupported configuration";
    default: return "unknown status";
  }
}

int lbeh_create(const lbeh_params *p, lbeh_handle **out) {
  if (!out) return LBEH_ERR_INVALID_ARG;
  *out = nullptr;
  int rc = check_params(p);
  if (rc) return rc;
  lbeh_handle *h = new (std::nothrow) lbeh_handle;
  if (!h) return LBEH_ERR_OOM;
  h->p = *p;
  Ctx &c = h->c;
  c.d = Dims{p->nx, p->ny, p->nz, (long long)p->nx * p->ny * p->nz};
  c.ncomp = p->ncomp;
  c.nions = p->nions;
  c.prec = p->prec;
  c.s = (cudaStream_t)p->stream;
  c.tau = p->tau;
  c.G = p->ncomp == 2 ? p->G : 0.0;
  c.D = p->D;
  const double eps_ref = p->bjerrum > 0 ? 1.0 / (4.0 * M_PI * p->bjerrum) : 0.0;
  c.eps_a = p->eps_r[0] * eps_ref;
  c.eps_b = p->eps_r[1] * eps_ref;
  c.eps_p = p->eps_r_colloid * eps_ref;
  c.eps_bar = 0.5 * (c.eps_a + c.eps_b);
  for (int s = 0; s < 2; ++s) {
    c.dmd[s] = p->nions && p->drho_a != 0.0 ? p->dmu[s] / p->drho_a : 0.0;
    c.gas[s] = c.dmd[s] * 3.0;  // G_{a+-} = dmu / (drho_a c_s^2)
    c.shift[s] = (p->prec == LBEH_FP32_BF16STORE || p->prec == LBEH_FP32_FP16STORE) ? p->rho0_shift[s] : 0.0;
  }
  c.solvation = p->nions && (p->dmu[0] != 0.0 || p->dmu[1] != 0.0);
  for (int a = 0; a < 3; ++a) c.Eext[a] = p->E_ext[a];
  const bool eext = p->E_ext[0] != 0.0 || p->E_ext[1] != 0.0 || p->E_ext[2] != 0.0;
  c.has_field = p->nions > 0 || p->ncolloid_max > 0 || eext;
  c.h = p->psi_subdiv;
  c.ncoll_max = p->ncolloid_max;
  c.psolver = p->poisson_solver;
  if (c.has_field && p->poisson_solver == LBEH_POISSON_SPECTRAL && !poisson_spectral_choice(c, p->prec == LBEH_FP64)) {
    delete h;
    return LBEH_ERR_UNSUPPORTED;
  }
  switch (p->prec) {
    case LBEH_FP64: h->ops = ops_f64(); break;
    case LBEH_FP32: h->ops = ops_f32(); break;
    case LBEH_FP32_BF16STORE: h->ops = ops_bf16(); break;
    default: h->ops = ops_f16(); break;
  }
  const long long N = c.d.N;
  const size_t T = p->prec == LBEH_FP64 ? 8 : 4;
  const size_t pb = pop_bytes(p->prec) * 19 * p->ncomp * N;
  bool ok = true;
  ok &= (c.f[0] = dalloc(h, pb)) != nullptr;
  ok &= (c.f[1] = dalloc(h, pb)) != nullptr;
  ok &= (c.rho = dalloc(h, T * p->ncomp * N)) != nullptr;
  ok &= (c.psi = dalloc(h, T * p->ncomp * N)) != nullptr;
  ok &= (c.eps = dalloc(h, T * N)) != nullptr;
  ok &= (c.q = dalloc(h, T * N)) != nullptr;
  ok &= (c.u = dalloc(h, T * 3 * N)) != nullptr;
  if (p->prec == LBEH_FP64) {
    ok &= (c.phi = (double *)dalloc(h, 8 * N)) != nullptr;
    c.phit = c.phi;
  } else {
    ok &= (c.phit = dalloc(h, 4 * N)) != nullptr;
    ok &= (c.phi_lo = (float *)dalloc(h, 4 * N)) != nullptr;
  }
  ok &= (c.J = dalloc(h, T * 3 * N)) != nullptr;
  ok &= (c.psi_s = dalloc(h, T * N)) != nullptr;
  ok &= (c.psi_f = dalloc(h, T * N)) != nullptr;
  ok &= (c.qc = dalloc(h, T * N)) != nullptr;
  ok &= (c.solid = (uint8_t *)dalloc(h, N)) != nullptr;
  ok &= (c.surface = (uint8_t *)dalloc(h, N)) != nullptr;
  ok &= (c.owner = (int *)dalloc(h, 4 * N)) != nullptr;
  if (p->nions) {
    ok &= (c.n[0] = dalloc(h, T * 2 * N)) != nullptr;
    ok &= (c.n[1] = dalloc(h, T * 2 * N)) != nullptr;
    ok &= (c.flux = dalloc(h, T * 6 * N)) != nullptr;
  }
  const int nc = p->ncolloid_max > 0 ? p->ncolloid_max : 1;
  ok &= (c.cx = (double *)dalloc(h, 8 * 3 * nc)) != nullptr;
  ok &= (c.cv = (double *)dalloc(h, 8 * 3 * nc)) != nullptr;
  ok &= (c.cq = (double *)dalloc(h, 8 * nc)) != nullptr;
  ok &= (c.cr = (double *)dalloc(h, 8 * nc)) != nullptr;
  ok &= (c.cforce = (double *)dalloc(h, 8 * 3 * nc)) != nullptr;
  ok &= (c.cdp = (double *)dalloc(h, 8 * 3 * nc)) != nullptr;
  c.moving = p->colloids_move != 0 && p->ncolloid_max > 0;
  c.rho_p = p->rho_p;
  c.k_hertz = p->k_hertz;
  if (c.moving) {
    ok &= (c.solid_old = (uint8_t *)dalloc(h, N)) != nullptr;
    ok &= (c.owner_old = (int *)dalloc(h, 4 * N)) != nullptr;
    if (p->nions) {
      ok &= (c.remap_share = dalloc(h, T * 2 * N)) != nullptr;
      ok &= (c.remap_flag = (uint8_t *)dalloc(h, N)) != nullptr;
    }
  }
  ok &= (c.ccount = (int *)dalloc(h, 4 * nc)) != nullptr;
  ok &= (c.status = (int *)dalloc(h, sizeof(int))) != nullptr;
  c.red_len = (size_t)kRedBlocks * kObsLen + 64;
  ok &= (c.red = (double *)dalloc(h, 8 * c.red_len)) != nullptr;
  if (ok && c.has_field) {
    h->pois = poisson_create(c, p->prec == LBEH_FP64);
    ok &= h->pois != nullptr;
    if (h->pois) ok &= poisson_configure(h->pois, p->poisson_tol, p->poisson_max_iter, c.s) == 0;
  }
  ok &= cudaStreamCreateWithFlags(&h->gs, cudaStreamNonBlocking) == cudaSuccess;
  ok &= cudaEventCreateWithFlags(&h->ev_in, cudaEventDisableTiming) == cudaSuccess;
  ok &= cudaEventCreateWithFlags(&h->ev_out, cudaEventDisableTiming) == cudaSuccess;
  ok &= cudaStreamCreateWithFlags(&h->cs, cudaStreamNonBlocking) == cudaSuccess;
  ok &= cudaEventCreateWithFlags(&h->ev_fence, cudaEventDisableTiming) == cudaSuccess;
  ok &= cudaEventCreateWithFlags(&h->ev_cp, cudaEventDisableTiming) == cudaSuccess;
  {
    const char *e = getenv("LBEH_EAGER");
    h->eager = e && e[0] == '1';
  }
  if (!ok) {
    lbeh_destroy(h);
    return LBEH_ERR_OOM;
  }
  cudaMemsetAsync(c.u, 0, T * 3 * N, c.s);
  if (c.phi) cudaMemsetAsync(c.phi, 0, 8 * N, c.s);
  if (c.phi_lo) {
    cudaMemsetAsync(c.phit, 0, 4 * N, c.s);
    cudaMemsetAsync(c.phi_lo, 0, 4 * N, c.s);
  }
  cudaMemsetAsync(c.status, 0, sizeof(int), c.s);
  if (c.remap_flag) cudaMemsetAsync(c.remap_flag, 0, N, c.s);
  cudaMemsetAsync(c.cv, 0, 8 * 3 * nc, c.s);
  cudaMemsetAsync(c.cforce, 0, 8 * 3 * nc, c.s);
  if (p->nions) {
    cudaMemsetAsync(c.flux, 0, T * 6 * N, c.s);
    cudaMemsetAsync(c.n[0], 0, T * 2 * N, c.s);
  }
  geometry_build(c);  // empty geometry: all fluid, psi_f = 1
  if (cudaStreamSynchronize(c.s) != cudaSuccess) {
    lbeh_destroy(h);
    return LBEH_ERR_CUDA;
  }
  *out = h;
  return LBEH_OK;
}

static int batch_advance(lbeh_handle *h, int nsteps, bool sequential);

int lbeh_create_batch(const lbeh_params *per_box, int nbox, lbeh_handle **out) {
  if (!out) return LBEH_ERR_INVALID_ARG;
  *out = nullptr;
  if (!per_box || nbox < 1) return LBEH_ERR_INVALID_ARG;
  for (int b = 0; b < nbox; ++b) {
    const lbeh_params &p = per_box[b];
    if (p.stream != per_box[0].stream || p.prec != per_box[0].prec || p.ncomp != per_box[0].ncomp ||
        p.nions != per_box[0].nions || p.ncolloid_max != 0)
      return LBEH_ERR_INVALID_ARG;
    const int rc = check_params(&p);
    if (rc) return rc;
  }
  if (per_box[0].prec != LBEH_FP64 && per_box[0].prec != LBEH_FP32) return LBEH_ERR_UNSUPPORTED;
  lbeh_handle *h = new (std::nothrow) lbeh_handle;
  if (!h) return LBEH_ERR_OOM;
  h->p = per_box[0];
  h->c.s = (cudaStream_t)per_box[0].stream;
  std::vector<BatchBox> boxes;
  int rc = LBEH_OK;
  for (int b = 0; b < nbox; ++b)
    if (per_box[b].poisson_solver == LBEH_POISSON_SPECTRAL) {
      delete h;
      return LBEH_ERR_UNSUPPORTED;
    }
  for (int b = 0; b < nbox && rc == LBEH_OK; ++b) {
    lbeh_handle *bx = nullptr;
    lbeh_params pb = per_box[b];
    pb.poisson_solver = LBEH_POISSON_MULTIGRID;  // the batched kernel cycles the multigrid
    rc = lbeh_create(&pb, &bx);
    if (rc != LBEH_OK) break;
    bx->parent = h;
    h->boxes.push_back(bx);
    boxes.push_back(BatchBox{&bx->c, bx->pois});
  }
  if (rc == LBEH_OK) h->batch = batch_create(boxes, h->c.s, &rc);
  if (rc != LBEH_OK || !h->batch) {
    lbeh_destroy(h);
    return rc != LBEH_OK ? rc : LBEH_ERR_CUDA;
  }
  *out = h;
  return LBEH_OK;
}

int lbeh_batch_box(lbeh_handle *h, int b, lbeh_handle **box) {
  if (!h || !box || !h->batch || b < 0 || b >= (int)h->boxes.size()) return LBEH_ERR_INVALID_ARG;
  *box = h->boxes[b];
  return LBEH_OK;
}

int lbeh_batch_step_sequential(lbeh_handle *h, int nsteps) {
  if (!h || !h->batch || nsteps < 0) return LBEH_ERR_INVALID_ARG;
  return batch_advance(h, nsteps, true);
}

int lbeh_batch_set_shape(lbeh_handle *h, int cluster_blocks) {
  if (!h || !h->batch) return LBEH_ERR_INVALID_ARG;
  return batch_set_shape(h->batch, cluster_blocks);
}

int lbeh_batch_shape(lbeh_handle *h) {
  if (!h || !h->batch) return LBEH_ERR_INVALID_ARG;
  return batch_shape(h->batch);
}

int lbeh_batch_tune(lbeh_handle *h, int probe_steps, int *cluster_blocks, double *ms_per_step) {
  if (!h || !h->batch || probe_steps < 1) return LBEH_ERR_INVALID_ARG;
  for (lbeh_handle *bx : h->boxes)
    if (!bx->loaded) return LBEH_ERR_INVALID_ARG;
  return batch_tune(h->batch, probe_steps, cluster_blocks, ms_per_step);
}

int lbeh_set_wait_limit(lbeh_handle *h, long long polls) {
  if (!h || h->batch) return LBEH_ERR_INVALID_ARG;
  h->wait_limit = polls;
  if (h->pois) poisson_set_wait_limit(h->pois, polls);
  if (h->adj_pois) poisson_set_wait_limit(h->adj_pois, polls);
  drop_graphs(h);  // the captured launches carry the limit by value
  return LBEH_OK;
}

int lbeh_profile_enable(lbeh_handle *h, int on) {
  if (!h) return LBEH_ERR_INVALID_ARG;
  flush_marks(h);
  for (int k = 0; k < LBEH_NSTAGES; ++k) {
    h->prof_ms[k] = 0.0;
    h->prof_calls[k] = 0;
  }
  h->prof = on != 0;
  h->launches0 = g_launches.load();
  h->cycles0 = h->total_iters_seen;
  return LBEH_OK;
}

int lbeh_profile_read(lbeh_handle *h, lbeh_profile *out) {
  if (!h || !out) return LBEH_ERR_INVALID_ARG;
  flush_marks(h);
  for (int k = 0; k < LBEH_NSTAGES; ++k) {
    out->ms[k] = h->prof_ms[k];
    out->calls[k] = h->prof_calls[k];
  }
  out->launches = g_launches.load() - h->launches0;
  out->poisson_cycles = h->total_iters_seen - h->cycles0;
  return cudaGetLastError() == cudaSuccess ? LBEH_OK : LBEH_ERR_CUDA;
}

static void destroy_handle(lbeh_handle *h);

void lbeh_destroy(lbeh_handle *h) {
  if (!h || h->parent) return;  // boxes of a batch go with their batch
  if (h->batch || !h->boxes.empty()) {
    if (h->c.s) cudaStreamSynchronize(h->c.s);
    batch_destroy(h->batch);
    for (lbeh_handle *bx : h->boxes) destroy_handle(bx);
    delete h;
    return;
  }
  destroy_handle(h);
}

static void destroy_handle(lbeh_handle *h) {
  if (h->c.s) cudaStreamSynchronize(h->c.s);
  flush_marks(h);
  for (cudaEvent_t e : h->pool) cudaEventDestroy(e);
  drop_graphs(h);
  if (h->gs) {
    cudaStreamSynchronize(h->gs);
    cudaStreamDestroy(h->gs);
  }
  if (h->ev_in) cudaEventDestroy(h->ev_in);
  if (h->ev_out) cudaEventDestroy(h->ev_out);
  if (h->cs) {
    cudaStreamSynchronize(h->cs);
    cudaStreamDestroy(h->cs);
  }
  if (h->ev_fence) cudaEventDestroy(h->ev_fence);
  if (h->ev_cp) cudaEventDestroy(h->ev_cp);
  poisson_destroy(h->pois);
  poisson_destroy(h->adj_pois);
  for (void *a : h->allocs) cudaFree(a);
  for (auto &b : h->stage) cudaFree(b.p);
  delete h;
}

int lbeh_set_fields(lbeh_handle *h, const lbeh_fields *in) {
  if (!h || !in) return LBEH_ERR_INVALID_ARG;
  if (h->batch) return LBEH_ERR_INVALID_ARG;
  if (in->dtype != LBEH_F64 && in->dtype != LBEH_F32) return LBEH_ERR_INVALID_ARG;
  Ctx &c = h->c;
  const long long N = c.d.N;
  if (in->ncolloid < 0 || in->ncolloid > c.ncoll_max) return LBEH_ERR_INVALID_ARG;
  if (in->ncolloid > 0 && (!in->cx || !in->cr)) return LBEH_ERR_INVALID_ARG;
  if (!in->f && !in->rho[0]) return LBEH_ERR_INVALID_ARG;
  if (!in->f && c.ncomp == 2 && !in->rho[1]) return LBEH_ERR_INVALID_ARG;
  if (c.nions && (!in->n[0] || !in->n[1])) return LBEH_ERR_INVALID_ARG;
  std::vector<void *> tmp;

  // colloids and geometry
  const int nc = in->ncolloid;
  h->hx.assign(3 * nc, 0.0);
  h->hv.assign(3 * nc, 0.0);
  h->hq.assign(nc, 0.0);
  h->hr.assign(nc, 0.0);
  h->hf.assign(3 * nc, 0.0);
  for (int j = 0; j < nc; ++j) {
    for (int a = 0; a < 3; ++a) {
      h->hx[3 * j + a] = in->cx[3 * j + a];
      h->hv[3 * j + a] = in->cv ? in->cv[3 * j + a] : 0.0;
    }
    h->hq[j] = in->cq ? in->cq[j] : 0.0;
    h->hr[j] = in->cr[j];
    if (!(h->hr[j] > 0.0)) return LBEH_ERR_INVALID_ARG;
  }
  // the captured step depends on the host-side configuration only through
  // the colloid count (grids of the colloid kernels, the solid-node paths);
  // the rest of what is loaded here lives in device memory
  if (nc != c.ncoll || c.solids != (nc > 0)) drop_graphs(h);
  c.ncoll = nc;
  c.solids = nc > 0;
  if (nc) {
    cudaMemcpyAsync(c.cx, h->hx.data(), 8 * 3 * nc, cudaMemcpyHostToDevice, c.s);
    cudaMemcpyAsync(c.cv, h->hv.data(), 8 * 3 * nc, cudaMemcpyHostToDevice, c.s);
    cudaMemcpyAsync(c.cq, h->hq.data(), 8 * nc, cudaMemcpyHostToDevice, c.s);
    cudaMemcpyAsync(c.cr, h->hr.data(), 8 * nc, cudaMemcpyHostToDevice, c.s);
    cudaMemsetAsync(c.cforce, 0, 8 * 3 * nc, c.s);
  }
  if (nc > 0 || !c.geom_empty) geometry_build(c);  // no colloids before or now: nothing to rebuild

  // the host arrays go out on the copy stream behind one fence; what does
  // not depend on them is issued first, so that it overlaps the copies
  cudaEventRecord(h->ev_fence, c.s);
  cudaStreamWaitEvent(h->cs, h->ev_fence, 0);
  h->fenced = true;
  struct Unfence {
    lbeh_handle *h;
    ~Unfence() { h->fenced = false; }
  } unfence{h};
  cudaMemsetAsync(c.u, 0, (c.prec == LBEH_FP64 ? 8 : 4) * 3 * N, c.s);
  cudaMemsetAsync(c.status, 0, sizeof(int), c.s);
  if (h->pois && poisson_reset(h->pois, c.s) != 0) return LBEH_ERR_CUDA;
  const bool phi_hi_only = in->phi && !c.phi && in->dtype == LBEH_F32;
  if (!in->phi && c.phi) cudaMemsetAsync(c.phi, 0, 8 * N, c.s);
  if (!in->phi && !c.phi) cudaMemsetAsync(c.phit, 0, 4 * N, c.s);
  if ((!in->phi && !c.phi) || phi_hi_only) cudaMemsetAsync(c.phi_lo, 0, 4 * N, c.s);

  // populations
  c.cur = 0;
  c.ncur = 0;
  if (in->f) {
    const double *fd = stage_in(h, in->f, in->dtype, in->on_device, (long long)c.ncomp * 19 * N, tmp);
    if (!fd) { free_tmp(h, tmp); return LBEH_ERR_OOM; }
    h->ops.init_f(c, fd);
  } else if (in->dtype == LBEH_F32) {
    // FP32 densities (and velocities) feed the equilibrium directly
    float *rd = (float *)stage_buf(h, 4 * c.ncomp * N, tmp);
    if (!rd) { free_tmp(h, tmp); return LBEH_ERR_OOM; }
    for (int s = 0; s < c.ncomp; ++s) copy_in(h, rd + s * N, in->rho[s], 4 * N, in->on_device);
    const float *ud = (const float *)in->u;
    if (in->u && !in->on_device) {
      float *st = (float *)stage_buf(h, 4 * 3 * N, tmp);
      if (!st) { free_tmp(h, tmp); return LBEH_ERR_OOM; }
      h2d(h, st, in->u, 4 * 3 * N);
      ud = st;
    }
    h->ops.init_eq(c, rd, ud, 1);
  } else {
    double *rd = (double *)stage_buf(h, 8 * c.ncomp * N, tmp);
    if (!rd) { free_tmp(h, tmp); return LBEH_ERR_OOM; }
    for (int s = 0; s < c.ncomp; ++s)
      if (!stage_in(h, in->rho[s], in->dtype, in->on_device, N, tmp, rd + s * N)) {
        free_tmp(h, tmp);
        return LBEH_ERR_OOM;
      }
    const double *ud = nullptr;
    if (in->u) {
      ud = stage_in(h, in->u, in->dtype, in->on_device, 3 * N, tmp);
      if (!ud) { free_tmp(h, tmp); return LBEH_ERR_OOM; }
    }
    h->ops.init_eq(c, rd, ud, 0);
  }
  // ions, zero on solid nodes
  if (c.nions) {
    for (int s = 0; s < 2; ++s)
      if (!load_compute(h, in->n[s], in->dtype, in->on_device, N,
                        (char *)c.n[0] + (size_t)s * N * (c.prec == LBEH_FP64 ? 8 : 4), tmp)) {
        free_tmp(h, tmp);
        return LBEH_ERR_OOM;
      }
    if (c.solids) {
      if (c.prec == LBEH_FP64)
        count_launch(), k_mask_fluid<double><<<grid_for(N, 256), 256, 0, c.s>>>((double *)c.n[0], c.solid, N, 2);
      else
        count_launch(), k_mask_fluid<float><<<grid_for(N, 256), 256, 0, c.s>>>((float *)c.n[0], c.solid, N, 2);
    }
  }
  // potential: the starting guess of the first solve
  if (phi_hi_only) {
    // FP32 values are the high words of the double-float pair
    copy_in(h, c.phit, in->phi, 4 * N, in->on_device);
  } else if (in->phi) {
    const double *pd = stage_in(h, in->phi, in->dtype, in->on_device, N, tmp, c.phi);
    if (!pd) { free_tmp(h, tmp); return LBEH_ERR_OOM; }
    if (!c.phi) phi_from_double(c, pd);
  }
  h->status = LBEH_OK;
  h->steps = 0;
  h->last_iters = 0;
  h->last_relres = 0.0;
  h->loaded = true;
  // synchronous with respect to the host arrays: their copies have ended;
  // the conversions queued on the stream may still run
  if (h->copied) {
    cudaEventSynchronize(h->ev_cp);
    h->copied = false;
  }
  const cudaError_t e = cudaGetLastError();
  free_tmp(h, tmp, false);
  if (e != cudaSuccess) return LBEH_ERR_CUDA;
  return LBEH_OK;
}

static int batch_advance(lbeh_handle *h, int nsteps, bool sequential) {
  for (lbeh_handle *bx : h->boxes)
    if (!bx->loaded) return LBEH_ERR_INVALID_ARG;
  int st = 0;
  const int rc = batch_step(h->batch, nsteps, sequential, &st);
  if (rc != LBEH_OK) return cuda_fail(h, "batched step");
  for (size_t i = 0; i < h->boxes.size(); ++i) {
    lbeh_handle *bx = h->boxes[i];
    bx->steps += nsteps;
    bx->stats_stale = true;
    const int dst = batch_box_status(h->batch, (int)i);
    if (dst & ST_POISSON) bx->status = LBEH_ERR_POISSON_NOT_CONVERGED;
    if (dst & ST_NONFINITE) bx->status = LBEH_ERR_NONFINITE;
    if (dst & ST_TIMEOUT) bx->status = LBEH_ERR_BARRIER_TIMEOUT;
  }
  h->steps += nsteps;
  if (st & ST_TIMEOUT) return LBEH_ERR_BARRIER_TIMEOUT;
  if (st & ST_NONFINITE) return LBEH_ERR_NONFINITE;
  if (st & ST_POISSON) return LBEH_ERR_POISSON_NOT_CONVERGED;
  return LBEH_OK;
}

int lbeh_step(lbeh_handle *h, int nsteps) {
  if (!h || nsteps < 0) return LBEH_ERR_INVALID_ARG;
  if (h->batch) return batch_advance(h, nsteps, false);
  if (!h->loaded) return LBEH_ERR_INVALID_ARG;
  Ctx &c = h->c;
  if (nsteps == 0) return h->status;
  const bool graph = !h->eager && !h->prof;
  if (graph) {
    if (!h->graphs_ready) {
      int rc = build_graphs(h);
      if (rc != LBEH_OK) return rc;
    }
    // replay on the capture stream, ordered after and before the caller's stream
    cudaEventRecord(h->ev_in, c.s);
    cudaStreamWaitEvent(h->gs, h->ev_in, 0);
    for (int t = 0; t < nsteps; ++t) {
      if (cudaGraphLaunch(h->exec[c.cur], h->gs) != cudaSuccess) return cuda_fail(h, "graph launch");
      g_launches.fetch_add(h->graph_launches);
      c.cur ^= 1;
      if (c.nions) c.ncur ^= 1;
      ++h->steps;
    }
    cudaEventRecord(h->ev_out, h->gs);
    cudaStreamWaitEvent(c.s, h->ev_out, 0);
  } else {
    for (int t = 0; t < nsteps; ++t) {
      int rc = enqueue_step(h, c, false, 0);
      if (rc != LBEH_OK) return rc;
      ++h->steps;
    }
  }
  if (h->pois) {
    PoissonStats ps;
    if (poisson_read(h->pois, graph ? h->gs : c.s, &ps) != 0) return cuda_fail(h, "Poisson read-back");
    if (cudaStreamSynchronize(c.s) != cudaSuccess) return cuda_fail(h, "step synchronise");
    if (graph) {
      g_launches.fetch_add((ps.total_iters - h->total_iters_seen) * ps.body_launches);
      h->last_iters = ps.iters;
      h->last_relres = ps.relres;
    }
    h->total_iters_seen = ps.total_iters;
    int dst = 0;
    cudaMemcpy(&dst, c.status, sizeof(int), cudaMemcpyDeviceToHost);
    if (dst & ST_POISSON) h->status = LBEH_ERR_POISSON_NOT_CONVERGED;
    if (dst & ST_NONFINITE) h->status = LBEH_ERR_NONFINITE;
    if (dst & ST_TIMEOUT) h->status = LBEH_ERR_BARRIER_TIMEOUT;
  }
  if (cudaPeekAtLastError() != cudaSuccess) return cuda_fail(h, "step");
  return h->status;
}

const char *lbeh_last_error(lbeh_handle *h) { return h ? h->last_error : "no handle"; }

// Fixed-order FP64 sums of the observables (layout of k_obs) on the host.
static int obs_sums(lbeh_handle *h, double v[kObsLen]) {
  Ctx &c = h->c;
  const int nb = h->ops.obs_partials(c, c.red, kRedBlocks);
  double *res = c.red + (size_t)kRedBlocks * kObsLen;
  reduce_partials_final(c.red, nb, kObsLen, res, c.s);
  cudaMemcpyAsync(v, res, sizeof(double) * kObsLen, cudaMemcpyDeviceToHost, c.s);
  return cudaStreamSynchronize(c.s) == cudaSuccess ? LBEH_OK : LBEH_ERR_CUDA;
}

int lbeh_observables(lbeh_handle *h, lbeh_obs *out) {
  if (!h || !out) return LBEH_ERR_INVALID_ARG;
  if (h->batch) return LBEH_ERR_INVALID_ARG;
  Ctx &c = h->c;
  std::memset(out, 0, sizeof(*out));
  double v[kObsLen];
  if (obs_sums(h, v) != LBEH_OK) return LBEH_ERR_CUDA;
  for (int m = 0; m < kObsLen; ++m)
    if (!std::isfinite(v[m])) h->status = LBEH_ERR_NONFINITE;
  out->mass[0] = v[0];
  out->mass[1] = v[1];
  out->ions[0] = v[2];
  out->ions[1] = v[3];
  out->charge = v[4];
  for (int a = 0; a < 3; ++a) out->momentum[a] = v[5 + a];
  if (v[8] > 0) {
    const double W = v[8];
    for (int a = 0; a < 3; ++a) out->centroid[a] = v[9 + a] / W;
    const double mxx = v[12] - W * out->centroid[0] * out->centroid[0];
    const double mzz = v[13] - W * out->centroid[2] * out->centroid[2];
    const double a = std::sqrt(mxx > 0 ? mxx : 0), b = std::sqrt(mzz > 0 ? mzz : 0);
    out->deformation = (a + b) > 0 ? (b - a) / (b + a) : 0.0;
  }
  if (c.ncoll) {
    std::vector<double> cv(3 * c.ncoll);
    cudaMemcpy(cv.data(), c.cv, 8 * 3 * c.ncoll, cudaMemcpyDeviceToHost);
    for (int j = 0; j < c.ncoll; ++j)
      for (int a = 0; a < 3; ++a) out->colloid_v[a] += cv[3 * j + a] / c.ncoll;
  }
  if (h->stats_stale && h->pois) {
    PoissonStats ps;
    if (poisson_read(h->pois, c.s, &ps) == 0) {
      h->last_iters = ps.iters;
      h->last_relres = ps.relres;
      h->total_iters_seen = ps.total_iters;
    }
    h->stats_stale = false;
  }
  out->poisson_relres = h->last_relres;
  out->poisson_iters = h->last_iters;
  out->status = h->status;
  out->steps = h->steps;
  out->poisson_solver = h->pois ? (poisson_is_spectral(h->pois) ? LBEH_POISSON_SPECTRAL : LBEH_POISSON_MULTIGRID) : 0;
  return LBEH_OK;
}

// ---------------------------------------------------------------- adjoint
namespace {
struct DevArena {
  std::vector<void *> blocks;
  bool ok = true;
  void *get(size_t bytes) {
    void *p = nullptr;
    if (bytes == 0) return nullptr;
    if (cudaMalloc(&p, bytes) != cudaSuccess) {
      ok = false;
      cudaGetLastError();
      return nullptr;
    }
    blocks.push_back(p);
    return p;
  }
  ~DevArena() {
    for (void *p : blocks) cudaFree(p);
  }
};
}  // namespace

int lbeh_step_adjoint(lbeh_handle *h, int nsteps, int ckpt_every, const lbeh_obs_seed *seed, lbeh_grads *out) {
  if (!h || h->batch || !seed || !out || nsteps < 1 || ckpt_every < 1 || !h->loaded) return LBEH_ERR_INVALID_ARG;
  Ctx &c = h->c;
  if (c.ncomp != 2 || c.ncoll_max > 0 || c.solvation || (c.prec != LBEH_FP64 && c.prec != LBEH_FP32))
    return LBEH_ERR_UNSUPPORTED;
  const AdjOps A = c.prec == LBEH_FP64 ? adj_ops_f64() : adj_ops_f32();
  const size_t e = A.elem;
  const long long N = c.d.N;
  const size_t popB = e * 38 * N, ionB = c.nions ? e * 2 * N : 0, phiB = e * N, stB = popB + ionB;
  const int K = std::min(ckpt_every, nsteps);
  const int nseg = (nsteps + K - 1) / K;
  const double *dn_user = out->dn0_dQ;
  double *f0_user = out->f0_bar, *n0_user = out->n0_bar;
  const int out_dev = out->on_device;

  DevArena M;
  char *ck = (char *)M.get(nseg * stB);
  char *phis = (char *)M.get((size_t)nsteps * phiB);
  char *seg = (char *)M.get((size_t)(K + 1) * stB);
  void *fb[2] = {M.get(popB), M.get(popB)};
  void *nbf[2] = {M.get(ionB), M.get(ionB)};
  AdjArgs a{};
  void *rb = M.get(e * 2 * N), *Jb = M.get(e * 3 * N), *Felb = M.get(e * 3 * N), *KC = M.get(e * 3 * N);
  void *Sb = M.get(e * 6 * N), *psib = M.get(e * 2 * N), *epsb = M.get(e * N), *Eb = M.get(e * 3 * N);
  void *qadj = M.get(e * N);
  void *Fb = M.get(c.nions ? e * 6 * N : 0), *Efb = M.get(c.nions ? e * 3 * N : 0);
  void *lam = M.get(c.prec == LBEH_FP64 ? 8 * N : 4 * N), *lam_lo = c.prec == LBEH_FP64 ? nullptr : M.get(4 * N);
  double *part = (double *)M.get(8 * (size_t)kAdjBlocks * kAdjPar);
  double *acc = (double *)M.get(8 * 16);
  int *astatus = (int *)M.get(sizeof(int));  // status word of the adjoint solves
  // last-step fields of the forward sweep (the reverse sweep reuses their buffers)
  void *keep_rho = M.get(e * 2 * N), *keep_eps = M.get(e * N), *keep_q = M.get(e * N), *keep_u = M.get(e * 3 * N);
  if (!M.ok) return LBEH_ERR_OOM;
  cudaMemsetAsync(astatus, 0, sizeof(int), c.s);

  // adjoint Poisson problem: same permittivity, right-hand side -(qadj - mean), no applied field
  Ctx ca = c;
  ca.q = qadj;
  ca.status = astatus;
  ca.Eext[0] = ca.Eext[1] = ca.Eext[2] = 0.0;
  if (c.prec == LBEH_FP64) {
    ca.phi = (double *)lam;
    ca.phit = lam;
  } else {
    ca.phit = lam;
    ca.phi_lo = (float *)lam_lo;
  }
  if (c.has_field) {
    if (!h->adj_pois) {
      h->adj_pois = poisson_create(ca, c.prec == LBEH_FP64);
      if (!h->adj_pois) return LBEH_ERR_OOM;
      poisson_set_wait_limit(h->adj_pois, h->wait_limit);
    }
    if (poisson_configure(h->adj_pois, h->p.poisson_tol, h->p.poisson_max_iter, c.s) != 0 ||
        poisson_reset(h->adj_pois, c.s) != 0)
      return cuda_fail(h, "adjoint Poisson setup");
  }
  cudaMemsetAsync(lam, 0, c.prec == LBEH_FP64 ? 8 * N : 4 * N, c.s);
  if (lam_lo) cudaMemsetAsync(lam_lo, 0, 4 * N, c.s);

  cudaEvent_t ev[3];
  for (auto &x : ev) cudaEventCreate(&x);
  auto finish = [&](int rc) {
    cudaStreamSynchronize(c.s);
    for (auto &x : ev) cudaEventDestroy(x);
    return rc;
  };

  // forward sweep: checkpoints of (f, n) every K steps, the potential of every step
  cudaEventRecord(ev[0], c.s);
  int worst = LBEH_OK;
  for (int t = 0; t < nsteps; ++t) {
    if (t % K == 0) {
      char *dst = ck + (size_t)(t / K) * stB;
      cudaMemcpyAsync(dst, c.f[c.cur], popB, cudaMemcpyDeviceToDevice, c.s);
      if (ionB) cudaMemcpyAsync(dst + popB, c.n[c.ncur], ionB, cudaMemcpyDeviceToDevice, c.s);
    }
    const int rc = lbeh_step(h, 1);
    if (rc != LBEH_OK && rc != LBEH_ERR_POISSON_NOT_CONVERGED) return finish(rc);
    if (rc != LBEH_OK) worst = rc;
    cudaMemcpyAsync(phis + (size_t)t * phiB, c.phit, phiB, cudaMemcpyDeviceToDevice, c.s);
  }
  cudaEventRecord(ev[1], c.s);
  cudaMemcpyAsync(keep_rho, c.rho, e * 2 * N, cudaMemcpyDeviceToDevice, c.s);
  cudaMemcpyAsync(keep_eps, c.eps, e * N, cudaMemcpyDeviceToDevice, c.s);
  cudaMemcpyAsync(keep_q, c.q, e * N, cudaMemcpyDeviceToDevice, c.s);
  cudaMemcpyAsync(keep_u, c.u, e * 3 * N, cudaMemcpyDeviceToDevice, c.s);

  // objective and its adjoint seed at the final state
  double v[kObsLen];
  if (obs_sums(h, v) != LBEH_OK) return finish(cuda_fail(h, "adjoint objective"));
  double mom[4] = {0, 0, 0, 0}, D = 0.0;
  if (v[8] > 0) {
    const double W = v[8], X = v[9] / W, Z = v[11] / W;
    const double mxx = v[12] - W * X * X, mzz = v[13] - W * Z * Z;
    const double ax = std::sqrt(mxx > 0 ? mxx : 0), bz = std::sqrt(mzz > 0 ? mzz : 0);
    D = (ax + bz) > 0 ? (bz - ax) / (bz + ax) : 0.0;
    mom[0] = X;
    mom[1] = Z;
    mom[2] = ax;
    mom[3] = bz;
  }
  std::vector<void *> tmp;
  cudaMemsetAsync(fb[0], 0, popB, c.s);
  if (ionB) cudaMemsetAsync(nbf[0], 0, ionB, c.s);
  if (seed->f_bar) {
    const double *s = stage_in(h, seed->f_bar, LBEH_F64, seed->on_device, 38 * N, tmp);
    if (!s) return finish(LBEH_ERR_OOM);
    to_compute(h, s, fb[0], 38 * N);
  }
  if (seed->n_bar && ionB) {
    const double *s = stage_in(h, seed->n_bar, LBEH_F64, seed->on_device, 2 * N, tmp);
    if (!s) return finish(LBEH_ERR_OOM);
    to_compute(h, s, nbf[0], 2 * N);
  }
  if (seed->d_deformation != 0.0 && v[8] > 0) A.seed(c, c.f[c.cur], fb[0], mom, seed->d_deformation);
  cudaMemsetAsync(acc, 0, 8 * 16, c.s);

  // reverse sweep, segment by segment from the last
  int cur = 0;
  long long cycles = 0;
  auto step_ctx = [&](int t, int j) {
    Ctx cc = c;
    cc.f[0] = seg + (size_t)j * stB;
    cc.f[1] = seg + (size_t)(j + 1) * stB;
    cc.cur = 0;
    if (ionB) {
      cc.n[0] = seg + (size_t)j * stB + popB;
      cc.n[1] = seg + (size_t)(j + 1) * stB + popB;
    }
    cc.ncur = 0;
    cc.phit = phis + (size_t)t * phiB;
    if (c.prec == LBEH_FP64) cc.phi = (double *)cc.phit;
    return cc;
  };
  for (int sg = nseg - 1; sg >= 0; --sg) {
    const int ts = sg * K, L = std::min(nsteps, ts + K) - ts;
    cudaMemcpyAsync(seg, ck + (size_t)sg * stB, stB, cudaMemcpyDeviceToDevice, c.s);
    for (int j = 0; j + 1 < L; ++j) {
      Ctx cc = step_ctx(ts + j, j);
      h->ops.macro(cc);
      h->ops.collide(cc);
      if (ionB) h->ops.np(cc);
    }
    for (int j = L - 1; j >= 0; --j) {
      Ctx cc = step_ctx(ts + j, j);
      h->ops.macro(cc);
      h->ops.collide(cc);  // fields of the step: rho, J, psi, eps, q, u, face fluxes
      a.f = cc.f[0];
      a.n = ionB ? cc.n[0] : nullptr;
      a.rho = c.rho;
      a.J = c.J;
      a.psi = c.psi;
      a.eps = c.eps;
      a.phi = cc.phit;
      a.u = c.u;
      a.flux = c.flux;
      a.fbo = fb[cur];
      a.fbn = fb[cur ^ 1];
      a.nbo = nbf[cur];
      a.nbn = nbf[cur ^ 1];
      a.rb = rb;
      a.Jb = Jb;
      a.Felb = Felb;
      a.KC = KC;
      a.Sb = Sb;
      a.psib = psib;
      a.epsb = epsb;
      a.Fb = Fb;
      a.Efb = Efb;
      a.Eb = Eb;
      a.qadj = qadj;
      a.lam = lam;
      cudaMemsetAsync(part, 0, 8 * (size_t)kAdjBlocks * kAdjPar, c.s);
      A.before_solve(cc, a, part);
      if (c.has_field) {
        double rr = 0.0;
        const int it = poisson_solve(h->adj_pois, ca, &rr);
        if (it == -1) return finish(cuda_fail(h, "adjoint Poisson solve"));
        if (it < -1) {
          worst = LBEH_ERR_POISSON_NOT_CONVERGED;
          cycles += -it - 2;
        } else {
          cycles += it;
        }
      }
      A.after_solve(cc, a, part);
      reduce_partials_final(part, kAdjBlocks, kAdjPar, acc + 8, c.s);
      count_launch(), k_add<<<1, 32, 0, c.s>>>(acc, acc + 8, kAdjPar);
      cur ^= 1;
    }
  }
  cudaEventRecord(ev[2], c.s);
  cudaMemcpyAsync(c.rho, keep_rho, e * 2 * N, cudaMemcpyDeviceToDevice, c.s);
  cudaMemcpyAsync(c.eps, keep_eps, e * N, cudaMemcpyDeviceToDevice, c.s);
  cudaMemcpyAsync(c.q, keep_q, e * N, cudaMemcpyDeviceToDevice, c.s);
  cudaMemcpyAsync(c.u, keep_u, e * 3 * N, cudaMemcpyDeviceToDevice, c.s);

  // results
  double hacc[kAdjPar];
  cudaMemcpyAsync(hacc, acc, sizeof(hacc), cudaMemcpyDeviceToHost, c.s);
  if (cudaStreamSynchronize(c.s) != cudaSuccess) return finish(cuda_fail(h, "adjoint sweep"));
  out->deformation = D;
  for (int k = 0; k < 3; ++k) out->dE_ext[k] = hacc[k];
  out->dG = hacc[3];
  out->dQ = 0.0;
  const double *n0 = nullptr;
  if (ionB) {
    n0 = as_f64(h, nbf[cur], 2 * N, tmp);
    if (!n0) return finish(LBEH_ERR_OOM);
  }
  if (dn_user && n0) {
    const double *dn = stage_in(h, dn_user, LBEH_F64, out_dev, 2 * N, tmp);
    if (!dn) return finish(LBEH_ERR_OOM);
    out->dQ = dot_f64(n0, dn, 2 * N, c.red, c.s);
  }
  if (n0_user) {
    if (n0) {
      if (!stage_out(h, n0, n0_user, LBEH_F64, out_dev, 2 * N, tmp)) return finish(LBEH_ERR_CUDA);
    } else if (out_dev) {
      cudaMemsetAsync(n0_user, 0, 8 * 2 * N, c.s);
    } else {
      std::memset(n0_user, 0, 8 * 2 * N);
    }
  }
  if (f0_user) {
    const double *f0 = as_f64(h, fb[cur], 38 * N, tmp);
    if (!f0 || !stage_out(h, f0, f0_user, LBEH_F64, out_dev, 38 * N, tmp)) return finish(LBEH_ERR_CUDA);
  }
  free_tmp(h, tmp);
  float ms1 = 0.f, ms2 = 0.f;
  cudaEventElapsedTime(&ms1, ev[0], ev[1]);
  cudaEventElapsedTime(&ms2, ev[1], ev[2]);
  out->forward_ms = ms1;
  out->adjoint_ms = ms2;
  out->adjoint_poisson_cycles = cycles;
  if (cudaPeekAtLastError() != cudaSuccess) return finish(cuda_fail(h, "adjoint"));
  return finish(worst);
}

int lbeh_get_fields(lbeh_handle *h, lbeh_fields *out) {
  if (!h || !out) return LBEH_ERR_INVALID_ARG;
  if (h->batch) return LBEH_ERR_INVALID_ARG;
  if (out->dtype != LBEH_F64 && out->dtype != LBEH_F32) return LBEH_ERR_INVALID_ARG;
  Ctx &c = h->c;
  const long long N = c.d.N;
  std::vector<void *> tmp;
  bool ok = true;
  if (out->rho[0] || out->rho[1]) {
    double *rd = (double *)stage_buf(h, 8 * c.ncomp * N, tmp);
    if (!rd) return LBEH_ERR_OOM;
    h->ops.get_rho(c, rd);
    for (int s = 0; s < c.ncomp; ++s)
      if (out->rho[s]) ok &= stage_out(h, rd + s * N, out->rho[s], out->dtype, out->on_device, N, tmp);
  }
  if (out->f) {
    double *fd = nullptr;
    fd = (decltype(fd))stage_buf(h, 8 * (size_t)c.ncomp * 19 * N, tmp);
    if (!fd) { free_tmp(h, tmp); return LBEH_ERR_OOM; }
    h->ops.get_f(c, fd);
    ok &= stage_out(h, fd, out->f, out->dtype, out->on_device, (long long)c.ncomp * 19 * N, tmp);
  }
  if (out->u) {
    const double *ud = as_f64(h, c.u, 3 * N, tmp);
    ok &= ud && stage_out(h, ud, out->u, out->dtype, out->on_device, 3 * N, tmp);
  }
  if (c.nions) {
    const double *nd = as_f64(h, c.n[c.ncur], 2 * N, tmp);
    for (int s = 0; s < 2; ++s)
      if (out->n[s]) ok &= nd && stage_out(h, nd + s * N, out->n[s], out->dtype, out->on_device, N, tmp);
  }
  if (out->phi) {
    double *pd = nullptr;
    pd = (decltype(pd))stage_buf(h, 8 * N, tmp);
    if (!pd) { free_tmp(h, tmp); return LBEH_ERR_OOM; }
    phi_to_double(c, pd);
    ok &= stage_out(h, pd, out->phi, out->dtype, out->on_device, N, tmp);
  }
  const int nc = c.ncoll;
  if (nc && (out->cx || out->cv || out->cf)) {
    if (out->cx) cudaMemcpyAsync(out->cx, c.cx, 8 * 3 * nc, cudaMemcpyDeviceToHost, c.s);
    if (out->cv) cudaMemcpyAsync(out->cv, c.cv, 8 * 3 * nc, cudaMemcpyDeviceToHost, c.s);
    if (out->cf) cudaMemcpyAsync(out->cf, c.cforce, 8 * 3 * nc, cudaMemcpyDeviceToHost, c.s);
  }
  if (nc && out->cq) std::memcpy(out->cq, h->hq.data(), 8 * nc);
  if (nc && out->cr) std::memcpy(out->cr, h->hr.data(), 8 * nc);
  out->ncolloid = nc;
  const cudaError_t e = cudaGetLastError();
  free_tmp(h, tmp);
  if (!ok || e != cudaSuccess) return LBEH_ERR_CUDA;
  return LBEH_OK;
}

int lbeh_get_aux(lbeh_handle *h, int which, void *out_host) {
  if (!h || !out_host) return LBEH_ERR_INVALID_ARG;
  Ctx &c = h->c;
  const long long N = c.d.N;
  std::vector<void *> tmp;
  bool ok = true;
  switch (which) {
    case LBEH_AUX_SOLID: ok = cuda_ok(cudaMemcpyAsync(out_host, c.solid, N, cudaMemcpyDeviceToHost, c.s)); break;
    case LBEH_AUX_SURFACE:
      ok = cuda_ok(cudaMemcpyAsync(out_host, c.surface, N, cudaMemcpyDeviceToHost, c.s));
      break;
    case LBEH_AUX_OWNER: ok = cuda_ok(cudaMemcpyAsync(out_host, c.owner, 4 * N, cudaMemcpyDeviceToHost, c.s)); break;
    case LBEH_AUX_PSI_S:
    case LBEH_AUX_QC:
    case LBEH_AUX_EPS:
    case LBEH_AUX_Q: {
      void *src = which == LBEH_AUX_PSI_S ? c.psi_s : which == LBEH_AUX_QC ? c.qc : which == LBEH_AUX_EPS ? c.eps : c.q;
      const double *d = as_f64(h, src, N, tmp);
      ok = d && stage_out(h, d, out_host, LBEH_F64, 0, N, tmp);
      break;
    }
    case LBEH_AUX_RHO_V: {
      const double *d = as_f64(h, c.rho, (long long)c.ncomp * N, tmp);
      ok = d && stage_out(h, d, out_host, LBEH_F64, 0, (long long)c.ncomp * N, tmp);
      break;
    }
    case LBEH_AUX_U: {
      const double *d = as_f64(h, c.u, 3 * N, tmp);
      ok = d && stage_out(h, d, out_host, LBEH_F64, 0, 3 * N, tmp);
      break;
    }
    default: return LBEH_ERR_INVALID_ARG;
  }
  const cudaError_t e = cudaGetLastError();
  free_tmp(h, tmp);
  return (ok && e == cudaSuccess) ? LBEH_OK : LBEH_ERR_CUDA;
}

}  // extern "C"
