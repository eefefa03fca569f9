// Host side of the batched step: the device table of systems, the cluster
// launch (one persistent launch for all systems, captured in a CUDA graph, or
// one launch per system), and the launch-shape autotuner.
//
// The table is ordered by decreasing system size, so the largest systems are
// dispatched first and the small ones fill in behind them.  The cluster size
// (blocks per system) is the tunable shape: it fixes how many SMs share one
// system and the order of its reductions; the batched and the per-system
// launches of one shape give identical results.
#include <algorithm>
#include <cstring>
#include <map>
#include <numeric>
#include <utility>
#include <vector>

#include "internal.h"

namespace lbeh {

namespace {
constexpr int kBatchThreads = 512;  // kPB of the Poisson team code
const int kShapes[] = {1, 2, 4, 8, 16};
}  // namespace

struct Batch {
  std::vector<BatchBox> boxes;  // user order
  std::vector<int> order;       // table position -> box
  std::vector<int> pos;         // box -> table position
  BatchKernels K;
  const void *kern = nullptr;
  void *table = nullptr;
  int *par = nullptr;   // device [2 * nbox] parities, table order
  int *hpar = nullptr;  // pinned host copy
  int *status = nullptr;   // device [nbox] status words, box order
  int *hstatus = nullptr;  // pinned host copy
  size_t smem = 0;
  int cpb = 4;
  cudaStream_t s = nullptr;
  std::map<std::pair<int, int>, cudaGraphExec_t> graphs;  // (nsteps, cluster blocks)
};

static bool feasible(Batch *b, int cpb) {
  if (cpb > 8 && cudaFuncSetAttribute(b->kern, cudaFuncAttributeNonPortableClusterSizeAllowed, 1) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(cpb);
  cfg.blockDim = dim3(kBatchThreads);
  cfg.dynamicSmemBytes = b->smem;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeClusterDimension;
  at[0].val.clusterDim.x = cpb;
  at[0].val.clusterDim.y = 1;
  at[0].val.clusterDim.z = 1;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  int n = 0;
  if (cudaOccupancyMaxActiveClusters(&n, b->kern, &cfg) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return n > 0;
}

static cudaError_t launch(Batch *b, int rec0, int nrec, int nsteps, cudaStream_t s) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(nrec * b->cpb);
  cfg.blockDim = dim3(kBatchThreads);
  cfg.dynamicSmemBytes = b->smem;
  cfg.stream = s;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeClusterDimension;
  at[0].val.clusterDim.x = b->cpb;
  at[0].val.clusterDim.y = 1;
  at[0].val.clusterDim.z = 1;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  const void *table = b->table;
  int *par = b->par;
  void *args[] = {(void *)&table, (void *)&par, (void *)&rec0, (void *)&nsteps};
  count_launch();
  return cudaLaunchKernelExC(&cfg, b->kern, args);
}

static void drop_graphs(Batch *b) {
  for (auto &g : b->graphs) cudaGraphExecDestroy(g.second);
  b->graphs.clear();
}

Batch *batch_create(const std::vector<BatchBox> &boxes, cudaStream_t s, int *rc) {
  *rc = LBEH_OK;
  if (boxes.empty()) {
    *rc = LBEH_ERR_INVALID_ARG;
    return nullptr;
  }
  const Ctx &c0 = *boxes[0].c;
  for (const auto &bx : boxes) {
    const Ctx &c = *bx.c;
    if (c.prec != c0.prec || c.ncomp != c0.ncomp || c.nions != c0.nions || c.ncoll_max > 0) {
      *rc = LBEH_ERR_INVALID_ARG;
      return nullptr;
    }
  }
  Batch *b = new Batch;
  b->boxes = boxes;
  b->s = s;
  if (c0.prec == LBEH_FP64) {
    b->K = batch_kernels_f64();
  } else if (c0.prec == LBEH_FP32) {
    b->K = batch_kernels_f32();
  } else {
    delete b;
    *rc = LBEH_ERR_UNSUPPORTED;
    return nullptr;
  }
  b->kern = b->K.kernel(c0.ncomp, c0.nions);
  const int nb = (int)boxes.size();
  bool ok = cudaMalloc(&b->par, sizeof(int) * 2 * nb) == cudaSuccess;
  ok &= cudaMalloc(&b->status, sizeof(int) * nb) == cudaSuccess;
  ok &= cudaMallocHost(&b->hpar, sizeof(int) * 2 * nb) == cudaSuccess;
  ok &= cudaMallocHost(&b->hstatus, sizeof(int) * nb) == cudaSuccess;
  ok &= cudaMalloc(&b->table, b->K.rec_bytes * nb) == cudaSuccess;
  if (!ok) {
    batch_destroy(b);
    *rc = LBEH_ERR_OOM;
    return nullptr;
  }
  cudaMemset(b->status, 0, sizeof(int) * nb);
  std::memset(b->hstatus, 0, sizeof(int) * nb);
  // the boxes' status words move into the batch array (before the records
  // capture the pointers)
  for (int i = 0; i < nb; ++i) b->boxes[i].c->status = b->status + i;
  b->order.resize(nb);
  std::iota(b->order.begin(), b->order.end(), 0);
  std::stable_sort(b->order.begin(), b->order.end(),
                   [&](int x, int y) { return b->boxes[x].c->d.N > b->boxes[y].c->d.N; });
  b->pos.assign(nb, 0);
  for (int t = 0; t < nb; ++t) b->pos[b->order[t]] = t;
  std::vector<unsigned char> host(b->K.rec_bytes * nb);
  long long smem = 0;
  for (int t = 0; t < nb; ++t) {
    const long long sm = b->K.fill(b->boxes[b->order[t]], host.data() + b->K.rec_bytes * t);
    if (sm < 0) {
      batch_destroy(b);
      *rc = LBEH_ERR_UNSUPPORTED;
      return nullptr;
    }
    smem = std::max(smem, sm);
  }
  b->smem = (size_t)smem;
  if (cudaMemcpy(b->table, host.data(), host.size(), cudaMemcpyHostToDevice) != cudaSuccess ||
      !raise_smem_limit(b->kern, b->smem)) {
    batch_destroy(b);
    *rc = LBEH_ERR_CUDA;
    return nullptr;
  }
  // default shape: the smallest portable cluster giving two waves of blocks
  int dev = 0, nsm = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  b->cpb = 0;
  for (int cpb : kShapes) {
    if (cpb > 8 || !feasible(b, cpb)) continue;
    b->cpb = cpb;
    if ((long long)cpb * nb >= 2LL * nsm) break;
  }
  if (b->cpb == 0) {
    batch_destroy(b);
    *rc = LBEH_ERR_UNSUPPORTED;
    return nullptr;
  }
  return b;
}

void batch_destroy(Batch *b) {
  if (!b) return;
  drop_graphs(b);
  if (b->table) cudaFree(b->table);
  if (b->par) cudaFree(b->par);
  if (b->status) cudaFree(b->status);
  if (b->hpar) cudaFreeHost(b->hpar);
  if (b->hstatus) cudaFreeHost(b->hstatus);
  delete b;
}

int batch_shape(const Batch *b) { return b->cpb; }
int batch_box_status(const Batch *b, int box) { return b->hstatus[box]; }

int batch_set_shape(Batch *b, int cpb) {
  bool known = false;
  for (int k : kShapes) known |= k == cpb;
  if (!known || !feasible(b, cpb)) return LBEH_ERR_UNSUPPORTED;
  b->cpb = cpb;
  return LBEH_OK;
}

static void upload_parities(Batch *b) {
  const int nb = (int)b->boxes.size();
  for (int t = 0; t < nb; ++t) {
    const Ctx &c = *b->boxes[b->order[t]].c;
    b->hpar[2 * t] = c.cur;
    b->hpar[2 * t + 1] = c.ncur;
  }
  cudaMemcpyAsync(b->par, b->hpar, sizeof(int) * 2 * nb, cudaMemcpyHostToDevice, b->s);
}

static cudaError_t run(Batch *b, int nsteps, bool sequential) {
  const int nb = (int)b->boxes.size();
  if (sequential) {
    for (int i = 0; i < nb; ++i) {
      const cudaError_t e = launch(b, b->pos[i], 1, nsteps, b->s);
      if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
  }
  const auto key = std::make_pair(nsteps, b->cpb);
  auto it = b->graphs.find(key);
  if (it == b->graphs.end()) {
    cudaStream_t cs = nullptr;
    if (cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking) != cudaSuccess) return cudaErrorUnknown;
    cudaGraph_t g = nullptr;
    cudaError_t e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
    if (e == cudaSuccess) {
      const cudaError_t el = launch(b, 0, nb, nsteps, cs);
      g_launches.fetch_sub(1);  // captured, not launched
      e = cudaStreamEndCapture(cs, &g);
      if (e == cudaSuccess) e = el;
    }
    cudaGraphExec_t ex = nullptr;
    if (e == cudaSuccess) e = cudaGraphInstantiate(&ex, g, 0);
    if (g) cudaGraphDestroy(g);
    cudaStreamDestroy(cs);
    if (e != cudaSuccess) return e;
    it = b->graphs.emplace(key, ex).first;
  }
  count_launch();
  return cudaGraphLaunch(it->second, b->s);
}

int batch_step(Batch *b, int nsteps, bool sequential, int *first_status) {
  *first_status = 0;
  if (nsteps <= 0) return LBEH_OK;
  upload_parities(b);
  if (run(b, nsteps, sequential) != cudaSuccess) return LBEH_ERR_CUDA;
  for (auto &bx : b->boxes) {
    bx.c->cur ^= (nsteps & 1);
    if (bx.c->nions) bx.c->ncur ^= (nsteps & 1);
  }
  const int nb = (int)b->boxes.size();
  cudaMemcpyAsync(b->hstatus, b->status, sizeof(int) * nb, cudaMemcpyDeviceToHost, b->s);
  if (cudaStreamSynchronize(b->s) != cudaSuccess) return LBEH_ERR_CUDA;
  for (int i = 0; i < nb; ++i)
    if (b->hstatus[i] && !*first_status) *first_status = b->hstatus[i];
  return LBEH_OK;
}

// ---------------------------------------------------------------- autotuner
namespace {
struct Snapshot {
  std::vector<std::pair<void *, size_t>> bufs;  // live state
  std::vector<void *> copies;
  std::vector<int> cur, ncur;
};

size_t elem_bytes(const Ctx &c) { return c.prec == LBEH_FP64 ? 8 : 4; }

bool take(Batch *b, Snapshot &sn) {
  for (auto &bx : b->boxes) {
    const Ctx &c = *bx.c;
    const size_t N = (size_t)c.d.N, e = elem_bytes(c);
    sn.bufs.emplace_back(c.f[0], e * 19 * c.ncomp * N);
    sn.bufs.emplace_back(c.f[1], e * 19 * c.ncomp * N);
    if (c.nions) {
      sn.bufs.emplace_back(c.n[0], e * 2 * N);
      sn.bufs.emplace_back(c.n[1], e * 2 * N);
    }
    if (c.prec == LBEH_FP64) {
      sn.bufs.emplace_back(c.phi, 8 * N);
    } else {
      sn.bufs.emplace_back(c.phit, 4 * N);
      sn.bufs.emplace_back(c.phi_lo, 4 * N);
    }
    if (bx.pois) poisson_state_buffers(bx.pois, c, sn.bufs);
    sn.cur.push_back(c.cur);
    sn.ncur.push_back(c.ncur);
  }
  sn.bufs.emplace_back(b->status, sizeof(int) * b->boxes.size());
  for (auto &bf : sn.bufs) {
    void *p = nullptr;
    if (cudaMalloc(&p, bf.second) != cudaSuccess) return false;
    sn.copies.push_back(p);
    cudaMemcpyAsync(p, bf.first, bf.second, cudaMemcpyDeviceToDevice, b->s);
  }
  return true;
}

void restore(Batch *b, const Snapshot &sn) {
  for (size_t k = 0; k < sn.copies.size(); ++k)
    cudaMemcpyAsync(sn.bufs[k].first, sn.copies[k], sn.bufs[k].second, cudaMemcpyDeviceToDevice, b->s);
  for (size_t i = 0; i < b->boxes.size(); ++i) {
    b->boxes[i].c->cur = sn.cur[i];
    b->boxes[i].c->ncur = sn.ncur[i];
  }
}

void release(Snapshot &sn) {
  for (void *p : sn.copies) cudaFree(p);
  sn.copies.clear();
}
}  // namespace

int batch_tune(Batch *b, int probe_steps, int *best_blocks, double *best_ms) {
  if (probe_steps < 1) return LBEH_ERR_INVALID_ARG;
  Snapshot sn;
  if (!take(b, sn)) {
    release(sn);
    cudaGetLastError();
    return LBEH_ERR_OOM;
  }
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  const int keep = b->cpb;
  int best = 0;
  double best_t = 0.0;
  int rc = LBEH_OK;
  for (int cpb : kShapes) {
    if (!feasible(b, cpb)) continue;
    b->cpb = cpb;
    // one warm-up pass, then the timed pass, each from the saved state
    float ms = 0.f;
    for (int pass = 0; pass < 2 && rc == LBEH_OK; ++pass) {
      restore(b, sn);
      upload_parities(b);
      cudaEventRecord(e0, b->s);
      if (launch(b, 0, (int)b->boxes.size(), probe_steps, b->s) != cudaSuccess) rc = LBEH_ERR_CUDA;
      cudaEventRecord(e1, b->s);
      if (cudaEventSynchronize(e1) != cudaSuccess) rc = LBEH_ERR_CUDA;
      cudaEventElapsedTime(&ms, e0, e1);
    }
    if (rc != LBEH_OK) break;
    const double t = double(ms) / probe_steps;
    if (best == 0 || t < best_t) {
      best = cpb;
      best_t = t;
    }
  }
  restore(b, sn);
  cudaStreamSynchronize(b->s);
  release(sn);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  b->cpb = best ? best : keep;
  if (best_blocks) *best_blocks = b->cpb;
  if (best_ms) *best_ms = best_t;
  return rc;
}

}  // namespace lbeh
