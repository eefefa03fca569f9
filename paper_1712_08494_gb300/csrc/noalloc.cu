// Allocation-free variant of the observables reduction (lbeh_observables).
//
// Some callers cannot allocate device memory at the point where they want
// the conserved sums: code under a memory pool budget that forbids
// cudaMalloc, plugins that only receive borrowed device buffers, or processes
// whose allocator is owned by another runtime.  This entry point takes the
// caller's device fields and a host output struct and allocates nothing: its
// only scratch (per-block partial sums) lives in the file-scope array below,
// which every GPU that loads the library holds until the process exits
// (LBEH_NOALLOC_SCRATCH_BYTES, 128 KiB + 128 B).  It ends with a
// device-to-host copy of the sums and a synchronisation of the caller's
// stream.
//
// Host code must not pass the array's name to a kernel: on the host it is a
// stand-in symbol, not a device address.  The first call in each CUDA context
// (the primary context of a device, or a context the caller created and made
// current) looks the address up with cudaGetSymbolAddress, with that context
// current, and caches it per context: each context loads its own copy of the
// module, so an address found in one context is not valid in another.  That
// first call may initialise the CUDA context.
//
// All calls share the array.  Every call overwrites all partials it later
// reads, so nothing has to start at zero, but two calls whose kernels overlap
// on the GPU (different streams, no ordering) race on it.
#include <cmath>
#include <cstring>
#include <mutex>
#include <vector>

#include <cuda.h>

#include "internal.h"
#include "dfloat.cuh"

namespace lbeh {
namespace {

constexpr int kNABlock = 256;
constexpr int kNAPerThread = 64;
constexpr long long kNAChunk = (long long)kNABlock * kNAPerThread;  // sites per block
constexpr int kNAMaxBlocks = 1024;
constexpr int kNALen = kObsLen;

static __device__ __align__(256) double g_obs_scratch[kNAMaxBlocks * kNALen + kNALen];

std::mutex g_mtx;
std::vector<std::pair<CUcontext, double *>> g_addr;  // CUDA context -> scratch address in it

// cuCtxGetCurrent through the runtime's driver entry point table (no link
// against the driver library)
using CtxGetCurrentFn = CUresult (*)(CUcontext *);
CtxGetCurrentFn ctx_get_current() {
  static CtxGetCurrentFn fn = [] {
    void *f = nullptr;
    cudaDriverEntryPointQueryResult q{};
    if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &f, 12000, cudaEnableDefault, &q) != cudaSuccess ||
        q != cudaDriverEntryPointSuccess)
      f = nullptr;
    return (CtxGetCurrentFn)f;
  }();
  return fn;
}

int scratch_address(double **out) {
  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess) return LBEH_ERR_CUDA;
  CtxGetCurrentFn get = ctx_get_current();
  if (!get) return LBEH_ERR_CUDA;
  CUcontext ctx = nullptr;
  if (get(&ctx) != CUDA_SUCCESS) return LBEH_ERR_CUDA;
  std::lock_guard<std::mutex> lock(g_mtx);
  if (ctx)
    for (auto &e : g_addr)
      if (e.first == ctx) {
        *out = e.second;
        return LBEH_OK;
      }
  // the lookup runs in the current context; with none current the runtime
  // initialises the device's primary context and makes it current first
  double *p = nullptr;
  if (cudaGetSymbolAddress((void **)&p, g_obs_scratch) != cudaSuccess || !p) return LBEH_ERR_CUDA;
  if (!ctx && (get(&ctx) != CUDA_SUCCESS || !ctx)) return LBEH_ERR_CUDA;
  g_addr.emplace_back(ctx, p);
  *out = p;
  return LBEH_OK;
}

// Block b sums the contiguous chunk [b*kNAChunk, (b+1)*kNAChunk) in a fixed
// order (thread-strided, then a shared-memory tree); layout of the 16 sums as
// in the handle's observables: mass[2], ions[2], charge, momentum[3], W,
// W x, W y, W z, W x^2, W z^2, unused[2].
template <typename F>
__global__ void __launch_bounds__(kNABlock)
    k_obs_na(Dims d, int ncomp, int nions, const F *__restrict__ f, const F *__restrict__ n,
             const uint8_t *__restrict__ solid, const double *__restrict__ qc, double *__restrict__ scratch) {
  const long long N = d.N;
  SumAcc<std::is_same<F, float>::value> acc[kNALen];
  const long long base = blockIdx.x * kNAChunk;
  for (int k = 0; k < kNAPerThread; ++k) {
    const long long i = base + (long long)k * kNABlock + threadIdx.x;
    if (i >= N) break;
    if (nions) {
      const F np = n[i], nm = n[N + i];
      acc[2].add(np);
      acc[3].add(nm);
      acc[4].add(np);
      acc[4].add(-nm);
    }
    if (qc) acc[4].add(F(qc[i]));
    if (solid && solid[i]) continue;
    // per-site arithmetic of the handle's observables: sums in the input's own
    // precision, running sums in double-float words (FP32) or FP64
    F rt[2] = {F(0), F(0)}, Jt[3] = {F(0), F(0), F(0)};
    for (int s = 0; s < ncomp; ++s)
#pragma unroll
      for (int q = 0; q < 19; ++q) {
        const F v = f[(size_t)(s * 19 + q) * N + i];
        rt[s] += v;
        if (cx(q)) Jt[0] += F(cx(q)) * v;
        if (cy(q)) Jt[1] += F(cy(q)) * v;
        if (cz(q)) Jt[2] += F(cz(q)) * v;
      }
    acc[0].add(rt[0]);
    acc[1].add(rt[1]);
    acc[5].add(Jt[0]);
    acc[6].add(Jt[1]);
    acc[7].add(Jt[2]);
    if (ncomp == 2) {
      const F tot = rt[0] + rt[1];
      const F c = tot > F(0) ? (rt[1] - rt[0]) / tot : F(0);
      if (c > F(0)) {
        int x, y, z;
        coords(d, i, x, y, z);
        acc[8].add(c);
        acc_prod(acc[9], c, F(x));
        acc_prod(acc[10], c, F(y));
        acc_prod(acc[11], c, F(z));
        acc_prod2(acc[12], c, F(x));
        acc_prod2(acc[13], c, F(z));
      }
    }
  }
  __shared__ double sh[kNALen][kNABlock];
#pragma unroll
  for (int t = 0; t < kNALen; ++t) sh[t][threadIdx.x] = acc[t].get();
  __syncthreads();
  for (int w = kNABlock / 2; w > 0; w >>= 1) {
    if (threadIdx.x < w)
#pragma unroll
      for (int t = 0; t < kNALen; ++t) sh[t][threadIdx.x] += sh[t][threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x < kNALen) scratch[blockIdx.x * kNALen + threadIdx.x] = sh[threadIdx.x][0];
}

__global__ void __launch_bounds__(kNABlock) k_obs_na_final(double *__restrict__ scratch, int nblocks) {
  __shared__ double sh[kNABlock];
  double *out = scratch + (size_t)kNAMaxBlocks * kNALen;
  for (int t = 0; t < kNALen; ++t) {
    double acc = 0.0;
    for (int b = threadIdx.x; b < nblocks; b += kNABlock) acc += scratch[(size_t)b * kNALen + t];
    sh[threadIdx.x] = acc;
    __syncthreads();
    for (int w = kNABlock / 2; w > 0; w >>= 1) {
      if (threadIdx.x < w) sh[threadIdx.x] += sh[threadIdx.x + w];
      __syncthreads();
    }
    if (threadIdx.x == 0) out[t] = sh[0];
    __syncthreads();
  }
}

}  // namespace
}  // namespace lbeh

using namespace lbeh;

extern "C" int lbeh_observables_noalloc(int nx, int ny, int nz, int ncomp, int nions, int dtype, const void *f,
                                        const void *n, const uint8_t *solid, const double *qc, lbeh_obs *out,
                                        void *stream) {
  if (!out || !f || nx < 1 || ny < 1 || nz < 1) return LBEH_ERR_INVALID_ARG;
  if ((ncomp != 1 && ncomp != 2) || (nions != 0 && nions != 2) || (nions && !n)) return LBEH_ERR_INVALID_ARG;
  if (dtype != LBEH_F64 && dtype != LBEH_F32) return LBEH_ERR_INVALID_ARG;
  const long long N = (long long)nx * ny * nz;
  if (N > LBEH_NOALLOC_MAX_SITES) return LBEH_ERR_INVALID_ARG;  // beyond the static scratch
  double *scratch = nullptr;
  int rc = scratch_address(&scratch);
  if (rc != LBEH_OK) return rc;
  cudaStream_t s = (cudaStream_t)stream;
  const Dims d{nx, ny, nz, N};
  const int nb = int((N + kNAChunk - 1) / kNAChunk);
  if (dtype == LBEH_F64)
    count_launch(), k_obs_na<double><<<nb, kNABlock, 0, s>>>(d, ncomp, nions, (const double *)f,
                                                             (const double *)n, solid, qc, scratch);
  else
    count_launch(), k_obs_na<float><<<nb, kNABlock, 0, s>>>(d, ncomp, nions, (const float *)f, (const float *)n,
                                                            solid, qc, scratch);
  count_launch(), k_obs_na_final<<<1, kNABlock, 0, s>>>(scratch, nb);
  double v[kNALen];
  if (cudaMemcpyAsync(v, scratch + (size_t)kNAMaxBlocks * kNALen, sizeof(v), cudaMemcpyDeviceToHost, s) !=
      cudaSuccess)
    return LBEH_ERR_CUDA;
  if (cudaStreamSynchronize(s) != cudaSuccess) return LBEH_ERR_CUDA;
  std::memset(out, 0, sizeof(*out));
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
  out->status = LBEH_OK;
  return LBEH_OK;
}
