// Deterministic FP64 reductions: a fixed grid of kRedBlocks blocks, each
// summing a block-strided subset in a fixed order and a shared-memory tree,
// then one block summing the partials in a fixed tree.  Results are bitwise
// reproducible for a given problem size.
#include "internal.h"

namespace lbeh {

template <int B>
__device__ __forceinline__ double block_sum(double v, double *sh) {
  sh[threadIdx.x] = v;
  __syncthreads();
  for (int w = B / 2; w > 0; w >>= 1) {
    if (threadIdx.x < w) sh[threadIdx.x] += sh[threadIdx.x + w];
    __syncthreads();
  }
  double r = sh[0];
  __syncthreads();
  return r;
}

__global__ void __launch_bounds__(256) k_dot_partial(const double *__restrict__ a, const double *__restrict__ b,
                                                     long long n, double *__restrict__ part) {
  __shared__ double sh[256];
  double acc = 0.0;
  for (long long i = blockIdx.x * 256LL + threadIdx.x; i < n; i += (long long)gridDim.x * 256)
    acc += b ? a[i] * b[i] : a[i];
  double r = block_sum<256>(acc, sh);
  if (threadIdx.x == 0) part[blockIdx.x] = r;
}

// Up to kFinalLen values reduced together: every thread adds its strided
// partials of all values (loads in flight together), then one shared-memory
// tree over all values; longer lists one value at a time.  The order of the
// additions per value is the same either way (fixed, deterministic).
constexpr int kFinalLen = 16;
__global__ void __launch_bounds__(256) k_final(const double *__restrict__ part, int nblocks, int len,
                                               double *__restrict__ out) {
  if (len <= kFinalLen) {
    __shared__ double shv[kFinalLen][256];
    double acc[kFinalLen];
#pragma unroll
    for (int t = 0; t < kFinalLen; ++t) acc[t] = 0.0;
    for (int b = threadIdx.x; b < nblocks; b += 256)
#pragma unroll
      for (int t = 0; t < kFinalLen; ++t)
        if (t < len) acc[t] += part[(long long)b * len + t];
#pragma unroll
    for (int t = 0; t < kFinalLen; ++t) shv[t][threadIdx.x] = acc[t];
    __syncthreads();
    for (int w = 128; w > 0; w >>= 1) {
      if (threadIdx.x < w)
#pragma unroll
        for (int t = 0; t < kFinalLen; ++t) shv[t][threadIdx.x] += shv[t][threadIdx.x + w];
      __syncthreads();
    }
    if (threadIdx.x < len) out[threadIdx.x] = shv[threadIdx.x][0];
    return;
  }
  __shared__ double sh[256];
  for (int t = 0; t < len; ++t) {
    double acc = 0.0;
    for (int b = threadIdx.x; b < nblocks; b += 256) acc += part[(long long)b * len + t];
    double r = block_sum<256>(acc, sh);
    if (threadIdx.x == 0) out[t] = r;
  }
}

void reduce_partials_final(const double *partials, int nblocks, int len, double *out, cudaStream_t s) {
  count_launch(), k_final<<<1, 256, 0, s>>>(partials, nblocks, len, out);
}

static double reduce_to_host(const double *a, const double *b, long long n, double *scratch, cudaStream_t s) {
  count_launch(), k_dot_partial<<<kRedBlocks, 256, 0, s>>>(a, b, n, scratch);
  count_launch(), k_final<<<1, 256, 0, s>>>(scratch, kRedBlocks, 1, scratch + kRedBlocks);
  double h = 0.0;
  cudaMemcpyAsync(&h, scratch + kRedBlocks, sizeof(double), cudaMemcpyDeviceToHost, s);
  cudaStreamSynchronize(s);
  return h;
}

double dot_f64(const double *a, const double *b, long long n, double *scratch, cudaStream_t s) {
  return reduce_to_host(a, b, n, scratch, s);
}

double sum_f64(const double *a, long long n, double *scratch, cudaStream_t s) {
  return reduce_to_host(a, nullptr, n, scratch, s);
}

}  // namespace lbeh
