// Small kernels: deterministic FP64 reductions, the power-method helpers,
// a counter-based start vector, and the plane permutation between the natural
// and the class-permuted layouts of U.
#include "device.cuh"
#include "internal.h"

namespace muffin {

// One block sums (op 0) or maxes (op 1) n partials in a fixed order.
__global__ void __launch_bounds__(1024) k_reduce_partials(const double* __restrict__ p, int n, double* out, int op) {
  __shared__ double red[32];
  double acc = 0.0;
  for (int i = threadIdx.x; i < n; i += blockDim.x) acc = op == 0 ? acc + p[i] : fmax(acc, p[i]);
  if (op == 0) {
    acc = block_sum(acc, red);
  } else {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) acc = fmax(acc, __shfl_down_sync(0xffffffffu, acc, o));
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x < 32) {
      acc = threadIdx.x < (blockDim.x + 31) / 32 ? red[threadIdx.x] : 0.0;
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) acc = fmax(acc, __shfl_down_sync(0xffffffffu, acc, o));
    }
  }
  if (threadIdx.x == 0) *out = acc;
}

__global__ void __launch_bounds__(256) k_dot(const float* __restrict__ a, const float* __restrict__ b, size_t n,
                                            double* partials) {
  __shared__ double red[32];
  double acc = 0.0;
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
    acc += (double)a[i] * (double)b[i];
  acc = block_sum(acc, red);
  if (threadIdx.x == 0) partials[blockIdx.x] = acc;
}

// x <- x * num / sqrt(den)   (num == nullptr: factor 1)
__global__ void k_scale(float* x, size_t n, const double* num, const double* den) {
  const double f = (num ? *num : 1.0) / sqrt(*den);
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
    x[i] = (float)(x[i] * f);
}

// SplitMix64 (Steele, Lea and Flood, OOPSLA 2014) of (seed + index): uniform in [-1, 1).
__device__ __forceinline__ uint64_t splitmix64(uint64_t z) {
  z += 0x9e3779b97f4a7c15ull;
  z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ull;
  z = (z ^ (z >> 27)) * 0x94d049bb133111ebull;
  return z ^ (z >> 31);
}

__global__ void k_fill_random(float* x, size_t n, uint64_t seed) {
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
    const uint64_t r = splitmix64(seed * 0x100000001b3ull + i);
    x[i] = (float)((double)(r >> 11) * (2.0 / 9007199254740992.0) - 1.0);
  }
}

// Planes j >= j1 of U between natural (to_class = 0) and class-permuted layout.
__global__ void k_permute(const float* __restrict__ src, float* __restrict__ dst, int n, int L, int J, int j1,
                          int to_class) {
  const size_t P = (size_t)n * n;
  const size_t total = (size_t)L * (J + 1) * P;
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < total; i += (size_t)gridDim.x * blockDim.x) {
    const size_t plane = i / P;
    const int j = (int)(plane % (J + 1));
    const int p = (int)(i % P);
    const int lgs = j >= j1 ? j1 : 0;
    const int ci = class_index(p / n, p % n, n, lgs);
    if (to_class) dst[plane * P + ci] = src[i];
    else dst[i] = src[plane * P + ci];
  }
}

__global__ void k_nonfinite(const float* __restrict__ x, size_t n, int* count) {
  int c = 0;
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
    c += isfinite(x[i]) ? 0 : 1;
  c = warp_sum(c);
  if ((threadIdx.x & 31) == 0 && c) atomicAdd(count, c);
}

static int grid_for(size_t n, int block, int cap) {
  size_t g = (n + block - 1) / block;
  if (g > (size_t)cap) g = cap;
  return g < 1 ? 1 : (int)g;
}

cudaError_t launch_sum_partials(const double* partials, int n, double* out, cudaStream_t s) {
  k_reduce_partials<<<1, 1024, 0, s>>>(partials, n, out, 0);
  return cudaGetLastError();
}

cudaError_t launch_max_partials(const double* partials, int n, double* out, cudaStream_t s) {
  k_reduce_partials<<<1, 1024, 0, s>>>(partials, n, out, 1);
  return cudaGetLastError();
}

cudaError_t launch_dot(const float* a, const float* b, size_t n, double* partials, int* nparts, cudaStream_t s) {
  const int g = grid_for(n, 256, 1024);
  *nparts = g;
  k_dot<<<g, 256, 0, s>>>(a, b, n, partials);
  return cudaGetLastError();
}

cudaError_t launch_scale(float* x, size_t n, const double* num, const double* den, cudaStream_t s) {
  k_scale<<<grid_for(n, 256, 4096), 256, 0, s>>>(x, n, num, den);
  return cudaGetLastError();
}

cudaError_t launch_fill_random(float* x, size_t n, uint64_t seed, cudaStream_t s) {
  k_fill_random<<<grid_for(n, 256, 4096), 256, 0, s>>>(x, n, seed);
  return cudaGetLastError();
}

cudaError_t launch_permute_planes(const float* src, float* dst, int n, int L, int J, int j1, int to_class,
                                  cudaStream_t s) {
  const size_t total = (size_t)L * (J + 1) * n * n;
  k_permute<<<grid_for(total, 256, 8192), 256, 0, s>>>(src, dst, n, L, J, j1, to_class);
  return cudaGetLastError();
}

cudaError_t launch_nonfinite_count(const float* x, size_t n, int* count, cudaStream_t s) {
  k_nonfinite<<<grid_for(n, 256, 4096), 256, 0, s>>>(x, n, count);
  return cudaGetLastError();
}

}  // namespace muffin
