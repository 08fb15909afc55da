// Persistent batch pass: one cooperative launch runs one pass of Algorithm 1
// (Eqs. 8-14) over every cube of a batch of uneven cubes.  The pass's stages
// run in order, each as a work list over (cube, channel, tile) items that
// the resident blocks take in turn, with a grid barrier between stages:
//   0 row FFTs (Eq. 8)            3 spatial analysis + dual update (Eq. 11)
//   1 column filter (Eq. 8)       4 coarse levels on class sub-images
//   2 inverse rows + primal step  5 spatial adjoint (Eq. 9) and the spectral
//     (Eq. 10)                      step (Eqs. 13-14), independent, together
// The block bodies are those of the one-stage kernels (fft_blocks.cuh,
// iuwt_vec.cuh, spectral_blocks.cuh) at 512 threads.  Every barrier wait is
// bounded: a block that gives up sets the error word, the others see it at
// their next barrier (or give up in turn), and every block then skips the
// remaining stages, so the launch always ends.
#include "device.cuh"
#include "fft_blocks.cuh"
#include "internal.h"
#include "iuwt_vec.cuh"
#include "spectral_blocks.cuh"

namespace muffin {

constexpr int kBNT = kBatchThreads;
template <int N> __host__ __device__ constexpr int batch_pairs() { return 4096 / N; }   // rows: pairs x N/8 = 512
template <int N> __host__ __device__ constexpr int batch_cols() { return 4096 / N; }    // cols: C x N/8 = 512

__host__ __device__ inline int ilog2(int v) { int r = 0; while ((1 << r) < v) ++r; return r; }
__host__ __device__ inline bool spec_pow2(int L) { return L >= 16 && L <= 256 && (L & (L - 1)) == 0; }

// items of stage s (5: adjoint; 6: spectral) for cube c
__host__ __device__ inline int stage_items(const BatchCube& c, int s) {
  const int n = c.n, L = c.L;
  switch (s) {
    case 0: case 1: case 2: return L * (n * n / 8192);
    case 3: case 5: return (c.spatial && c.j1 > 0) ? L * (n / 64) * (n / 64) : 0;
    case 4: return (c.spatial && c.J > c.j1) ? L * (1 << (2 * c.j1)) : 0;
    case 6: {
      if (!c.spectral) return 0;
      const int tiles = n * n / 32;
      if (!spec_pow2(L)) return tiles;
      const int G = kBNT / (2 * L);
      return (tiles + G - 1) / G;
    }
  }
  return 0;
}

// Grid barrier with a bounded wait (see the file comment); false once any block gave up.
__device__ __forceinline__ bool grid_barrier(const BatchArgs& a) {
  __syncthreads();
  if (threadIdx.x == 0 && *(volatile int*)a.err == 0) {
    volatile unsigned* vb = a.bar;
    const unsigned gen = vb[1];
    __threadfence();
    const unsigned arrived = atomicAdd(a.bar, 1u) + 1u;
    if (arrived == gridDim.x) {
      vb[0] = 0u;
      __threadfence();
      atomicAdd(a.bar + 1, 1u);
    } else {
      long long i = 0;
      while (vb[1] == gen && i < a.polls) {
        __nanosleep(128);
        ++i;
      }
      if (vb[1] == gen) atomicExch(a.err, 1);
    }
    __threadfence();
  }
  __syncthreads();
  return *(volatile int*)a.err == 0;
}

template <int N>
__device__ __noinline__ void rows_item(const BatchCube& c, int item, int inverse, unsigned char* sm) {
  constexpr int PAIRS = batch_pairs<N>(), PER = N * N / 8192;
  cpx<float>* tw = reinterpret_cast<cpx<float>*>(sm);
  cpx<float>* buf = tw + N;
  const cpx<float>* twg = reinterpret_cast<const cpx<float>*>(c.twf);
  for (int i = threadIdx.x; i < N; i += kBNT) tw[i] = twg[i];
  __syncthreads();
  const int l = item / PER, bx = item % PER;
  if (inverse)
    rows_inv_block<N, PAIRS, 0>(reinterpret_cast<const cpx<float>*>(c.spec), c.pa, nullptr, tw, buf, l, bx);
  else
    rows_fwd_block<N, PAIRS>(c.pa.X, reinterpret_cast<cpx<float>*>(c.spec), tw, buf, l, bx);
}

template <int N>
__device__ __noinline__ void cols_item(const BatchCube& c, int item, unsigned char* sm) {
  constexpr int C = batch_cols<N>(), PER = (N / 2) / C;
  cpx<float>* tw = reinterpret_cast<cpx<float>*>(sm);
  cpx<float>* buf = tw + N;
  const cpx<float>* twg = reinterpret_cast<const cpx<float>*>(c.twf);
  for (int i = threadIdx.x; i < N; i += kBNT) tw[i] = twg[i];
  __syncthreads();
  cols_block<N, C>(reinterpret_cast<cpx<float>*>(c.spec), c.Kp, c.Kb, tw, buf, item / PER, item % PER);
}

#define BATCH_N(n, CALL) \
  switch (n) {           \
    case 128: CALL(128); break; \
    case 256: CALL(256); break; \
    case 512: CALL(512); break; \
    case 1024: CALL(1024); break; \
  }

template <int J1>
__device__ __noinline__ void fine_an_item(const BatchCube& c, int l, int ty0, int tx0, float* sm) {
  const IuwtArgs& a = c.ia;
  vec::fine_analysis_tile<kBNT, J1>(sm, c.n, c.J, a.D, a.U, a.cr, a.k, a.rho, l, ty0, tx0);
}

template <int J1>
__device__ __noinline__ void fine_adj_item(const BatchCube& c, int l, int ty0, int tx0, float* sm) {
  const IuwtArgs& a = c.ia;
  const size_t P = (size_t)c.n * c.n;
  const bool from_u = c.J == c.j1;
  const float* rin = from_u ? a.U + (size_t)c.J * P : a.rin;
  const size_t stride = from_u ? (size_t)(c.J + 1) * P : P;
  vec::fine_adjoint_tile<kBNT, J1>(sm, c.n, c.J, rin, stride, a.U, a.S, l, ty0, tx0);
}

__device__ __forceinline__ void fine_item(const BatchCube& c, int item, int adjoint, unsigned char* smc) {
  float* sm = reinterpret_cast<float*>(smc);
  const int n = c.n, tpd = n / 64, per = tpd * tpd;
  const int l = item / per, t = item % per, ty0 = (t / tpd) * 64, tx0 = (t % tpd) * 64;
  switch (c.j1 * 2 + adjoint) {
    case 2: fine_an_item<1>(c, l, ty0, tx0, sm); break;
    case 3: fine_adj_item<1>(c, l, ty0, tx0, sm); break;
    case 4: fine_an_item<2>(c, l, ty0, tx0, sm); break;
    case 5: fine_adj_item<2>(c, l, ty0, tx0, sm); break;
    case 6: fine_an_item<3>(c, l, ty0, tx0, sm); break;
    case 7: fine_adj_item<3>(c, l, ty0, tx0, sm); break;
  }
}

template <int M, int NL>
__device__ __noinline__ void coarse_item_t(const BatchCube& c, int cls, int l, float* sm) {
  const IuwtArgs& a = c.ia;
  if constexpr (M == 128)
    vec::coarse_sub_s<kBNT, 128, NL>(sm, c.n, c.J, c.j1, a.cr, a.cr, a.U, a.k, a.rho, cls, l);
  else
    vec::coarse_sub<kBNT, M, NL>(sm, c.n, c.J, c.j1, a.cr, a.cr, a.U, a.k, a.rho, cls, l);
}

__device__ __forceinline__ void coarse_item(const BatchCube& c, int item, unsigned char* smc) {
  float* sm = reinterpret_cast<float*>(smc);
  const int per = 1 << (2 * c.j1), l = item / per, cls = item % per;
  const int M = c.n >> c.j1, NL = c.J - c.j1;
#define CO(MM, LL) \
  if (M == MM && NL == LL) { coarse_item_t<MM, LL>(c, cls, l, sm); return; }
  CO(32, 1) CO(32, 2) CO(32, 3) CO(64, 1) CO(64, 2) CO(64, 3) CO(128, 1) CO(128, 2) CO(128, 3)
#undef CO
}

template <int L>
__device__ __noinline__ void spectral_item_t(const BatchCube& c, int item, unsigned char* sm) {
  const int npix = c.n * c.n;
  spectral_update_block<L, kBNT>(c.sa, npix, item * (kBNT / (2 * L)), npix / 32, sm);
}

__device__ __noinline__ void spectral_item_dense(const BatchCube& c, int item, unsigned char* sm) {
  spectral_dense_block<kBNT>(c.sa, c.n * c.n, c.L, item, reinterpret_cast<float*>(sm));
}

__device__ __forceinline__ void spectral_item(const BatchCube& c, int item, unsigned char* sm) {
  switch (c.L) {
    case 16: spectral_item_t<16>(c, item, sm); return;
    case 32: spectral_item_t<32>(c, item, sm); return;
    case 64: spectral_item_t<64>(c, item, sm); return;
    case 128: spectral_item_t<128>(c, item, sm); return;
    case 256: spectral_item_t<256>(c, item, sm); return;
  }
  spectral_item_dense(c, item, sm);
}

// (the item bodies are separate functions so that each gets the registers of
// its own path)
// Run item w of stage s (s = 5 lists the adjoint items of every cube, then the spectral items).
__device__ __forceinline__ void run_item(const BatchArgs& a, int s, int w, unsigned char* sm) {
  for (int pass = 0; pass < (s == 5 ? 2 : 1); ++pass) {
    const int st = (s == 5 && pass == 1) ? 6 : s;
    for (int i = 0; i < a.nc; ++i) {
      const BatchCube& c = a.c[i];
      const int k = stage_items(c, st);
      if (w < k) {
        switch (st) {
#define RF(NN) rows_item<NN>(c, w, 0, sm)
#define RI(NN) rows_item<NN>(c, w, 1, sm)
#define CL(NN) cols_item<NN>(c, w, sm)
          case 0: BATCH_N(c.n, RF) break;
          case 1: BATCH_N(c.n, CL) break;
          case 2: BATCH_N(c.n, RI) break;
#undef RF
#undef RI
#undef CL
          case 3: fine_item(c, w, 0, sm); break;
          case 4: coarse_item(c, w, sm); break;
          case 5: fine_item(c, w, 1, sm); break;
          case 6: spectral_item(c, w, sm); break;
        }
        return;
      }
      w -= k;
    }
  }
}

__global__ void __launch_bounds__(kBNT, 1) k_batch_pass(const __grid_constant__ BatchArgs a) {
  extern __shared__ __align__(16) unsigned char smb[];
  for (int s = 0; s < 6; ++s) {
    int total = 0;
    for (int i = 0; i < a.nc; ++i) total += stage_items(a.c[i], s) + (s == 5 ? stage_items(a.c[i], 6) : 0);
    for (int w = blockIdx.x; w < total; w += gridDim.x) {
      run_item(a, s, w, smb);
      __syncthreads();          // the next item reuses the shared memory
    }
    if (s < 5 && !grid_barrier(a)) return;
  }
}

// ------------------------------------------------------------------ host side
bool batch_cube_ok(const Geom& g, int spatial, int spectral) {
  if (g.gen != 1 || g.dict != 0) return false;
  if (g.n != 128 && g.n != 256 && g.n != 512 && g.n != 1024) return false;
  if (spatial && g.J > 0) {
    if (g.j1 < 1 || g.j1 > 3) return false;
    const int M = g.n >> g.j1, NL = g.J - g.j1;
    if (NL > 0 && !((M == 32 || M == 64 || M == 128) && NL <= 3)) return false;
  } else if (spatial) {
    return false;          // J = 0 (W_s = I) has no path here
  }
  if (spectral && !spec_pow2(g.L) && g.L > 256) return false;
  return true;
}

static size_t fine_an_smem(int j1) {
  switch (j1) {
    case 1: return vec::FineA<1>::SMEM;
    case 2: return vec::FineA<2>::SMEM;
    case 3: return vec::FineA<3>::SMEM;
  }
  return 0;
}
static size_t fine_adj_smem(int j1) {
  switch (j1) {
    case 1: return vec::FineT<1>::SMEM;
    case 2: return vec::FineT<2>::SMEM;
    case 3: return vec::FineT<3>::SMEM;
  }
  return 0;
}
static size_t coarse_smem(int M, int NL) {
  if (M == 128) return NL == 1 ? vec::CoarseS<128, 1>::SMEM : NL == 2 ? vec::CoarseS<128, 2>::SMEM : vec::CoarseS<128, 3>::SMEM;
  if (M == 64) return NL == 1 ? vec::CoarseV<64, 1>::SMEM : NL == 2 ? vec::CoarseV<64, 2>::SMEM : vec::CoarseV<64, 3>::SMEM;
  return NL == 1 ? vec::CoarseV<32, 1>::SMEM : NL == 2 ? vec::CoarseV<32, 2>::SMEM : vec::CoarseV<32, 3>::SMEM;
}
static size_t spec_smem(int L) {
  switch (L) {
    case 16: return SpecBlock<16, kBNT>::SMEM;
    case 32: return SpecBlock<32, kBNT>::SMEM;
    case 64: return SpecBlock<64, kBNT>::SMEM;
    case 128: return SpecBlock<128, kBNT>::SMEM;
    case 256: return SpecBlock<256, kBNT>::SMEM;
  }
  return (size_t)2 * L * 32 * sizeof(float);
}

size_t batch_smem_bytes(const BatchArgs& a) {
  size_t m = 0;
  auto up = [&](size_t v) { if (v > m) m = v; };
  for (int i = 0; i < a.nc; ++i) {
    const BatchCube& c = a.c[i];
    const size_t n = c.n;
    up(n * 8 + (size_t)(4096 / n) * (n + n / 8) * 8);     // rows: twiddles + padded row pairs
    up(n * 8 + n * (4096 / n) * 8);                        // cols: twiddles + C columns
    if (c.spatial && c.j1 > 0) {
      up(fine_an_smem(c.j1));
      up(fine_adj_smem(c.j1));
    }
    if (c.spatial && c.J > c.j1) up(coarse_smem(c.n >> c.j1, c.J - c.j1));
    if (c.spectral) up(spec_smem(c.L));
  }
  return m;
}

cudaError_t batch_configure() { return allow_max_dyn_smem(k_batch_pass); }

int batch_grid(size_t smem) {
  int dev = 0, sms = 0, occ = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return 0;
  if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_batch_pass, kBNT, smem) != cudaSuccess) {
    cudaGetLastError();
    return 0;
  }
  return occ * sms;
}

cudaError_t launch_batch_pass(const BatchArgs& a, size_t smem, int grid, cudaStream_t s) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(grid);
  cfg.blockDim = dim3(kBNT);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeCooperative;   // every block resident at once: the barriers can complete
  attr[0].val.cooperative = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, k_batch_pass, a);
}

}  // namespace muffin
