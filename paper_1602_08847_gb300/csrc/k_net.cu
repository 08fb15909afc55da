// Warm-start network: six zero-padded 3x3x3 convolution layers over the
// cube (1 -> 32 -> 32 -> 32 -> 32 -> 32 -> K feature maps, K <= 8), its
// loss, its gradients and Adam, all in bfloat16 with float32 accumulation.
// Output map 0 predicts the cube X of Algorithm 1, maps 1 .. K-1 further
// fields of its state (the planes of the wavelet dual U).
//
// Feature maps are [nz][ny][nx][32] bfloat16 (64 bytes per voxel).  The
// tensor-core kernels (below) walk tiles of 1 x 16 x 8 voxels whose halos
// arrive by TMA.  The CUDA-core kernels work on output tiles of 2 x 8 x 16
// voxels (channel, row, column) whose inputs, with a one-voxel halo
// (4 x 10 x 18), are staged in shared memory by cp.async with zero fill
// outside the cube (the zero padding of the layers); there a voxel's 64 bytes
// are four 16-byte chunks, chunk c of row r stored at chunk c ^ ((r >> 1) & 3),
// so that eight consecutive rows read at the same chunk hit eight different
// bank groups.
//
// The 32 -> 32 layers are implicit GEMMs on the tensor cores, bfloat16 in,
// float32 accumulate:
//   forward      z[p][co]  = sum_tap sum_ci a[p + d(tap)][ci] W[tap][co][ci]
//                 (M = voxels, N = co, K = 27 taps x 32 ci), tcgen05.mma with the
//                 accumulator in tensor memory,
//   input grad   da[p][ci] = sum_tap sum_co dz[p - d(tap)][co] W[tap][co][ci],
//                 the same kernel on the flipped, transposed weights,
//   weight grad  dW[tap][co][ci] = sum_p dz[p][co] a[p + d(tap)][ci]
//                 (M = (row offset, ci), N = co, K = voxels), tcgen05.mma with nine
//                 accumulators resident in tensor memory for the CTA's whole run.
// The last layer's forward (prediction, or the loss and its gradient d6) is
// the same tcgen05 kernel with N = 16 (weights of maps K .. 15 zero).  The
// 1 -> 32 layer and the last layer's gradients (27 or 864 multiply-adds per
// voxel and output, with float32 d6) run on the CUDA cores.  Every reduction
// over voxels is a per-block partial sum followed by a fixed-order sum:
// results do not depend on scheduling.
#include <cuda.h>            // CUtensorMap (the encoder is reached through the runtime's driver entry point)
#include <cuda_runtime.h>
#include <cuda_bf16.h>
#include <stdint.h>

#include <cmath>
#include <cstdio>
#include <cstring>
#include <string>

#include "device.cuh"
#include "muffin.h"
#include "muffin_net.h"

namespace mnet {

using bf16 = __nv_bfloat16;
using bf162 = __nv_bfloat162;

constexpr int C = 32;                        // features of the hidden layers
constexpr int NTAP = 27;
constexpr int TZ = 2, TY = 8, TX = 16;       // output tile (channel, row, column)
constexpr int TV = TZ * TY * TX;             // 256 voxels
constexpr int HZ = TZ + 2, HY = TY + 2, HX = TX + 2;
constexpr int HV = HZ * HY * HX;             // 720 voxels with halo
constexpr int ROWB = C * 2;                  // 64 bytes per voxel of a map
constexpr int WMID = NTAP * C * C;           // 27648 weights of a 32 -> 32 layer
constexpr int kMaxOut = 8;                   // output maps of the last layer, at most
constexpr int kMaxPart = 512;                // cap of per-block partial slots (weight gradients)
constexpr int kMaxLossPart = 1024;


struct Dims {
  int nz, ny, nx;
  int tx, ty, tz;   // tiles along each axis
  int ntiles;
  long long nvox;
};

inline Dims make_dims(int nz, int ny, int nx) {
  Dims d;
  d.nz = nz; d.ny = ny; d.nx = nx;
  d.tx = (nx + TX - 1) / TX; d.ty = (ny + TY - 1) / TY; d.tz = (nz + TZ - 1) / TZ;
  d.ntiles = d.tx * d.ty * d.tz;
  d.nvox = (long long)nz * ny * nx;
  return d;
}

// ------------------------------------------------------------------ helpers

__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ uint32_t swz(int row, int chunk) {
  return (uint32_t)(row * ROWB + ((chunk ^ ((row >> 1) & 3)) << 4));
}

__device__ __forceinline__ void cp_async16(uint32_t dst, const void* src, int src_bytes) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;\n" ::"r"(dst), "l"(src), "r"(src_bytes) : "memory");
}

__device__ __forceinline__ void cp_async_wait_all() {
  asm volatile("cp.async.commit_group;\ncp.async.wait_group 0;\n" ::: "memory");
}

__device__ __forceinline__ void tile_origin(int tile, const Dims& d, int& z0, int& y0, int& x0) {
  const int tx = tile % d.tx;
  const int r = tile / d.tx;
  x0 = tx * TX;
  y0 = (r % d.ty) * TY;
  z0 = (r / d.ty) * TZ;
}

__device__ __forceinline__ bool inside(const Dims& d, int z, int y, int x) {
  return (unsigned)z < (unsigned)d.nz && (unsigned)y < (unsigned)d.ny && (unsigned)x < (unsigned)d.nx;
}

__device__ __forceinline__ size_t vox(const Dims& d, int z, int y, int x) {
  return ((size_t)z * d.ny + y) * d.nx + x;
}

// NZS slices of a map starting at channel zs, rows y0-1 .. y0+TY, columns
// x0-1 .. x0+TX, into swizzled shared rows h = (hz*HY + hy)*HX + hx.
template <int NZS>
__device__ __forceinline__ void load_map_halo(uint32_t s, const bf16* __restrict__ g, const Dims& d, int zs, int y0,
                                              int x0) {
  constexpr int N = NZS * HY * HX * 4;
  for (int i = threadIdx.x; i < N; i += blockDim.x) {
    const int c = i & 3, h = i >> 2;
    const int hx = h % HX, t = h / HX, hy = t % HY, hz = t / HY;
    const int gz = zs + hz, gy = y0 - 1 + hy, gx = x0 - 1 + hx;
    const bool ok = inside(d, gz, gy, gx);
    const bf16* src = ok ? g + vox(d, gz, gy, gx) * C + c * 8 : g;
    cp_async16(s + swz(h, c), src, ok ? 16 : 0);
  }
}

// Scalar field halo (float32 cube or bfloat16 single-feature map) into s[h], zero outside.
template <typename T>
__device__ __forceinline__ void load_scalar_halo(float* s, const T* __restrict__ g, const Dims& d, int z0, int y0,
                                                 int x0) {
  for (int h = threadIdx.x; h < HV; h += blockDim.x) {
    const int hx = h % HX, t = h / HX, hy = t % HY, hz = t / HY;
    const int gz = z0 - 1 + hz, gy = y0 - 1 + hy, gx = x0 - 1 + hx;
    float v = 0.f;
    if (inside(d, gz, gy, gx)) v = static_cast<float>(g[vox(d, gz, gy, gx)]);
    s[h] = v;
  }
}

__device__ __forceinline__ void unpack8(uint4 q, float* f) {
  const bf162* p = reinterpret_cast<const bf162*>(&q);
#pragma unroll
  for (int e = 0; e < 4; ++e) {
    const float2 t = __bfloat1622float2(p[e]);
    f[2 * e] = t.x;
    f[2 * e + 1] = t.y;
  }
}

__device__ __forceinline__ uint4 pack8(const float* f) {
  uint4 q;
  bf162* p = reinterpret_cast<bf162*>(&q);
#pragma unroll
  for (int e = 0; e < 4; ++e) p[e] = __floats2bfloat162_rn(f[2 * e], f[2 * e + 1]);
  return q;
}

// ------------------------------------------------------------------ 32 -> 32 layers on the tensor cores

// Epilogues of the tcgen05 layer: the 32 -> 32 layers (bias + ReLU, bias, or
// the ReLU mask of an input gradient) and the last layer (prediction, or loss).
enum { EPI_RELU = 0, EPI_BIAS = 1, EPI_MASK = 2, EPI_PRED = 3, EPI_LOSS = 4 };

// Per-output-map constants of the last layer (at most kMaxOut maps), by value.
struct Lam {
  float v[kMaxOut];
};

// Operands of the last layer's epilogues (unused by the 32 -> 32 layers).
struct LastArgs {
  int K;                      // output maps
  Lam lam;                    // loss weights
  const float* s;             // input scale (device scalar)
  const float* tx;            // EPI_LOSS: target cube [V]
  const bf16* taux;           // EPI_LOSS: target fields [nz][K-1][ny][nx]
  float* d6;                  // EPI_LOSS: loss gradient [V][K]
  double* lpart;              // EPI_LOSS: per-CTA partial sums [grid][K+1]
  float* out_x;               // EPI_PRED: cube [V]
  float* out_aux;             // EPI_PRED: fields [nz][K-1][ny][nx]
};

// ------------------------------------------------------------------ 32 -> 32 layers on tcgen05 (UMMA), fed by TMA
//
// One CTA of 128 threads walks output tiles of 128 voxels (one channel, 16
// rows, 8 columns).  For each tile D[128 voxels][32 features] accumulates in
// tensor memory over 27 taps x 2 steps of K = 16 by tcgen05.mma (kind::f16,
// bfloat16 A and B, float32 D, M = 128, N = 32; N = 16 for the last layer,
// whose epilogue writes the prediction or the loss terms); both operands are read from
// shared memory through descriptors in the canonical K-major layout without
// swizzle (8-row x 16-byte core matrices).
//
// The tile's input halo (3 x 18 x 10 voxels) arrives by TMA: one
// cp.async.bulk.tensor per 8-feature chunk, from a 4-D tensor map over
// (8 features, x, y, z) of the [z][y][x][32] map (strides 64 B, 64 nx B,
// 64 nx ny B; base offset 16 B per chunk).  A box lands as one chunk plane
// [z][y][x][16 B], so the 8 consecutive voxels of an output row are one core
// matrix in every tap's shifted window: rows of a window are 16 B apart, the
// next output row (next 8-row group) is one halo row (160 B) further, the next
// 8 input features one chunk plane further (planes padded to 8704 B, TMA wants
// 128-byte aligned destinations).  Outside the cube the copy fills zeros: the
// zero padding of the layer.  Weights are [tap][chunk][co][16 B] (next 8
// outputs 128 B, next 8 inputs 512 B), loaded once per CTA.
//
// One halo buffer (90 KB of shared memory in all, two CTAs per SM): thread 0
// issues tile i's MMAs (commit -> mbarrier mdone); once they have read the
// halo, it issues the TMA of tile i+1 (mbarrier full), which then runs under
// tile i's epilogue, while the SM's other CTA keeps the tensor core busy.
// Every wait is bounded: on timeout the CTA records it in g_tc_timeouts,
// waits (bounded) for its copy in flight, skips its remaining tiles and still
// frees its tensor memory.
constexpr int U_TY = 16, U_TX = 8;                          // output tile: 16 rows x 8 columns, one channel
constexpr int U_HY = U_TY + 2, U_HX = U_TX + 2;             // 18 x 10 halo per channel slice
constexpr int U_HV = 3 * U_HY * U_HX;                       // 540 voxels
constexpr int U_BOX = U_HV * 16;                            // bytes of one chunk box: 8640
constexpr int U_CHUNK = 8704;                               // chunk plane stride (128-byte multiple)
constexpr int U_HALO = 4 * U_CHUNK;                         // 34816
constexpr int kLastN = 16;                                  // MMA width of the last layer (K <= 8 maps used)
template <int EPI> __host__ __device__ constexpr int epi_n() { return EPI >= EPI_PRED ? kLastN : C; }
// weights: 55296 B (N = 32), 27648 B (N = 16); then 2 mbarriers and the TMEM address slot; alignment slack
__host__ __device__ constexpr int u_w(int no) { return NTAP * 4 * no * 16; }
__host__ __device__ constexpr int u_bar(int no) { return U_HALO + u_w(no); }
__host__ __device__ constexpr int conv05_smem(int no) { return u_bar(no) + 64 + 128; }
// D f32, A/B bf16, both K-major, N = no, M = 128
__host__ __device__ constexpr uint32_t idesc_bf16(int no) {
  return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(no >> 3) << 17) | ((uint32_t)(128 >> 4) << 24);
}
constexpr long long kWaitLimit = 1LL << 20;   // polls; each may suspend for a bounded time

__device__ int g_tc_timeouts;
// Poll bound of the pipeline waits (settable through muffin_net_set_wait_limit).
// The drain waits after a give-up keep the full bound kWaitLimit, so that no
// copy or MMA lands in shared or tensor memory after the CTA has left.
__device__ long long g_wait_polls = kWaitLimit;

struct HaloMaps {
  CUtensorMap m[4];   // one per 8-feature chunk
};

__device__ __forceinline__ uint64_t umma_desc(uint32_t addr, uint32_t lbo, uint32_t sbo) {
  uint64_t d = (uint64_t)((addr >> 4) & 0x3FFFu);
  d |= (uint64_t)((lbo >> 4) & 0x3FFFu) << 16;
  d |= (uint64_t)((sbo >> 4) & 0x3FFFu) << 32;
  d |= (uint64_t)1 << 46;   // descriptor version of sm_100 and later; swizzle mode 0 (none)
  return d;
}

__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

__device__ __forceinline__ bool mbar_wait_n(uint32_t bar, uint32_t parity, long long limit) {
  uint32_t done = 0;
  for (long long it = 0; it < limit && !done; ++it) {
    asm volatile(
        "{\n.reg .pred p;\nmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\nselp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(done)
        : "r"(bar), "r"(parity)
        : "memory");
  }
  return done != 0;
}
// pipeline wait: gives up after g_wait_polls polls
__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity) {
  return mbar_wait_n(bar, parity, *(volatile long long*)&g_wait_polls);
}
// drain wait after a give-up: the full bound
__device__ __forceinline__ bool mbar_drain(uint32_t bar, uint32_t parity) { return mbar_wait_n(bar, parity, kWaitLimit); }

// Thread 0: the four chunk boxes of the tile at (x0, y0, z0) into halo buffer s_dst.
__device__ __forceinline__ void issue_halo(const HaloMaps& maps, uint32_t s_dst, uint32_t bar, int x0, int y0,
                                           int z0) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(4 * U_BOX) : "memory");
#pragma unroll
  for (int c = 0; c < 4; ++c)
    asm volatile(
        "cp.async.bulk.tensor.4d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4, %5}], "
        "[%6];" ::"r"(s_dst + (uint32_t)(c * U_CHUNK)),
        "l"(reinterpret_cast<uint64_t>(&maps.m[c])), "r"(0), "r"(x0 - 1), "r"(y0 - 1), "r"(z0 - 1), "r"(bar)
        : "memory");
}

template <int EPI>
__global__ void __launch_bounds__(128)
k_conv_tc05(const __grid_constant__ HaloMaps maps, const bf16* __restrict__ wk, const float* __restrict__ bias,
            const bf16* __restrict__ mask, bf16* __restrict__ out, Dims d, int tiles_x, int tiles_y, int ntiles,
            LastArgs la) {
  constexpr int NO = epi_n<EPI>();
  constexpr bool kLast = EPI >= EPI_PRED;
  extern __shared__ __align__(128) unsigned char smem[];
  __shared__ double s_red[32];
  const uint32_t s0 = (smem_u32(smem) + 127u) & ~127u;
  const uint32_t s_halo = s0;
  const uint32_t s_w = s0 + U_HALO;
  const uint32_t s_full = s0 + u_bar(NO);         // TMA landed
  const uint32_t s_done = s_full + 8;              // MMAs finished
  const uint32_t s_tm = s_full + 16;               // TMEM address written by tcgen05.alloc
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;

  // weights [tap][co][ci] -> [tap][chunk][co][16 B], once per CTA
  for (int i = threadIdx.x; i < NTAP * NO * 4; i += blockDim.x) {
    const int c = i & 3, co = (i >> 2) % NO, t = i / (4 * NO);
    cp_async16(s_w + (uint32_t)(((t * 4 + c) * NO + co) * 16), wk + (t * NO + co) * C + c * 8, 16);
  }
  cp_async_wait_all();
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");   // generic-proxy writes, read by the MMA
  if (threadIdx.x == 0) {
#pragma unroll
    for (int b = 0; b < 2; ++b) asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(s_full + 8 * b) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], 32;" ::"r"(s_tm) : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  uint32_t tmem;
  asm volatile("ld.shared.b32 %0, [%1];" : "=r"(tmem) : "r"(s_tm) : "memory");

  float bn[NO];
#pragma unroll
  for (int c = 0; c < NO; ++c) bn[c] = (EPI != EPI_MASK && bias && (!kLast || c < la.K)) ? bias[c] : 0.f;
  // last layer: input scale, and this thread's loss sums
  const float sc = kLast ? *la.s : 1.f;
  const float inv_sc = 1.0f / sc;
  const double gs = 2.0 / (double)d.nvox;
  const size_t plane = (size_t)d.ny * d.nx;
  double l2 = 0.0;
  double lsum[kMaxOut];
#pragma unroll
  for (int k = 0; k < kMaxOut; ++k) lsum[k] = 0.0;

  auto origin = [&](int tile, int& x0, int& y0, int& z0) {
    const int txi = tile % tiles_x, rr = tile / tiles_x;
    x0 = txi * U_TX;
    y0 = (rr % tiles_y) * U_TY;
    z0 = rr / tiles_y;
  };
  // thread 0 tracks the halo copy it may have in flight, so that an early
  // exit can wait for it before the CTA's shared memory goes away
  bool pending = false;
  uint32_t pend_ph = 0;
  // and the MMAs it committed but has not yet seen finish
  bool mma_pending = false;
  uint32_t mma_ph = 0;
  if (threadIdx.x == 0 && (int)blockIdx.x < ntiles) {
    int x0, y0, z0;
    origin(blockIdx.x, x0, y0, z0);
    issue_halo(maps, s_halo, s_full, x0, y0, z0);
    pending = true;
  }

  int it = 0;
  for (int tile = blockIdx.x; tile < ntiles; tile += gridDim.x, ++it) {
    const uint32_t ph = (uint32_t)it & 1u;
    int x0, y0, z0;
    origin(tile, x0, y0, z0);
    if (threadIdx.x == 0) {
      if (mbar_wait(s_full, ph)) {
        pending = false;
        tc_fence_after();
        const uint32_t hb = s_halo;
        const uint32_t dt = tmem;
#pragma unroll 1
        for (int t = 0; t < NTAP; ++t) {
          const int kz = t / 9, ky = (t / 3) % 3, kx = t % 3;
          const uint32_t a0 = hb + (uint32_t)(((kz * U_HY + ky) * U_HX + kx) * 16);
          const uint32_t b0 = s_w + (uint32_t)(t * 4 * NO * 16);
#pragma unroll
          for (int kk = 0; kk < 2; ++kk) {
            const uint64_t ad = umma_desc(a0 + kk * 2 * U_CHUNK, U_CHUNK, U_HX * 16);
            const uint64_t bd = umma_desc(b0 + kk * 2 * NO * 16, NO * 16, 8 * 16);
            const uint32_t acc = (t | kk) != 0;
            asm volatile(
                "{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\n"
                "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(dt),
                "l"(ad), "l"(bd), "r"(idesc_bf16(NO)), "r"(acc)
                : "memory");
          }
        }
        asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(s_done)
                     : "memory");
        mma_pending = true;
        mma_ph = ph;
      }
    }
    const bool done = mbar_wait(s_done, ph);
    if (threadIdx.x == 0 && done) mma_pending = false;
    if (__syncthreads_or(!done)) {          // one decision for the whole block
      if (threadIdx.x == 0) atomicAdd(&g_tc_timeouts, 1);
      break;
    }
    // the MMAs have read the halo: the next tile's copy runs under this epilogue
    if (threadIdx.x == 0 && tile + (int)gridDim.x < ntiles) {
      int nx0, ny0, nz0;
      origin(tile + gridDim.x, nx0, ny0, nz0);
      issue_halo(maps, s_halo, s_full, nx0, ny0, nz0);
      pending = true;
      pend_ph = (uint32_t)(it + 1) & 1u;
    }
    tc_fence_after();
    // row m = 32 warp + lane of D is output voxel (y0 + m / 8, x0 + m % 8) of channel z0
    const int m = warp * 32 + lane;
    const int z = z0, y = y0 + (m >> 3), x = x0 + (m & 7);
    const uint32_t taddr = tmem + ((uint32_t)(warp * 32) << 16);
    if constexpr (!kLast) {
      uint32_t r[C];
      asm volatile(
          "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
          "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];\n"
          : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
            "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]),
            "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]),
            "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
          : "r"(taddr));
      asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
      if (inside(d, z, y, x)) {
        const size_t base = vox(d, z, y, x) * C;
        float v[C];
#pragma unroll
        for (int c = 0; c < C; ++c) v[c] = __uint_as_float(r[c]);
        if (EPI == EPI_MASK) {
          if (mask) {
            const uint4* mp = reinterpret_cast<const uint4*>(mask + base);
#pragma unroll
            for (int q = 0; q < 4; ++q) {
              float mf[8];
              unpack8(mp[q], mf);
#pragma unroll
              for (int e = 0; e < 8; ++e)
                if (!(mf[e] > 0.f)) v[8 * q + e] = 0.f;
            }
          }
        } else {
#pragma unroll
          for (int c = 0; c < C; ++c) {
            v[c] += bn[c];
            if (EPI == EPI_RELU) v[c] = fmaxf(v[c], 0.f);
          }
        }
        uint4* o = reinterpret_cast<uint4*>(out + base);
#pragma unroll
        for (int q = 0; q < 4; ++q) o[q] = pack8(v + 8 * q);
      }
    } else {
      // last layer: z_k = D[m][k] + b_k for the K maps (columns K .. 15 hold zero weights)
      uint32_t r[kLastN];
      asm volatile(
          "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];\n"
          : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
            "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
          : "r"(taddr));
      asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
      if (inside(d, z, y, x)) {
        const int K = la.K;
        const size_t v = vox(d, z, y, x);
        const size_t a0 = ((size_t)z * (K > 1 ? K - 1 : 1)) * plane + (size_t)y * d.nx + x;
#pragma unroll
        for (int k = 0; k < kMaxOut; ++k) {
          if (k < K) {
            const float zk = __uint_as_float(r[k]) + bn[k];
            if constexpr (EPI == EPI_LOSS) {
              const float tk = k == 0 ? la.tx[v] * inv_sc : __bfloat162float(la.taux[a0 + (size_t)(k - 1) * plane]);
              const float rk = zk - tk;
              la.d6[v * K + k] = (float)(gs * la.lam.v[k]) * rk;
              l2 += (double)la.lam.v[k] * rk * rk;
              lsum[k] += rk;
            } else {
              if (k == 0) la.out_x[v] = fmaxf(sc * zk, 0.f);
              else la.out_aux[a0 + (size_t)(k - 1) * plane] = fminf(fmaxf(zk, -1.f), 1.f);
            }
          }
        }
      }
    }
    tc_fence_before();
    __syncthreads();     // the accumulator is read before the next tile's MMAs overwrite it
    tc_fence_after();
  }
  // only after a give-up: the copy and the MMAs still in flight land before the CTA leaves
  if (threadIdx.x == 0 && pending) mbar_drain(s_full, pend_ph);
  if (threadIdx.x == 0 && mma_pending) mbar_drain(s_done, mma_ph);
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, 32;" ::"r"(tmem) : "memory");
  if constexpr (EPI == EPI_LOSS) {
    // lpart[block] = (sum_k lam_k sum_p r_k^2, sum_p r_0, ..., sum_p r_{K-1}), fixed order
    const double t2 = muffin::block_sum(l2, s_red);
    if (threadIdx.x == 0) la.lpart[(size_t)blockIdx.x * (la.K + 1)] = t2;
#pragma unroll
    for (int k = 0; k < kMaxOut; ++k) {
      if (k >= la.K) break;
      __syncthreads();
      const double tk = muffin::block_sum(lsum[k], s_red);
      if (threadIdx.x == 0) la.lpart[(size_t)blockIdx.x * (la.K + 1) + 1 + k] = tk;
    }
  }
}

// ------------------------------------------------------------------ 32 -> 32 weight gradient on tcgen05, fed by TMA
//
// dW[tap][co][ci] = sum_p dz[p][co] a[p + d(tap)][ci] as tensor-core products
// D[m][n] += A[m][k] B[k][n] with k = output voxel p, n = co and
// m = (ky, ci): one 128-row accumulator per (kz, kx) holds the three row
// offsets ky = 0..2 of the tap (rows 96..127, "ky = 3", are computed and
// dropped).  Nine accumulators of 32 float32 columns stay in tensor memory for
// the CTA's whole run over its tiles; the sums leave TMEM once, at the end.
//
// Both operands are MN-major (M or N contiguous: the 8 features of a chunk),
// canonical layout without swizzle: core matrices of 8 voxels x 16 bytes.
// The input halo of a tile (3 x 19 x 10 voxels: rows y0-1 .. y0+17, the last
// one only feeding the dropped rows) lands by one TMA copy as
// [y][chunk][z][x][16 B] (a 5-D tensor map over (8 features, x, z, chunk, y)
// with a 16-byte chunk stride): the next 8 rows of m (next chunk, or next ky
// after four chunks) are 480 B apart, the next 8 voxels of k (next output
// row) 1920 B.  The tile's own dz lands as [y][chunk][x][16 B]: next 8 co
// 128 B, next 8 voxels 512 B.
//
// Thread 0 keeps a three-stage TMA ring ahead of its MMAs (72 per tile:
// 9 accumulators x 8 steps of K = 16); warp 1 sums the dz tiles into the bias
// gradient as they land and releases each stage through an mbarrier.  One CTA
// per SM (the ring takes 146 KB of shared memory; the accumulators take all
// 512 TMEM columns).  Every wait is bounded; a CTA that gives up records it in
// g_tc_timeouts, waits (bounded) for its copies and MMAs in flight, writes
// nothing and frees its tensor memory.
constexpr int WG_HY = U_TY + 3;                        // 19 halo rows (one extra for the dropped rows)
constexpr int WG_A = WG_HY * 4 * 3 * U_HX * 16;        // 36480 B: [19][4][3][10][16 B]
constexpr int WG_ROW = 4 * 3 * U_HX * 16;              // 1920 B per halo row
constexpr int WG_B = U_TY * 4 * U_TX * 16;             // 8192 B: [16][4][8][16 B]
constexpr int WG_STAGE = WG_A + WG_B;                  // 44672 B (a multiple of 128)
constexpr int WG_NS = 3;                               // ring stages
constexpr int WG_SLACK = 16384;                        // room past the ring that no descriptor layout can leave
constexpr int WG_BAR = WG_NS * WG_STAGE + WG_SLACK;    // full[3], done[3], freed[3], fin, TMEM slot
constexpr int wgrad05_smem = WG_BAR + 128 + 128;
// D f32, A/B bf16, both MN-major, N = 32, M = 128
constexpr uint32_t kIdescWgrad = (1u << 4) | (1u << 7) | (1u << 10) | (1u << 15) | (1u << 16) |
                                 ((uint32_t)(C >> 3) << 17) | ((uint32_t)(128 >> 4) << 24);

struct WgradMaps {
  CUtensorMap a;    // (8, x, z, chunk, y) of the layer input
  CUtensorMap dz;   // (8, x, chunk, y, z) of the output gradient
};

__device__ __forceinline__ void wg_issue(const WgradMaps& maps, uint32_t stage, uint32_t bar, int x0, int y0, int z0) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(WG_STAGE) : "memory");
  asm volatile(
      "cp.async.bulk.tensor.5d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4, %5, %6}], "
      "[%7];" ::"r"(stage),
      "l"(reinterpret_cast<uint64_t>(&maps.a)), "r"(0), "r"(x0 - 1), "r"(z0 - 1), "r"(0), "r"(y0 - 1), "r"(bar)
      : "memory");
  asm volatile(
      "cp.async.bulk.tensor.5d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4, %5, %6}], "
      "[%7];" ::"r"(stage + WG_A),
      "l"(reinterpret_cast<uint64_t>(&maps.dz)), "r"(0), "r"(x0), "r"(0), "r"(y0), "r"(z0), "r"(bar)
      : "memory");
}

__global__ void __launch_bounds__(128)
k_wgrad_tc05(const __grid_constant__ WgradMaps maps, float* __restrict__ part, float* __restrict__ bpart, Dims d,
             int tiles_x, int tiles_y, int ntiles) {
  extern __shared__ __align__(128) unsigned char smem[];
  const uint32_t s0 = (smem_u32(smem) + 127u) & ~127u;
  const uint32_t s_full = s0 + WG_BAR;          // TMA landed, per stage
  const uint32_t s_done = s_full + 8 * WG_NS;   // MMAs of the stage's tile finished
  const uint32_t s_freed = s_done + 8 * WG_NS;  // warp 1 has read the stage's dz
  const uint32_t s_fin = s_freed + 8 * WG_NS;   // every MMA of the CTA finished
  const uint32_t s_tm = s_fin + 8;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (threadIdx.x == 0) {
    for (int b = 0; b < WG_NS; ++b) {
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(s_full + 8 * b) : "memory");
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(s_done + 8 * b) : "memory");
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 32;" ::"r"(s_freed + 8 * b) : "memory");
    }
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(s_fin) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], 512;" ::"r"(s_tm) : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  uint32_t tmem;
  asm volatile("ld.shared.b32 %0, [%1];" : "=r"(tmem) : "r"(s_tm) : "memory");

  auto origin = [&](int tile, int& x0, int& y0, int& z0) {
    const int txi = tile % tiles_x, rr = tile / tiles_x;
    x0 = txi * U_TX;
    y0 = (rr % tiles_y) * U_TY;
    z0 = rr / tiles_y;
  };
  const int nmine = ntiles > (int)blockIdx.x ? (ntiles - (int)blockIdx.x + (int)gridDim.x - 1) / (int)gridDim.x : 0;
  bool ok = true;
  float bacc = 0.f;
  if (threadIdx.x == 0) {
    // per stage: bit b of `used` once a copy was issued into it, bit b of
    // `odd` the parity of the number of copies (what an early exit waits for)
    uint32_t used = 0, odd = 0;
    for (int i = 0; i < WG_NS && i < nmine; ++i) {
      int x0, y0, z0;
      origin(blockIdx.x + i * gridDim.x, x0, y0, z0);
      wg_issue(maps, s0 + i * WG_STAGE, s_full + 8 * i, x0, y0, z0);
      used |= 1u << i;
      odd ^= 1u << i;
    }
    for (int it = 0; it < nmine && ok; ++it) {
      const int s = it % WG_NS;
      const uint32_t ph = (uint32_t)(it / WG_NS) & 1u;
      if (!mbar_wait(s_full + 8 * s, ph)) { ok = false; break; }
      tc_fence_after();
      const uint32_t sa = s0 + s * WG_STAGE, sb = sa + WG_A;
#pragma unroll 1
      for (int acc = 0; acc < 9; ++acc) {
        const int kz = acc / 3, kx = acc % 3;
#pragma unroll
        for (int rp = 0; rp < U_TY / 2; ++rp) {
          const uint64_t ad = umma_desc(sa + (uint32_t)(2 * rp * WG_ROW + kz * U_HX * 16 + kx * 16), WG_ROW, 3 * U_HX * 16);
          const uint64_t bd = umma_desc(sb + (uint32_t)(2 * rp * 4 * U_TX * 16), 4 * U_TX * 16, U_TX * 16);
          const uint32_t accum = (it | rp) != 0;
          asm volatile(
              "{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\n"
              "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem + (uint32_t)(acc * C)),
              "l"(ad), "l"(bd), "r"(kIdescWgrad), "r"(accum)
              : "memory");
        }
      }
      asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(s_done + 8 * s)
                   : "memory");
      // refill the stage of the previous tile once its MMAs and warp 1 are done with it
      if (it >= 1 && it - 1 + WG_NS < nmine) {
        const int sp = (it - 1) % WG_NS;
        const uint32_t pp = (uint32_t)((it - 1) / WG_NS) & 1u;
        if (!mbar_wait(s_done + 8 * sp, pp) || !mbar_wait(s_freed + 8 * sp, pp)) { ok = false; break; }
        int x0, y0, z0;
        origin(blockIdx.x + (it - 1 + WG_NS) * gridDim.x, x0, y0, z0);
        wg_issue(maps, s0 + sp * WG_STAGE, s_full + 8 * sp, x0, y0, z0);
        odd ^= 1u << sp;
      }
    }
    // every MMA issued so far, then the copies still in flight (only after a timeout)
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(s_fin) : "memory");
    if (!ok)
      for (int b = 0; b < WG_NS; ++b)
        if ((used >> b) & 1u) mbar_drain(s_full + 8 * b, ((odd >> b) & 1u) ^ 1u);
  } else if (warp == 1) {
    // bias gradient: bacc = sum of dz[p][co = lane] over this CTA's voxels
    for (int it = 0; it < nmine && ok; ++it) {
      const int s = it % WG_NS;
      const uint32_t ph = (uint32_t)(it / WG_NS) & 1u;
      if (!mbar_wait(s_full + 8 * s, ph)) { ok = false; break; }
      const unsigned char* b = smem + (s0 - smem_u32(smem)) + s * WG_STAGE + WG_A;
      const int c = lane >> 3, e = lane & 7;
#pragma unroll 8
      for (int v = 0; v < U_TY * U_TX; ++v)
        bacc += __bfloat162float(*reinterpret_cast<const bf16*>(b + ((v >> 3) * 4 + c) * 128 + (v & 7) * 16 + e * 2));
      asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(s_freed + 8 * s) : "memory");
    }
  }
  const bool fin = mbar_drain(s_fin, 0);   // every MMA issued, also after a give-up: TMEM is freed below
  if (__syncthreads_or(!ok || !fin)) {
    if (threadIdx.x == 0) atomicAdd(&g_tc_timeouts, 1);
  } else {
    tc_fence_after();
    if (warp < 3) {
      // lane = ci, TMEM lanes 32 ky .. 32 ky + 31; accumulator (kz, kx) -> tap kz*9 + ky*3 + kx
#pragma unroll 1
      for (int q = 0; q < 18; ++q) {            // accumulator q / 2, columns (co) 16 (q % 2) .. + 15
        const int acc = q >> 1, co0 = (q & 1) * 16;
        uint32_t r[16];
        asm volatile(
            "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];\n"
            : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
              "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
            : "r"(tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)(acc * C + co0)));
        asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
        const int tap = (acc / 3) * 9 + warp * 3 + acc % 3;
        float* pp = part + ((size_t)blockIdx.x * NTAP + tap) * (C * C) + co0 * C + lane;
#pragma unroll
        for (int j = 0; j < 16; ++j) pp[j * C] = __uint_as_float(r[j]);
      }
    }
    if (warp == 1 && bpart) bpart[(size_t)blockIdx.x * C + lane] = bacc;
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, 512;" ::"r"(tmem) : "memory");
}

// ------------------------------------------------------------------ first and last layers (CUDA cores)

// Thread -> voxel (tz, ty, tx) of the tile.
__device__ __forceinline__ void thread_voxel(int& tz, int& ty, int& tx) {
  tx = threadIdx.x & 15;
  ty = (threadIdx.x >> 4) & 7;
  tz = threadIdx.x >> 7;
}

// a1[p][co] = relu(b[co] + sum_tap a0[p + d(tap)] w[tap][co]).
__global__ void __launch_bounds__(256)
k_first_fwd(const bf16* __restrict__ a0, const float* __restrict__ w, const float* __restrict__ b,
            bf16* __restrict__ a1, Dims d) {
  __shared__ __align__(16) float s_w[NTAP * C];
  __shared__ float s_b[C];
  __shared__ float s_h[HV];
  for (int i = threadIdx.x; i < NTAP * C; i += blockDim.x) s_w[i] = w[i];
  if (threadIdx.x < C) s_b[threadIdx.x] = b[threadIdx.x];
  int tz, ty, tx;
  thread_voxel(tz, ty, tx);
  for (int tile = blockIdx.x; tile < d.ntiles; tile += gridDim.x) {
    int z0, y0, x0;
    tile_origin(tile, d, z0, y0, x0);
    __syncthreads();
    load_scalar_halo(s_h, a0, d, z0, y0, x0);
    __syncthreads();
    float acc[C];
#pragma unroll
    for (int c = 0; c < C; ++c) acc[c] = s_b[c];
#pragma unroll 1
    for (int t = 0; t < NTAP; ++t) {
      const int kz = t / 9, ky = (t / 3) % 3, kx = t % 3;
      const float av = s_h[((tz + kz) * HY + ty + ky) * HX + tx + kx];
      const float4* wr = reinterpret_cast<const float4*>(s_w + t * C);
#pragma unroll
      for (int q = 0; q < C / 4; ++q) {
        const float4 wv = wr[q];
        acc[4 * q] = fmaf(av, wv.x, acc[4 * q]);
        acc[4 * q + 1] = fmaf(av, wv.y, acc[4 * q + 1]);
        acc[4 * q + 2] = fmaf(av, wv.z, acc[4 * q + 2]);
        acc[4 * q + 3] = fmaf(av, wv.w, acc[4 * q + 3]);
      }
    }
    const int z = z0 + tz, y = y0 + ty, x = x0 + tx;
    if (inside(d, z, y, x)) {
#pragma unroll
      for (int c = 0; c < C; ++c) acc[c] = fmaxf(acc[c], 0.f);
      uint4* o = reinterpret_cast<uint4*>(a1 + vox(d, z, y, x) * C);
#pragma unroll
      for (int q = 0; q < 4; ++q) o[q] = pack8(acc + 8 * q);
    }
  }
}

// g5[p][ci] = (a5[p][ci] > 0) * sum_tap sum_k d6[p - d(tap)][k] w[tap][k][ci].
template <int K>
__global__ void __launch_bounds__(256)
k_last_bwd_data(const float* __restrict__ d6, const float* __restrict__ w, const bf16* __restrict__ a5,
                bf16* __restrict__ g5, Dims d) {
  extern __shared__ __align__(16) float smf[];
  float* s_w = smf;                      // [27][K][32]
  float* s_h = smf + NTAP * K * C;       // [HV][K]
  for (int i = threadIdx.x; i < NTAP * K * C; i += blockDim.x) s_w[i] = w[i];
  int tz, ty, tx;
  thread_voxel(tz, ty, tx);
  for (int tile = blockIdx.x; tile < d.ntiles; tile += gridDim.x) {
    int z0, y0, x0;
    tile_origin(tile, d, z0, y0, x0);
    __syncthreads();
    for (int i = threadIdx.x; i < HV * K; i += blockDim.x) {
      const int h = i / K, k = i - h * K;
      const int hx = h % HX, r = h / HX, hy = r % HY, hz = r / HY;
      const int gz = z0 - 1 + hz, gy = y0 - 1 + hy, gx = x0 - 1 + hx;
      s_h[i] = inside(d, gz, gy, gx) ? d6[vox(d, gz, gy, gx) * K + k] : 0.f;
    }
    __syncthreads();
    float acc[C];
#pragma unroll
    for (int c = 0; c < C; ++c) acc[c] = 0.f;
#pragma unroll 1
    for (int t = 0; t < NTAP; ++t) {
      const int kz = t / 9, ky = (t / 3) % 3, kx = t % 3;
      const int hh = ((tz + 2 - kz) * HY + ty + 2 - ky) * HX + tx + 2 - kx;
#pragma unroll
      for (int k = 0; k < K; ++k) {
        const float dv = s_h[hh * K + k];
        const float4* wr = reinterpret_cast<const float4*>(s_w + (t * K + k) * C);
#pragma unroll
        for (int q = 0; q < C / 4; ++q) {
          const float4 wv = wr[q];
          acc[4 * q] = fmaf(dv, wv.x, acc[4 * q]);
          acc[4 * q + 1] = fmaf(dv, wv.y, acc[4 * q + 1]);
          acc[4 * q + 2] = fmaf(dv, wv.z, acc[4 * q + 2]);
          acc[4 * q + 3] = fmaf(dv, wv.w, acc[4 * q + 3]);
        }
      }
    }
    const int z = z0 + tz, y = y0 + ty, x = x0 + tx;
    if (inside(d, z, y, x)) {
      const size_t v = vox(d, z, y, x);
      const uint4* m = reinterpret_cast<const uint4*>(a5 + v * C);
      uint4* o = reinterpret_cast<uint4*>(g5 + v * C);
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        float mf[8];
        unpack8(m[q], mf);
#pragma unroll
        for (int e = 0; e < 8; ++e)
          if (!(mf[e] > 0.f)) acc[8 * q + e] = 0.f;
        o[q] = pack8(acc + 8 * q);
      }
    }
  }
}

// part[b][tap][co] = sum_p g1[p][co] a0[p + d(tap)]; bpart[b][co] = sum_p g1[p][co].
// 288 threads: thread (kz, ky, co) keeps the three taps kx = 0..2 of its row
// offset and walks each tile row along x with a sliding window of three a0
// values (one a0 and one g1 read per 3 multiply-adds).
__global__ void __launch_bounds__(288)
k_wgrad_first(const bf16* __restrict__ a0, const bf16* __restrict__ g1, float* __restrict__ part,
              float* __restrict__ bpart, Dims d) {
  __shared__ float s_h[HV];
  __shared__ __align__(16) float s_g[TV * C];
  const int co = threadIdx.x & 31, kzy = threadIdx.x >> 5, kz = kzy / 3, ky = kzy % 3;
  float acc0 = 0.f, acc1 = 0.f, acc2 = 0.f, bacc = 0.f;
  for (int tile = blockIdx.x; tile < d.ntiles; tile += gridDim.x) {
    int z0, y0, x0;
    tile_origin(tile, d, z0, y0, x0);
    __syncthreads();
    load_scalar_halo(s_h, a0, d, z0, y0, x0);
    for (int i = threadIdx.x; i < TV * 4; i += blockDim.x) {
      const int c = i & 3, r = i >> 2;
      const int gz = z0 + (r >> 7), gy = y0 + ((r >> 4) & 7), gx = x0 + (r & 15);
      float f[8] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
      if (inside(d, gz, gy, gx)) unpack8(*reinterpret_cast<const uint4*>(g1 + vox(d, gz, gy, gx) * C + c * 8), f);
      float4* dst = reinterpret_cast<float4*>(s_g + r * C + c * 8);
      dst[0] = make_float4(f[0], f[1], f[2], f[3]);
      dst[1] = make_float4(f[4], f[5], f[6], f[7]);
    }
    __syncthreads();
#pragma unroll 1
    for (int row = 0; row < TZ * TY; ++row) {
      const int tz = row >> 3, ty = row & 7;
      const float* hr = s_h + ((tz + kz) * HY + ty + ky) * HX;
      const float* gr = s_g + row * TX * C + co;
      float w0 = hr[0], w1 = hr[1];
#pragma unroll 4
      for (int tx = 0; tx < TX; ++tx) {
        const float w2 = hr[tx + 2], g = gr[tx * C];
        acc0 = fmaf(g, w0, acc0);
        acc1 = fmaf(g, w1, acc1);
        acc2 = fmaf(g, w2, acc2);
        bacc += g;
        w0 = w1;
        w1 = w2;
      }
    }
  }
  float* pp = part + (size_t)blockIdx.x * (NTAP * C) + (kz * 9 + ky * 3) * C + co;
  pp[0] = acc0;
  pp[C] = acc1;
  pp[2 * C] = acc2;
  if (kzy == 0) bpart[(size_t)blockIdx.x * C + co] = bacc;
}


// part[b][tap][ci][k] = sum_p d6[p][k] a5[p + d(tap)][ci].  288 threads:
// thread (kz, ky, ci) keeps the three taps kx = 0..2 of its row offset for
// all K maps in registers and walks each tile row along x with a sliding
// window of three a5 values, so that one a5 read and the voxel's K d6 values
// (read by the whole block at once) feed 3 K multiply-adds.
template <int K>
__global__ void __launch_bounds__(288)
k_wgrad_last(const float* __restrict__ d6, const bf16* __restrict__ a5, float* __restrict__ part, Dims d) {
  extern __shared__ __align__(128) unsigned char smem[];
  const uint32_t sa = smem_u32(smem);
  float* s_d = reinterpret_cast<float*>(smem + HV * ROWB);   // [TV][K]
  const int ci = threadIdx.x & 31, kzy = threadIdx.x >> 5, kz = kzy / 3, ky = kzy % 3;
  const unsigned char* a_ci = smem + (ci & 7) * 2;
  float acc[3][K];
#pragma unroll
  for (int kx = 0; kx < 3; ++kx)
#pragma unroll
    for (int k = 0; k < K; ++k) acc[kx][k] = 0.f;
  for (int tile = blockIdx.x; tile < d.ntiles; tile += gridDim.x) {
    int z0, y0, x0;
    tile_origin(tile, d, z0, y0, x0);
    __syncthreads();
    load_map_halo<HZ>(sa, a5, d, z0 - 1, y0, x0);
    for (int i = threadIdx.x; i < TV * K; i += blockDim.x) {
      const int r = i / K, k = i - r * K;
      const int gz = z0 + (r >> 7), gy = y0 + ((r >> 4) & 7), gx = x0 + (r & 15);
      s_d[i] = inside(d, gz, gy, gx) ? d6[vox(d, gz, gy, gx) * K + k] : 0.f;
    }
    cp_async_wait_all();
    __syncthreads();
#pragma unroll 1
    for (int row = 0; row < TZ * TY; ++row) {
      const int tz = row >> 3, ty = row & 7;
      const int h0 = ((tz + kz) * HY + ty + ky) * HX;   // halo row of this thread's taps
      auto av = [&](int hx) {
        return __bfloat162float(*reinterpret_cast<const bf16*>(a_ci + swz(h0 + hx, ci >> 3)));
      };
      float w0 = av(0), w1 = av(1);
#pragma unroll 4
      for (int tx = 0; tx < TX; ++tx) {
        const float w2 = av(tx + 2);
        const float* dv = s_d + (row * TX + tx) * K;
#pragma unroll
        for (int k = 0; k < K; ++k) {
          const float g = dv[k];
          acc[0][k] = fmaf(g, w0, acc[0][k]);
          acc[1][k] = fmaf(g, w1, acc[1][k]);
          acc[2][k] = fmaf(g, w2, acc[2][k]);
        }
        w0 = w1;
        w1 = w2;
      }
    }
  }
#pragma unroll
  for (int kx = 0; kx < 3; ++kx) {
    float* pp = part + ((size_t)blockIdx.x * (NTAP * C) + (kz * 9 + ky * 3 + kx) * C + ci) * K;
#pragma unroll
    for (int k = 0; k < K; ++k) pp[k] = acc[kx][k];
  }
}

// ------------------------------------------------------------------ reductions, input, parameters

enum { MAP_PLAIN = 0, MAP_MID = 1, MAP_FIRST = 2, MAP_LAST = 3 };

// out[map(i)] = sum_b part[b*n + i] (fixed order, double accumulation).
// MAP_MID: i = (tap*32 + co)*32 + ci -> (co*32 + ci)*27 + tap; MAP_FIRST:
// i = tap*32 + co -> co*27 + tap; MAP_LAST: i = (tap*32 + ci)*K + k -> (k*32 + ci)*27 + tap.
__global__ void k_reduce_part(const float* __restrict__ part, int P, int n, float* __restrict__ out, int map, int K) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  double s = 0.0;
  for (int b = 0; b < P; ++b) s += part[(size_t)b * n + i];
  int j = i;
  if (map == MAP_MID) {
    const int t = i >> 10, co = (i >> 5) & 31, ci = i & 31;
    j = (co * C + ci) * NTAP + t;
  } else if (map == MAP_FIRST) {
    const int t = i >> 5, c = i & 31;
    j = c * NTAP + t;
  } else if (map == MAP_LAST) {
    const int k = i % K, r = i / K, ci = r & 31, t = r >> 5;
    j = (k * C + ci) * NTAP + t;
  }
  out[j] = (float)s;
}

// loss = sum_b lpart[b][0] / V; gradient of the last biases: 2 lam_k sum_b lpart[b][1+k] / V.
__global__ void k_loss_final(const double* __restrict__ lpart, int P, int K, Lam lam, long long nvox,
                             double* __restrict__ loss, float* __restrict__ grad_b6) {
  if (blockIdx.x != 0) return;
  const int k = (int)threadIdx.x - 1;
  if (k >= K) return;
  double acc = 0.0;
  for (int b = 0; b < P; ++b) acc += lpart[(size_t)b * (K + 1) + 1 + k];
  if (k < 0) {
    if (loss) *loss = acc / (double)nvox;
  } else if (grad_b6) {
    grad_b6[k] = (float)(2.0 * lam.v[k] * acc / (double)nvox);
  }
}

__global__ void k_maxabs_part(const float* __restrict__ y, long long n, float* __restrict__ part) {
  float m = 0.f;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    m = fmaxf(m, fabsf(y[i]));
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_down_sync(0xffffffffu, m, o));
  __shared__ float s[32];
  if ((threadIdx.x & 31) == 0) s[threadIdx.x >> 5] = m;
  __syncthreads();
  if (threadIdx.x == 0) {
    float r = 0.f;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) r = fmaxf(r, s[w]);
    part[blockIdx.x] = r;
  }
}

// s = max |y| (1 if the cube is zero).
__global__ void k_scale_final(const float* __restrict__ part, int P, float* __restrict__ s) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  float m = 0.f;
  for (int b = 0; b < P; ++b) m = fmaxf(m, part[b]);
  *s = m > 0.f ? m : 1.f;
}

// a0 = bf16(y / s).
__global__ void k_prep_input(const float* __restrict__ y, const float* __restrict__ s, bf16* __restrict__ a0,
                             long long n) {
  const float inv = 1.0f / *s;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    a0[i] = __float2bfloat16_rn(y[i] * inv);
}

struct KernelWeights {
  float* w1;    // [27][32] (tap, co), bfloat16 values
  float* b1;    // [32]
  bf16* wf;     // [4][27][32 co][32 ci]   forward operands of layers 2..5
  bf16* wb;     // [4][27][32 ci][32 co]   flipped, transposed: input gradients
  float* bm;    // [4][32]
  float* w6f;   // [27][32 ci][K]  last layer, forward; bfloat16 values
  float* w6b;   // [27][K][32 ci]  last layer, input gradient
  bf16* w6t;    // [27][16 co][32 ci]  last layer, tcgen05 operand (rows K .. 15 zero)
  float* b6;    // [K]
};

__device__ __forceinline__ float round_bf16(float v) { return __bfloat162float(__float2bfloat16_rn(v)); }

// Packed float32 parameters -> the layouts the kernels read.
__global__ void k_unpack_params(const float* __restrict__ theta, KernelWeights kw, int K) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  constexpr int L1 = NTAP * C + C;           // 896
  constexpr int LM = WMID + C;               // 27680
  const int N = L1 + 4 * LM + K * NTAP * C + K;
  if (i >= N) return;
  const float v = theta[i];
  if (i < L1) {
    if (i < NTAP * C) kw.w1[(i % NTAP) * C + i / NTAP] = round_bf16(v);
    else kw.b1[i - NTAP * C] = v;
    return;
  }
  int j = i - L1;
  if (j < 4 * LM) {
    const int l = j / LM, li = j % LM;
    if (li < WMID) {
      const int co = li / (C * NTAP), rem = li % (C * NTAP), ci = rem / NTAP, t = rem % NTAP;
      const bf16 q = __float2bfloat16_rn(v);
      kw.wf[(size_t)l * WMID + (t * C + co) * C + ci] = q;
      kw.wb[(size_t)l * WMID + ((NTAP - 1 - t) * C + ci) * C + co] = q;
    } else {
      kw.bm[l * C + li - WMID] = v;
    }
    return;
  }
  j -= 4 * LM;
  if (j < K * NTAP * C) {
    const int k = j / (C * NTAP), rem = j % (C * NTAP), ci = rem / NTAP, t = rem % NTAP;
    const float r = round_bf16(v);
    kw.w6f[(t * C + ci) * K + k] = r;
    kw.w6b[(t * K + k) * C + ci] = r;
    kw.w6t[(t * kLastN + k) * C + ci] = __float2bfloat16_rn(v);
  } else {
    kw.b6[j - K * NTAP * C] = v;
  }
}

// One 32 -> 32 layer's weights [co][ci][27] float32 -> forward ([27][co][ci])
// or input-gradient ([27 flipped][ci][co]) bfloat16 operands.
__global__ void k_pack_layer(const float* __restrict__ w, bf16* __restrict__ out, int backward) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= WMID) return;
  const int co = i / (C * NTAP), rem = i % (C * NTAP), ci = rem / NTAP, t = rem % NTAP;
  const bf16 q = __float2bfloat16_rn(w[i]);
  if (backward) out[((NTAP - 1 - t) * C + ci) * C + co] = q;
  else out[(t * C + co) * C + ci] = q;
}

// Adam (Kingma and Ba 2015, Algorithm 1); c1 = 1/(1 - beta1^t), c2 = 1/(1 - beta2^t).
__global__ void k_adam(float* __restrict__ theta, const float* __restrict__ g, float* __restrict__ m,
                       float* __restrict__ v, int n, float lr, float c1, float c2) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  // a layer of this step (or an unchecked earlier call) gave up a wait: its
  // gradient is incomplete, so the step is dropped; muffin_net_check reports it
  if (*(volatile int*)&g_tc_timeouts != 0) return;
  const float gi = g[i];
  const float mi = 0.9f * m[i] + 0.1f * gi;
  const float vi = 0.999f * v[i] + 0.001f * gi * gi;
  m[i] = mi;
  v[i] = vi;
  theta[i] -= lr * (mi * c1) / (sqrtf(vi * c2) + 1e-8f);
}

// ------------------------------------------------------------------ host side

constexpr int kFixedParams = NTAP * C + C + 4 * (WMID + C);   // layers 1..5

int param_count(int K) { return kFixedParams + K * (NTAP * C + 1); }

int w_offset(int k) {  // packed offset of layer k's weights (k = 0..5)
  if (k == 0) return 0;
  return NTAP * C + C + (k - 1) * (WMID + C);
}
int b_offset(int k, int K) {
  const int co = k == 5 ? K : C, ci = k == 0 ? 1 : C;
  return w_offset(k) + co * ci * NTAP;
}

inline size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

bool dims_ok(int nz, int ny, int nx) {
  if (nz < 1 || ny < 1 || nx < 1) return false;
  const long long v = (long long)nz * ny * nx;
  return v < (1LL << 31) / C;
}

int part_slots(const Dims& d) { return d.ntiles < kMaxPart ? d.ntiles : kMaxPart; }
int loss_slots(const Dims& d) { return d.ntiles < kMaxLossPart ? d.ntiles : kMaxLossPart; }

int sm_count() {
  int dev = 0, n = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return 148;
  if (cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || n <= 0) return 148;
  return n;
}

constexpr int last_bwd_smem(int K) { return K * (NTAP * C + HV) * 4; }
constexpr int wgrad_last_smem(int K) { return HV * ROWB + TV * K * 4; }

template <int K>
cudaError_t configure_last() {
  cudaError_t e;
  if ((e = muffin::allow_max_dyn_smem(k_last_bwd_data<K>)) != cudaSuccess) return e;
  return muffin::allow_max_dyn_smem(k_wgrad_last<K>);
}

#define MNET_SWITCH_K(K, EXPR)     \
  switch (K) {                     \
    case 1: { constexpr int KK = 1; EXPR; } break; \
    case 2: { constexpr int KK = 2; EXPR; } break; \
    case 3: { constexpr int KK = 3; EXPR; } break; \
    case 4: { constexpr int KK = 4; EXPR; } break; \
    case 5: { constexpr int KK = 5; EXPR; } break; \
    case 6: { constexpr int KK = 6; EXPR; } break; \
    case 7: { constexpr int KK = 7; EXPR; } break; \
    case 8: { constexpr int KK = 8; EXPR; } break; \
    default: break;                \
  }

cudaError_t configure_once(int K) {
  static bool mid_done = false;
  static cudaError_t mid_err = cudaSuccess;
  static bool last_done[kMaxOut + 1] = {};
  static cudaError_t last_err[kMaxOut + 1] = {};
  if (!mid_done) {
    mid_done = true;
    if ((mid_err = muffin::allow_max_dyn_smem(k_conv_tc05<EPI_RELU>)) == cudaSuccess &&
        (mid_err = muffin::allow_max_dyn_smem(k_conv_tc05<EPI_BIAS>)) == cudaSuccess &&
        (mid_err = muffin::allow_max_dyn_smem(k_conv_tc05<EPI_MASK>)) == cudaSuccess &&
        (mid_err = muffin::allow_max_dyn_smem(k_conv_tc05<EPI_PRED>)) == cudaSuccess &&
        (mid_err = muffin::allow_max_dyn_smem(k_conv_tc05<EPI_LOSS>)) == cudaSuccess)
      mid_err = muffin::allow_max_dyn_smem(k_wgrad_tc05);
  }
  if (mid_err != cudaSuccess) return mid_err;
  if (K < 1 || K > kMaxOut) return cudaSuccess;
  if (!last_done[K]) {
    last_done[K] = true;
    MNET_SWITCH_K(K, last_err[K] = configure_last<KK>());
  }
  return last_err[K];
}

// Launch helpers (all persistent: grids bounded by the tile count).
typedef CUresult (*EncodeTiledFn)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                  const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                  CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

EncodeTiledFn encode_tiled() {
  static EncodeTiledFn fn = nullptr;
  static bool tried = false;
  if (!tried) {
    tried = true;
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
            cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<EncodeTiledFn>(p);
  }
  return fn;
}

// The four 4-D tensor maps (8 features, x, y, z) of a [z][y][x][32] bfloat16 map, one per chunk.
cudaError_t halo_maps(const bf16* in, const Dims& d, HaloMaps* maps) {
  EncodeTiledFn enc = encode_tiled();
  if (!enc) return cudaErrorNotSupported;
  const cuuint64_t dims[4] = {8, (cuuint64_t)d.nx, (cuuint64_t)d.ny, (cuuint64_t)d.nz};
  const cuuint64_t strides[3] = {(cuuint64_t)C * 2, (cuuint64_t)d.nx * C * 2, (cuuint64_t)d.ny * d.nx * C * 2};
  const cuuint32_t box[4] = {8, U_HX, U_HY, 3};
  const cuuint32_t estr[4] = {1, 1, 1, 1};
  for (int c = 0; c < 4; ++c) {
    const CUresult r = enc(&maps->m[c], CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 4, (void*)(in + c * 8), dims, strides,
                           box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                           CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) return cudaErrorInvalidValue;
  }
  return cudaSuccess;
}

// A host-side failure of a layer launch (a tensor map that could not be
// encoded), reported by the next status check of the calling entry point.
cudaError_t g_launch_err = cudaSuccess;

cudaError_t take_launch_error() {
  const cudaError_t e = g_launch_err;
  g_launch_err = cudaSuccess;
  return e != cudaSuccess ? e : cudaGetLastError();
}

// Tiles of 128 voxels and the persistent grid of k_conv_tc05 (two CTAs per SM).
int tc05_tiles(const Dims& d, int& tx, int& ty) {
  tx = (d.nx + U_TX - 1) / U_TX;
  ty = (d.ny + U_TY - 1) / U_TY;
  return tx * ty * d.nz;
}
int tc05_grid(const Dims& d, int sms) {
  int tx, ty;
  int g = tc05_tiles(d, tx, ty);
  if (g > 2 * sms) g = 2 * sms;
  return g < kMaxLossPart ? g : kMaxLossPart;   // also the last layer's loss partial slots
}

template <int EPI>
cudaError_t launch_tc05(const bf16* in, const bf16* wk, const float* bias, const bf16* mask, bf16* out,
                        const Dims& d, int sms, cudaStream_t st, const LastArgs& la) {
  HaloMaps maps;
  const cudaError_t e = halo_maps(in, d, &maps);
  if (e != cudaSuccess) {
    g_launch_err = e;
    return e;
  }
  int tx, ty;
  const int ntiles = tc05_tiles(d, tx, ty);
  k_conv_tc05<EPI><<<tc05_grid(d, sms), 128, conv05_smem(epi_n<EPI>()), st>>>(maps, wk, bias, mask, out, d, tx, ty,
                                                                             ntiles, la);
  return cudaGetLastError();
}

cudaError_t launch_conv(int epi, const bf16* in, const bf16* wk, const float* bias, const bf16* mask, bf16* out,
                        const Dims& d, int sms, cudaStream_t st) {
  const LastArgs none{};
  if (epi == EPI_RELU) return launch_tc05<EPI_RELU>(in, wk, bias, mask, out, d, sms, st, none);
  if (epi == EPI_BIAS) return launch_tc05<EPI_BIAS>(in, wk, bias, mask, out, d, sms, st, none);
  return launch_tc05<EPI_MASK>(in, wk, bias, mask, out, d, sms, st, none);
}

// The two 5-D tensor maps of k_wgrad_tc05 over [z][y][x][32] bfloat16 maps.
cudaError_t wgrad_maps(const bf16* a, const bf16* dz, const Dims& d, WgradMaps* maps) {
  EncodeTiledFn enc = encode_tiled();
  if (!enc) return cudaErrorNotSupported;
  const cuuint64_t row = (cuuint64_t)C * 2, line = row * d.nx, plane = line * d.ny;
  const cuuint32_t estr[5] = {1, 1, 1, 1, 1};
  {
    const cuuint64_t dims[5] = {8, (cuuint64_t)d.nx, (cuuint64_t)d.nz, 4, (cuuint64_t)d.ny};
    const cuuint64_t strides[4] = {row, plane, 16, line};
    const cuuint32_t box[5] = {8, U_HX, 3, 4, WG_HY};
    if (enc(&maps->a, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 5, (void*)a, dims, strides, box, estr,
            CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
            CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
      return cudaErrorInvalidValue;
  }
  {
    const cuuint64_t dims[5] = {8, (cuuint64_t)d.nx, 4, (cuuint64_t)d.ny, (cuuint64_t)d.nz};
    const cuuint64_t strides[4] = {row, 16, line, plane};
    const cuuint32_t box[5] = {8, U_TX, 4, U_TY, 1};
    if (enc(&maps->dz, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 5, (void*)dz, dims, strides, box, estr,
            CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
            CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
      return cudaErrorInvalidValue;
  }
  return cudaSuccess;
}

// Weight and bias gradients of a 32 -> 32 layer: per-CTA partial sums (one
// CTA per SM, at most part_slots(d) of them), then fixed-order reductions.
void launch_wgrad_mid(const bf16* a, const bf16* dz, float* part, float* bpart, float* dw, float* db, const Dims& d,
                      int sms, cudaStream_t st) {
  WgradMaps maps;
  const cudaError_t e = wgrad_maps(a, dz, d, &maps);
  if (e != cudaSuccess) {
    g_launch_err = e;
    return;
  }
  int tx, ty;
  const int ntiles = tc05_tiles(d, tx, ty);
  int P = part_slots(d);
  if (P > sms) P = sms;
  if (P > ntiles) P = ntiles;
  k_wgrad_tc05<<<P, 128, wgrad05_smem, st>>>(maps, part, bpart, d, tx, ty, ntiles);
  k_reduce_part<<<(WMID + 255) / 256, 256, 0, st>>>(part, P, WMID, dw, MAP_MID, 1);
  if (db) k_reduce_part<<<1, 32, 0, st>>>(bpart, P, C, db, MAP_PLAIN, 1);
}

}  // namespace mnet

using namespace mnet;

// ====================================================================== network context

struct muffin_net {
  int training = 0;
  int K = 1;          // output maps
  Lam lam{};
  Dims d{};
  cudaStream_t st = nullptr;
  int sms = 148;
  long long step = 0;
  std::string err;
  // parameters and optimiser
  float *theta = nullptr, *mom1 = nullptr, *mom2 = nullptr, *grad = nullptr;
  KernelWeights kw{};
  // scalars and partials
  float* s = nullptr;
  float* mpart = nullptr;
  double* lpart = nullptr;
  double* loss = nullptr;
  float* part = nullptr;
  float* bpart = nullptr;
  // maps
  bf16* a0 = nullptr;
  bf16* act = nullptr;   // training: a1..a5; inference: two ping-pong maps
  bf16* gA = nullptr;
  bf16* gB = nullptr;
  float* d6 = nullptr;   // [V][K]

  bf16* map(int i) const { return act + (size_t)i * d.nvox * C; }
};

namespace {

// Workspace carve-up; with base == nullptr only the size is computed.
size_t net_layout(muffin_net* n, const Dims& d, int K, int training, char* base) {
  size_t off = 0;
  auto take = [&](size_t bytes) -> char* {
    char* p = base ? base + off : nullptr;
    off = align256(off + bytes);
    return p;
  };
  const int np = param_count(K);
  const size_t V = (size_t)d.nvox;
  float* theta = (float*)take(np * 4);
  float* m1 = (float*)take(training ? np * 4 : 0);
  float* m2 = (float*)take(training ? np * 4 : 0);
  float* grad = (float*)take(training ? np * 4 : 0);
  KernelWeights kw;
  kw.w1 = (float*)take(NTAP * C * 4);
  kw.b1 = (float*)take(C * 4);
  kw.wf = (bf16*)take(4 * WMID * 2);
  kw.wb = (bf16*)take(4 * WMID * 2);
  kw.bm = (float*)take(4 * C * 4);
  kw.w6f = (float*)take(NTAP * C * K * 4);
  kw.w6b = (float*)take(NTAP * C * K * 4);
  kw.w6t = (bf16*)take(NTAP * kLastN * C * 2);
  kw.b6 = (float*)take(K * 4);
  float* s = (float*)take(4);
  float* mpart = (float*)take(kMaxLossPart * 4);
  double* lpart = (double*)take((size_t)(K + 1) * kMaxLossPart * 8);
  double* loss = (double*)take(8);
  const int P = part_slots(d);
  float* part = (float*)take(training ? (size_t)P * WMID * 4 : 0);
  float* bpart = (float*)take(training ? (size_t)P * C * 4 : 0);
  bf16* a0 = (bf16*)take(V * 2);
  bf16* act = (bf16*)take((training ? 5 : 2) * V * C * 2);
  bf16* gA = (bf16*)take(training ? V * C * 2 : 0);
  bf16* gB = (bf16*)take(training ? V * C * 2 : 0);
  float* d6 = (float*)take(training ? V * K * 4 : 0);
  if (n) {
    n->theta = theta; n->mom1 = m1; n->mom2 = m2; n->grad = grad; n->kw = kw;
    n->s = s; n->mpart = mpart; n->lpart = lpart; n->loss = loss; n->part = part; n->bpart = bpart;
    n->a0 = a0; n->act = act; n->gA = gA; n->gB = gB; n->d6 = d6;
  }
  return off;
}

int fail(muffin_net* n, int code, const std::string& msg) {
  if (n) n->err = msg;
  return code;
}

int cuda_check(muffin_net* n, const char* what) {
  const cudaError_t e = take_launch_error();
  if (e != cudaSuccess) return fail(n, MUFFIN_ERR_CUDA, std::string(what) + ": " + cudaGetErrorString(e));
  return MUFFIN_OK;
}

// s, a0 and the forward pass through layer 5 (training keeps every map).
void forward_to_a5(muffin_net* n, const float* y) {
  const Dims& d = n->d;
  const int PL = loss_slots(d);
  const int grid_s = (int)((d.nvox + 255) / 256 < PL ? (d.nvox + 255) / 256 : PL);
  k_maxabs_part<<<grid_s, 256, 0, n->st>>>(y, d.nvox, n->mpart);
  k_scale_final<<<1, 32, 0, n->st>>>(n->mpart, grid_s, n->s);
  const int grid_p = (int)((d.nvox + 255) / 256 < 4 * n->sms ? (d.nvox + 255) / 256 : 4 * n->sms);
  k_prep_input<<<grid_p, 256, 0, n->st>>>(y, n->s, n->a0, d.nvox);
  const int gsimt = d.ntiles < 4 * n->sms ? d.ntiles : 4 * n->sms;
  bf16* out = n->map(0);
  k_first_fwd<<<gsimt, 256, 0, n->st>>>(n->a0, n->kw.w1, n->kw.b1, out, d);
  for (int l = 0; l < 4; ++l) {
    bf16* in = out;
    out = n->training ? n->map(l + 1) : n->map((l + 1) & 1);
    launch_conv(EPI_RELU, in, n->kw.wf + (size_t)l * WMID, n->kw.bm + l * C, nullptr, out, d, n->sms, n->st);
  }
}

bf16* a5_of(muffin_net* n) { return n->training ? n->map(4) : n->map(0); }

LastArgs last_args(muffin_net* n) {
  LastArgs la{};
  la.K = n->K;
  la.lam = n->lam;
  la.s = n->s;
  return la;
}

void last_predict(muffin_net* n, float* x, float* aux) {
  LastArgs la = last_args(n);
  la.out_x = x;
  la.out_aux = aux;
  launch_tc05<EPI_PRED>(a5_of(n), n->kw.w6t, n->kw.b6, nullptr, nullptr, n->d, n->sms, n->st, la);
}

// Last layer of the training pass: loss, d6, its weight and bias gradients,
// and the gradient of a5's pre-activation into g5.
template <int K>
void last_train(muffin_net* n, const float* tx, const bf16* taux, bf16* g5) {
  const Dims& d = n->d;
  bf16* a5 = a5_of(n);
  LastArgs la = last_args(n);
  la.tx = tx;
  la.taux = taux;
  la.d6 = n->d6;
  la.lpart = n->lpart;
  launch_tc05<EPI_LOSS>(a5, n->kw.w6t, n->kw.b6, nullptr, nullptr, d, n->sms, n->st, la);
  k_loss_final<<<1, K + 1, 0, n->st>>>(n->lpart, tc05_grid(d, n->sms), K, n->lam, d.nvox, n->loss,
                                       n->grad + b_offset(5, K));
  int P = part_slots(d);
  if (P > 2 * n->sms) P = 2 * n->sms;
  k_wgrad_last<K><<<P, 288, wgrad_last_smem(K), n->st>>>(n->d6, a5, n->part, d);
  k_reduce_part<<<(NTAP * C * K + 255) / 256, 256, 0, n->st>>>(n->part, P, NTAP * C * K, n->grad + w_offset(5),
                                                               MAP_LAST, K);
  const int gsimt = d.ntiles < 4 * n->sms ? d.ntiles : 4 * n->sms;
  k_last_bwd_data<K><<<gsimt, 256, last_bwd_smem(K), n->st>>>(n->d6, n->kw.w6b, a5, g5, d);
}

// Loss and gradient into n->grad (training contexts).
void loss_and_grad(muffin_net* n, const float* y, const float* tx, const bf16* taux) {
  const Dims& d = n->d;
  forward_to_a5(n, y);
  bf16* g = n->gA;
  bf16* other = n->gB;
  MNET_SWITCH_K(n->K, last_train<KK>(n, tx, taux, g));
  for (int k = 4; k >= 1; --k) {          // layers 5..2 (index k), input map a_k = map(k - 1)
    const bf16* a_in = n->map(k - 1);
    launch_wgrad_mid(a_in, g, n->part, n->bpart, n->grad + w_offset(k), n->grad + b_offset(k, n->K), d, n->sms,
                     n->st);
    launch_conv(EPI_MASK, g, n->kw.wb + (size_t)(k - 1) * WMID, nullptr, a_in, other, d, n->sms, n->st);
    bf16* tmp = g; g = other; other = tmp;
  }
  int P = part_slots(d);
  if (P > 2 * n->sms) P = 2 * n->sms;
  k_wgrad_first<<<P, 288, 0, n->st>>>(n->a0, g, n->part, n->bpart, d);
  k_reduce_part<<<(NTAP * C + 255) / 256, 256, 0, n->st>>>(n->part, P, NTAP * C, n->grad + w_offset(0), MAP_FIRST, 1);
  k_reduce_part<<<1, 32, 0, n->st>>>(n->bpart, P, C, n->grad + b_offset(0, n->K), MAP_PLAIN, 1);
}

void unpack_params(muffin_net* n) {
  const int np = param_count(n->K);
  cudaMemsetAsync(n->kw.w6t, 0, NTAP * kLastN * C * 2, n->st);
  k_unpack_params<<<(np + 255) / 256, 256, 0, n->st>>>(n->theta, n->kw, n->K);
}

}  // namespace

extern "C" {

int muffin_net_num_params(int n_out) {
  if (n_out < 1 || n_out > kMaxOut) return 0;
  return param_count(n_out);
}

size_t muffin_net_workspace_bytes(int nz, int ny, int nx, int n_out, int training) {
  if (!dims_ok(nz, ny, nx) || n_out < 1 || n_out > kMaxOut) return 0;
  return net_layout(nullptr, make_dims(nz, ny, nx), n_out, training != 0, nullptr);
}

int muffin_net_create(muffin_net** out, int nz, int ny, int nx, int n_out, const float* h_out_weight, int training,
                      void* d_ws, size_t ws_bytes, cudaStream_t stream) {
  if (!out) return MUFFIN_ERR_ARG;
  *out = nullptr;
  if (!dims_ok(nz, ny, nx) || n_out < 1 || n_out > kMaxOut) return MUFFIN_ERR_ARG;
  Lam lam;
  for (int k = 0; k < kMaxOut; ++k) lam.v[k] = 1.f;
  if (h_out_weight)
    for (int k = 0; k < n_out; ++k) {
      if (!(h_out_weight[k] >= 0.f) || !std::isfinite(h_out_weight[k])) return MUFFIN_ERR_ARG;
      lam.v[k] = h_out_weight[k];
    }
  if (!d_ws || ((uintptr_t)d_ws & 255)) return MUFFIN_ERR_ARG;
  const Dims d = make_dims(nz, ny, nx);
  const size_t need = net_layout(nullptr, d, n_out, training != 0, nullptr);
  if (ws_bytes < need) return MUFFIN_ERR_NOMEM;
  if (configure_once(n_out) != cudaSuccess) return MUFFIN_ERR_CUDA;
  muffin_net* n = new muffin_net();
  n->training = training != 0;
  n->K = n_out;
  n->lam = lam;
  n->d = d;
  n->st = stream;
  n->sms = sm_count();
  net_layout(n, d, n_out, n->training, (char*)d_ws);
  const int np = param_count(n_out);
  cudaMemsetAsync(n->theta, 0, np * 4, stream);
  if (n->training) {
    cudaMemsetAsync(n->mom1, 0, np * 4, stream);
    cudaMemsetAsync(n->mom2, 0, np * 4, stream);
  }
  unpack_params(n);
  if (cudaGetLastError() != cudaSuccess) {
    delete n;
    return MUFFIN_ERR_CUDA;
  }
  *out = n;
  return MUFFIN_OK;
}

int muffin_net_set_params(muffin_net* n, const float* d_theta) {
  if (!n) return MUFFIN_ERR_ARG;
  if (!d_theta) return fail(n, MUFFIN_ERR_ARG, "d_theta is NULL");
  const int np = param_count(n->K);
  cudaMemcpyAsync(n->theta, d_theta, np * 4, cudaMemcpyDeviceToDevice, n->st);
  if (n->training) {
    cudaMemsetAsync(n->mom1, 0, np * 4, n->st);
    cudaMemsetAsync(n->mom2, 0, np * 4, n->st);
  }
  n->step = 0;
  unpack_params(n);
  return cuda_check(n, "muffin_net_set_params");
}

int muffin_net_get_params(const muffin_net* n, float* d_theta) {
  if (!n || !d_theta) return MUFFIN_ERR_ARG;
  cudaMemcpyAsync(d_theta, n->theta, param_count(n->K) * 4, cudaMemcpyDeviceToDevice, n->st);
  return cuda_check(const_cast<muffin_net*>(n), "muffin_net_get_params");
}

// Synchronise the context's stream, then read and clear the device's count of
// tensor-core waits that gave up; MUFFIN_ERR_TIMEOUT if it was not zero.
static int check_waits(muffin_net* n, const char* what) {
  cudaError_t e = cudaStreamSynchronize(n->st);
  if (e != cudaSuccess) return fail(n, MUFFIN_ERR_CUDA, std::string(what) + ": " + cudaGetErrorString(e));
  int v = 0, zero = 0;
  if ((e = cudaMemcpyFromSymbol(&v, g_tc_timeouts, sizeof(int))) != cudaSuccess ||
      (e = cudaMemcpyToSymbol(g_tc_timeouts, &zero, sizeof(int))) != cudaSuccess)
    return fail(n, MUFFIN_ERR_CUDA, std::string(what) + ": " + cudaGetErrorString(e));
  if (v != 0)
    return fail(n, MUFFIN_ERR_TIMEOUT, std::string(what) + ": " + std::to_string(v) +
                                           " thread block(s) of the tensor-core layers gave up a bounded wait; "
                                           "their output tiles (and any Adam step queued after them) were skipped");
  return MUFFIN_OK;
}

int muffin_net_predict(muffin_net* n, const float* d_dirty, float* d_x, float* d_aux) {
  if (!n) return MUFFIN_ERR_ARG;
  if (!d_dirty || !d_x) return fail(n, MUFFIN_ERR_ARG, "NULL cube pointer");
  if (n->K > 1 && !d_aux) return fail(n, MUFFIN_ERR_ARG, "NULL d_aux with more than one output map");
  forward_to_a5(n, d_dirty);
  last_predict(n, d_x, d_aux);
  const int r = cuda_check(n, "muffin_net_predict");
  if (r != MUFFIN_OK) return r;
  return check_waits(n, "muffin_net_predict");
}

int muffin_net_check(muffin_net* n) {
  if (!n) return MUFFIN_ERR_ARG;
  const int r = cuda_check(n, "muffin_net_check");
  if (r != MUFFIN_OK) return r;
  return check_waits(n, "muffin_net_check");
}

int muffin_net_set_wait_limit(long long polls) {
  const long long v = polls < 0 ? kWaitLimit : polls;
  return cudaMemcpyToSymbol(g_wait_polls, &v, sizeof(v)) == cudaSuccess ? MUFFIN_OK : MUFFIN_ERR_CUDA;
}

static int check_targets(muffin_net* n, const float* d_dirty, const float* d_tx, const void* d_taux) {
  if (!n->training) return fail(n, MUFFIN_ERR_STATE, "not a training context");
  if (!d_dirty || !d_tx) return fail(n, MUFFIN_ERR_ARG, "NULL pointer");
  if (n->K > 1 && !d_taux) return fail(n, MUFFIN_ERR_ARG, "NULL d_target_aux with more than one output map");
  return MUFFIN_OK;
}

int muffin_net_loss_grad(muffin_net* n, const float* d_dirty, const float* d_tx, const void* d_taux, float* d_grad,
                         double* h_loss) {
  if (!n) return MUFFIN_ERR_ARG;
  int r = check_targets(n, d_dirty, d_tx, d_taux);
  if (r != MUFFIN_OK) return r;
  if (!d_grad) return fail(n, MUFFIN_ERR_ARG, "NULL d_grad");
  loss_and_grad(n, d_dirty, d_tx, (const bf16*)d_taux);
  cudaMemcpyAsync(d_grad, n->grad, param_count(n->K) * 4, cudaMemcpyDeviceToDevice, n->st);
  r = cuda_check(n, "muffin_net_loss_grad");
  if (r != MUFFIN_OK) return r;
  if (h_loss) {
    cudaMemcpyAsync(h_loss, n->loss, 8, cudaMemcpyDeviceToHost, n->st);
    return check_waits(n, "muffin_net_loss_grad");
  }
  return MUFFIN_OK;
}

int muffin_net_train_step(muffin_net* n, const float* d_dirty, const float* d_tx, const void* d_taux, float lr,
                          double* d_loss) {
  if (!n) return MUFFIN_ERR_ARG;
  int r = check_targets(n, d_dirty, d_tx, d_taux);
  if (r != MUFFIN_OK) return r;
  if (!(lr >= 0.f) || !std::isfinite(lr)) return fail(n, MUFFIN_ERR_ARG, "learning rate must be finite and >= 0");
  loss_and_grad(n, d_dirty, d_tx, (const bf16*)d_taux);
  if (d_loss) cudaMemcpyAsync(d_loss, n->loss, 8, cudaMemcpyDeviceToDevice, n->st);
  n->step += 1;
  const double c1 = 1.0 / (1.0 - std::pow(0.9, (double)n->step));
  const double c2 = 1.0 / (1.0 - std::pow(0.999, (double)n->step));
  const int np = param_count(n->K);
  k_adam<<<(np + 255) / 256, 256, 0, n->st>>>(n->theta, n->grad, n->mom1, n->mom2, np, lr, (float)c1, (float)c2);
  unpack_params(n);
  return cuda_check(n, "muffin_net_train_step");
}

int muffin_net_wait_timeouts(void) {
  int v = 0, zero = 0;
  if (cudaMemcpyFromSymbol(&v, g_tc_timeouts, sizeof(int)) != cudaSuccess) return -1;
  if (cudaMemcpyToSymbol(g_tc_timeouts, &zero, sizeof(int)) != cudaSuccess) return -1;
  return v;
}

const char* muffin_net_last_error(const muffin_net* n) {
  if (!n) return "invalid arguments to muffin_net_create (sizes, output maps, weights, workspace) or CUDA set-up failed";
  return n->err.c_str();
}

void muffin_net_destroy(muffin_net* n) { delete n; }

// ---------------------------------------------------------------------- single layers

static thread_local std::string g_conv_err;

static int conv_fail(int code, const std::string& msg) {
  g_conv_err = msg;
  return code;
}

static int conv_cuda(const char* what) {
  const cudaError_t e = take_launch_error();
  if (e != cudaSuccess) return conv_fail(MUFFIN_ERR_CUDA, std::string(what) + ": " + cudaGetErrorString(e));
  return MUFFIN_OK;
}

static bool aligned16(const void* p) { return ((uintptr_t)p & 15) == 0; }

size_t muffin_conv3d_scratch_bytes(int nz, int ny, int nx) {
  if (!dims_ok(nz, ny, nx)) return 0;
  const Dims d = make_dims(nz, ny, nx);
  const int P = part_slots(d);
  return align256(WMID * 2) + align256((size_t)P * WMID * 4) + align256((size_t)P * C * 4);
}

static int layer_args(const void* a, const void* b, int nz, int ny, int nx, void* scratch, size_t bytes) {
  if (!dims_ok(nz, ny, nx)) return conv_fail(MUFFIN_ERR_ARG, "sizes must be >= 1 with nz*ny*nx*32 < 2^31");
  if (!a || !b || !scratch) return conv_fail(MUFFIN_ERR_ARG, "NULL pointer");
  if (!aligned16(a) || !aligned16(b) || ((uintptr_t)scratch & 255))
    return conv_fail(MUFFIN_ERR_ARG, "maps must be 16-byte aligned, scratch 256-byte aligned");
  if (bytes < muffin_conv3d_scratch_bytes(nz, ny, nx)) return conv_fail(MUFFIN_ERR_NOMEM, "scratch too small");
  if (configure_once(0) != cudaSuccess) return conv_fail(MUFFIN_ERR_CUDA, "kernel attributes could not be set");
  return MUFFIN_OK;
}

int muffin_conv3d_forward(const void* d_a, const float* d_w, const float* d_b, int relu, void* d_z, int nz, int ny,
                          int nx, void* d_scratch, size_t scratch_bytes, cudaStream_t stream) {
  int r = layer_args(d_a, d_z, nz, ny, nx, d_scratch, scratch_bytes);
  if (r != MUFFIN_OK) return r;
  if (!d_w) return conv_fail(MUFFIN_ERR_ARG, "NULL weights");
  const Dims d = make_dims(nz, ny, nx);
  bf16* wk = (bf16*)d_scratch;
  k_pack_layer<<<(WMID + 255) / 256, 256, 0, stream>>>(d_w, wk, 0);
  launch_conv(relu ? EPI_RELU : EPI_BIAS, (const bf16*)d_a, wk, d_b, nullptr, (bf16*)d_z, d, sm_count(), stream);
  return conv_cuda("muffin_conv3d_forward");
}

int muffin_conv3d_backward_data(const void* d_dz, const float* d_w, const void* d_mask, void* d_da, int nz, int ny,
                                int nx, void* d_scratch, size_t scratch_bytes, cudaStream_t stream) {
  int r = layer_args(d_dz, d_da, nz, ny, nx, d_scratch, scratch_bytes);
  if (r != MUFFIN_OK) return r;
  if (!d_w) return conv_fail(MUFFIN_ERR_ARG, "NULL weights");
  if (d_mask && !aligned16(d_mask)) return conv_fail(MUFFIN_ERR_ARG, "mask must be 16-byte aligned");
  const Dims d = make_dims(nz, ny, nx);
  bf16* wk = (bf16*)d_scratch;
  k_pack_layer<<<(WMID + 255) / 256, 256, 0, stream>>>(d_w, wk, 1);
  launch_conv(EPI_MASK, (const bf16*)d_dz, wk, nullptr, (const bf16*)d_mask, (bf16*)d_da, d, sm_count(), stream);
  return conv_cuda("muffin_conv3d_backward_data");
}

int muffin_conv3d_backward_weights(const void* d_a, const void* d_dz, float* d_dw, float* d_db, int nz, int ny,
                                   int nx, void* d_scratch, size_t scratch_bytes, cudaStream_t stream) {
  int r = layer_args(d_a, d_dz, nz, ny, nx, d_scratch, scratch_bytes);
  if (r != MUFFIN_OK) return r;
  if (!d_dw) return conv_fail(MUFFIN_ERR_ARG, "NULL weight gradient");
  const Dims d = make_dims(nz, ny, nx);
  char* base = (char*)d_scratch + align256(WMID * 2);
  const int P = part_slots(d);
  float* part = (float*)base;
  float* bpart = (float*)(base + align256((size_t)P * WMID * 4));
  launch_wgrad_mid((const bf16*)d_a, (const bf16*)d_dz, part, bpart, d_dw, d_db, d, sm_count(), stream);
  return conv_cuda("muffin_conv3d_backward_weights");
}

const char* muffin_conv3d_last_error(void) { return g_conv_err.c_str(); }

}  // extern "C"
