// Spectral transform W_lambda (orthonormal DCT-II along the channel axis at
// every pixel, Eq. 6) fused with the spectral dual step of Algorithm 1 (fourth
// line; Eq. 13):  V <- rho sat(V + sigma mu_lambda DCT(D)) + (1 - rho) V, and
// with the spectral adjoint of the next pass: T = W_lambda^T V = DCT^-1(V)
// (first step of the master node in Sec. 3, computed here per pixel).
//
// One block handles 32 consecutive pixels (one per lane) and all L channels;
// reads and writes of D, V and T are coalesced along the pixels.
//  * L a power of two in [16, 256]: Makhoul's O(L log L) DCT (reorder x -> v
//    with v[m] = x[2m], v[L-1-m] = x[2m+1]; DCT[k] = Re(exp(-i pi k / 2L)
//    FFT(v)[k]); the inverse runs the same steps backwards), the real FFT of
//    length L done as one complex FFT of length L/2.  Warp w is FFT thread w
//    of all 32 transforms.
//  * other L (<= 512): the dense orthonormal DCT matrix.
#include <cuda.h>   // CUtensorMap (the encoder is reached through the runtime's driver entry point)

#include "device.cuh"
#include "internal.h"
#include "spectral_blocks.cuh"

namespace muffin {

bool spectral_uses_fft(int L) { return L >= 16 && L <= 256 && (L & (L - 1)) == 0; }


// Power-of-two L: the reordered sequence v is real, so its length-L FFT comes
// from one length-L/2 complex FFT of z[m] = v[2m] + i v[2m+1] (even/odd
// split: V[k] = E[k] + w^k O[k], V[k + L/2] = E[k] - w^k O[k], w = e^{-2 pi i/L},
// E and O recovered from Z[k] and conj Z[L/2 - k]); the inverse runs the same
// split backwards.  Thread (lane, t) owns coefficients k and k + L/2 for
// k = t + q L/16, q < 8.
template <int L, int MODE>
__global__ void __launch_bounds__(2 * L, 2)
k_spectral_fft(SpecArgs a, int npix) {
  constexpr int H = L / 2, T16 = L / 16;
  extern __shared__ __align__(16) unsigned char smraw[];
  cpx<float>* work = reinterpret_cast<cpx<float>*>(smraw);        // [H][32]
  float* vb = reinterpret_cast<float*>(work + H * 32);            // [L][32]
  cpx<float>* twh = reinterpret_cast<cpx<float>*>(vb + L * 32);   // [H], e^{-2 pi i m / H}
  __shared__ double red[32];
  const cpx<float>* twl = reinterpret_cast<const cpx<float>*>(a.tw);   // e^{-2 pi i m / L}
  const cpx<float>* post = reinterpret_cast<const cpx<float>*>(a.post);
  const cpx<float>* pre = reinterpret_cast<const cpx<float>*>(a.pre);
  const int lane = threadIdx.x, t = threadIdx.y;
  const int tid = t * 32 + lane, nth = 32 * T16;
  for (int i = tid; i < H; i += nth) twh[i] = twl[2 * i];
  const int pix = blockIdx.x * 32 + lane;
  const bool ok = pix < npix;
  const size_t P = (size_t)npix;
  cpx<float> z[8];
  double acc = 0.0;
  if constexpr (MODE != SPEC_TONLY) {
    float vold[16];
#pragma unroll
    for (int q = 0; q < 8; ++q) {
      const int m = t + q * T16;
      z[q] = ok ? mk<float>(__ldg(a.D + (size_t)makhoul_src(2 * m, L) * P + pix),
                            __ldg(a.D + (size_t)makhoul_src(2 * m + 1, L) * P + pix))
                : mk<float>(0.0f, 0.0f);
    }
    __syncthreads();
    fft_regs<float, H, -1, 32>(z, work + lane, twh, t);
    // the old duals arrive while the spectrum is exchanged through shared memory
    if constexpr (MODE == SPEC_UPDATE) {
#pragma unroll
      for (int q = 0; q < 8; ++q) {
        const int m = t + q * T16;
        vold[q] = ok ? a.V[(size_t)m * P + pix] : 0.0f;
        vold[q + 8] = ok ? a.V[(size_t)(m + H) * P + pix] : 0.0f;
      }
    }
    __syncthreads();
#pragma unroll
    for (int q = 0; q < 8; ++q) work[(t + q * T16) * 32 + lane] = z[q];
    __syncthreads();
#pragma unroll
    for (int q = 0; q < 8; ++q) {
      const int k = t + q * T16;
      const cpx<float> zk = z[q], zm = conj(work[((H - k) & (H - 1)) * 32 + lane]);
      const cpx<float> e = scale(add(zk, zm), 0.5f);
      const cpx<float> d = sub(zk, zm);
      const cpx<float> o = mk<float>(0.5f * d.y, -0.5f * d.x);      // (zk - zm) / 2i
      const cpx<float> wo = mul(twl[k], o);
      const cpx<float> v0 = add(e, wo), v1 = sub(e, wo);
      const cpx<float> p0 = post[k], p1 = post[k + H];
      const float c0 = p0.x * v0.x - p0.y * v0.y, c1 = p1.x * v1.x - p1.y * v1.y;
      if constexpr (MODE == SPEC_NORM) {
        acc += fabs((double)c0) + fabs((double)c1);
      } else {
        const float n0 = a.rho * sat1(vold[q] + a.k * c0) + (1.0f - a.rho) * vold[q];
        const float n1 = a.rho * sat1(vold[q + 8] + a.k * c1) + (1.0f - a.rho) * vold[q + 8];
        if (ok) {
          a.V[(size_t)k * P + pix] = n0;
          a.V[(size_t)(k + H) * P + pix] = n1;
        }
        vb[k * 32 + lane] = ok ? n0 * a.invs[k] : 0.0f;
        vb[(k + H) * 32 + lane] = ok ? n1 * a.invs[k + H] : 0.0f;
      }
    }
    if constexpr (MODE == SPEC_NORM) {
      const double tot = block_sum(acc, red);
      if (tid == 0) a.partials[blockIdx.x] = tot;
      return;
    }
  } else {
#pragma unroll
    for (int q = 0; q < 8; ++q) {
      const int k = t + q * T16;
      vb[k * 32 + lane] = ok ? __ldg(a.V + (size_t)k * P + pix) * a.invs[k] : 0.0f;
      vb[(k + H) * 32 + lane] = ok ? __ldg(a.V + (size_t)(k + H) * P + pix) * a.invs[k + H] : 0.0f;
    }
  }
  __syncthreads();
  // inverse: W[k] = pre[k] (y[k] - i y[L-k]) with y[L] = 0, folded to half length
#pragma unroll
  for (int q = 0; q < 8; ++q) {
    const int k = t + q * T16;
    const float ya = vb[k * 32 + lane], yb = k == 0 ? 0.0f : vb[(L - k) * 32 + lane];
    const float yc = vb[(k + H) * 32 + lane], yd = vb[(H - k) * 32 + lane];
    const cpx<float> w0 = mul(pre[k], mk<float>(ya, -yb));
    const cpx<float> w1 = mul(pre[k + H], mk<float>(yc, -yd));
    const cpx<float> A = add(w0, w1);
    const cpx<float> B = mul(sub(w0, w1), conj(twl[k]));
    z[q] = mk<float>(A.x - B.y, A.y + B.x);                          // A + i B
  }
  fft_regs<float, H, 1, 32>(z, work + lane, twh, t);
  if (ok) {
#pragma unroll
    for (int q = 0; q < 8; ++q) {
      const int m = t + q * T16;
      a.T[(size_t)makhoul_src(2 * m, L) * P + pix] = z[q].x;
      a.T[(size_t)makhoul_src(2 * m + 1, L) * P + pix] = z[q].y;
    }
  }
}

// ------------------------------------------------------------------ pipelined update (TMA)
// The update pass of the kernel above as a persistent kernel: one block per SM
// walks 32-pixel tiles; the [L][32] tiles of D and V arrive by one 2-D TMA copy
// each into a double buffer, so the next tile's loads run under this tile's
// transforms, and the new V and T leave by TMA stores from the same buffers
// (V in place of the old V, T in place of D).  Every mbarrier wait is bounded:
// a block that gives up records it in g_spec_timeouts, waits (bounded) for
// its copies in flight and returns.
__device__ int g_spec_timeouts;
constexpr long long kSpecPolls = 1LL << 22;

struct SpecMaps {
  CUtensorMap d, v, t;   // [L][P] float32, box [L][32]
};

template <int L> struct SpecTma {
  static constexpr int H = L / 2;
  static constexpr size_t TILE = (size_t)L * 32 * sizeof(float);              // one [L][32] tile
  static constexpr size_t OFF_D = 0, OFF_V = 2 * TILE, OFF_W = 4 * TILE;       // D[2], V[2], work
  static constexpr size_t OFF_TW = OFF_W + (size_t)H * 32 * sizeof(cpx<float>);
  // tables, read every tile: half-length twiddles [H], twiddles, post- and pre-twiddles [L], 1/(s_k L) [L]
  static constexpr size_t OFF_TWL = OFF_TW + (size_t)H * sizeof(cpx<float>);
  static constexpr size_t OFF_POST = OFF_TWL + (size_t)L * sizeof(cpx<float>);
  static constexpr size_t OFF_PRE = OFF_POST + (size_t)L * sizeof(cpx<float>);
  static constexpr size_t OFF_INVS = OFF_PRE + (size_t)L * sizeof(cpx<float>);
  static constexpr size_t OFF_BAR = OFF_INVS + (size_t)L * sizeof(float);
  static constexpr size_t SMEM = OFF_BAR + 64 + 128;                            // + alignment slack
};

template <int L>
__global__ void __launch_bounds__(2 * L, (256 / L) < 1 ? 1 : 256 / L)
k_spectral_tma(const __grid_constant__ SpecMaps maps, SpecArgs a, int ntiles) {
  using G = SpecTma<L>;
  constexpr int H = L / 2, T16 = L / 16;
  extern __shared__ __align__(16) unsigned char smraw[];
  unsigned char* sm = reinterpret_cast<unsigned char*>((reinterpret_cast<uintptr_t>(smraw) + 127) & ~(uintptr_t)127);
  float* Db = reinterpret_cast<float*>(sm + G::OFF_D);
  float* Vb = reinterpret_cast<float*>(sm + G::OFF_V);
  cpx<float>* work = reinterpret_cast<cpx<float>*>(sm + G::OFF_W);
  cpx<float>* twh = reinterpret_cast<cpx<float>*>(sm + G::OFF_TW);
  cpx<float>* twl = reinterpret_cast<cpx<float>*>(sm + G::OFF_TWL);
  cpx<float>* post = reinterpret_cast<cpx<float>*>(sm + G::OFF_POST);
  cpx<float>* pre = reinterpret_cast<cpx<float>*>(sm + G::OFF_PRE);
  float* invs = reinterpret_cast<float*>(sm + G::OFF_INVS);
  const uint32_t bar0 = smem_addr(sm + G::OFF_BAR);
  const int lane = threadIdx.x, t = threadIdx.y;
  const int tid = t * 32 + lane, nth = 32 * T16;
  {
    const cpx<float>* g_tw = reinterpret_cast<const cpx<float>*>(a.tw);
    const cpx<float>* g_post = reinterpret_cast<const cpx<float>*>(a.post);
    const cpx<float>* g_pre = reinterpret_cast<const cpx<float>*>(a.pre);
    for (int i = tid; i < L; i += nth) {
      twl[i] = g_tw[i];
      post[i] = g_post[i];
      pre[i] = g_pre[i];
      invs[i] = a.invs[i];
      if (i < H) twh[i] = g_tw[2 * i];
    }
  }
  constexpr uint32_t kBytes = 2 * (uint32_t)G::TILE;
  // thread 0: which stages have a load in flight (bit s) and its parity (bit s of pend_ph)
  uint32_t pend = 0, pend_ph = 0;
  if (tid == 0) {
    for (int b = 0; b < 2; ++b) asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(bar0 + 8 * b) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    for (int b = 0; b < 2; ++b) {
      const int tile = blockIdx.x + b * gridDim.x;
      if (tile < ntiles) {
        const uint32_t bar = bar0 + 8 * b;
        asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(kBytes) : "memory");
        tma_load2(smem_addr(Db + b * L * 32), &maps.d, tile * 32, 0, bar);
        tma_load2(smem_addr(Vb + b * L * 32), &maps.v, tile * 32, 0, bar);
        pend |= 1u << b;
      }
    }
  }
  __syncthreads();
  bool gave_up = false;
  int it = 0;
  for (int tile = blockIdx.x; tile < ntiles; tile += gridDim.x, ++it) {
    const int s = it & 1;
    const uint32_t ph = (uint32_t)(it >> 1) & 1u;
    const bool ok = mbar_try(bar0 + 8 * s, ph, kSpecPolls);
    if (__syncthreads_or(!ok)) { gave_up = true; break; }
    if (tid == 0) { pend &= ~(1u << s); }
    float* D = Db + s * L * 32;     // [L][32]; becomes T
    float* V = Vb + s * L * 32;     // [L][32]; becomes the new V
    cpx<float> z[8];
#pragma unroll
    for (int q = 0; q < 8; ++q) {
      const int m = t + q * T16;
      z[q] = mk<float>(D[makhoul_src(2 * m, L) * 32 + lane], D[makhoul_src(2 * m + 1, L) * 32 + lane]);
    }
    fft_regs<float, H, -1, 32>(z, work + lane, twh, t);
    __syncthreads();
#pragma unroll
    for (int q = 0; q < 8; ++q) work[(t + q * T16) * 32 + lane] = z[q];
    __syncthreads();
#pragma unroll
    for (int q = 0; q < 8; ++q) {
      const int k = t + q * T16;
      const cpx<float> zk = z[q], zm = conj(work[((H - k) & (H - 1)) * 32 + lane]);
      const cpx<float> e = scale(add(zk, zm), 0.5f);
      const cpx<float> d = sub(zk, zm);
      const cpx<float> o = mk<float>(0.5f * d.y, -0.5f * d.x);
      const cpx<float> wo = mul(twl[k], o);
      const cpx<float> v0 = add(e, wo), v1 = sub(e, wo);
      const cpx<float> p0 = post[k], p1 = post[k + H];
      const float c0 = p0.x * v0.x - p0.y * v0.y, c1 = p1.x * v1.x - p1.y * v1.y;
      const float o0 = V[k * 32 + lane], o1 = V[(k + H) * 32 + lane];
      V[k * 32 + lane] = a.rho * sat1(o0 + a.k * c0) + (1.0f - a.rho) * o0;
      V[(k + H) * 32 + lane] = a.rho * sat1(o1 + a.k * c1) + (1.0f - a.rho) * o1;
    }
    __syncthreads();
#pragma unroll
    for (int q = 0; q < 8; ++q) {
      const int k = t + q * T16;
      const float ya = V[k * 32 + lane] * invs[k];
      const float yb = k == 0 ? 0.0f : V[(L - k) * 32 + lane] * invs[L - k];
      const float yc = V[(k + H) * 32 + lane] * invs[k + H];
      const float yd = V[(H - k) * 32 + lane] * invs[H - k];
      const cpx<float> w0 = mul(pre[k], mk<float>(ya, -yb));
      const cpx<float> w1 = mul(pre[k + H], mk<float>(yc, -yd));
      const cpx<float> A = add(w0, w1);
      const cpx<float> B = mul(sub(w0, w1), conj(twl[k]));
      z[q] = mk<float>(A.x - B.y, A.y + B.x);
    }
    fft_regs<float, H, 1, 32>(z, work + lane, twh, t);
#pragma unroll
    for (int q = 0; q < 8; ++q) {
      const int m = t + q * T16;
      D[makhoul_src(2 * m, L) * 32 + lane] = z[q].x;
      D[makhoul_src(2 * m + 1, L) * 32 + lane] = z[q].y;
    }
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");   // the stores below read these writes
    __syncthreads();
    if (tid == 0) {
      tma_store2(&maps.v, tile * 32, 0, smem_addr(V));
      tma_store2(&maps.t, tile * 32, 0, smem_addr(D));
      asm volatile("cp.async.bulk.commit_group;" ::: "memory");
      const int next = tile + 2 * gridDim.x;
      if (next < ntiles) {
        // the stores must have read stage s before the next tile lands there
        asm volatile("cp.async.bulk.wait_group.read 0;" ::: "memory");
        const uint32_t bar = bar0 + 8 * s;
        asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(kBytes) : "memory");
        tma_load2(smem_addr(D), &maps.d, next * 32, 0, bar);
        tma_load2(smem_addr(V), &maps.v, next * 32, 0, bar);
        pend |= 1u << s;
        pend_ph = (pend_ph & ~(1u << s)) | ((((uint32_t)(it >> 1) + 1u) & 1u) << s);
      }
    }
  }
  if (tid == 0) {
    if (gave_up) {
      atomicAdd(&g_spec_timeouts, 1);
      // copies still in flight land before the block's shared memory goes away
      for (int b = 0; b < 2; ++b)
        if ((pend >> b) & 1u) mbar_try(bar0 + 8 * b, (pend_ph >> b) & 1u, kSpecPolls);
    }
    asm volatile("cp.async.bulk.wait_group 0;" ::: "memory");
  }
}

typedef CUresult (*SpecEncodeFn)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                 const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                 CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

static SpecEncodeFn spec_encoder() {
  static SpecEncodeFn fn = nullptr;
  static bool tried = false;
  if (!tried) {
    tried = true;
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<SpecEncodeFn>(p);
  }
  return fn;
}

// 2-D map of a [L][npix] float32 array with [L][32] boxes.
static bool spec_map(CUtensorMap* m, const float* base, int npix, int L) {
  SpecEncodeFn enc = spec_encoder();
  if (!enc) return false;
  const cuuint64_t dims[2] = {(cuuint64_t)npix, (cuuint64_t)L};
  const cuuint64_t strides[1] = {(cuuint64_t)npix * sizeof(float)};
  const cuuint32_t box[2] = {32, (cuuint32_t)L};
  const cuuint32_t estr[2] = {1, 1};
  return enc(m, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, const_cast<float*>(base), dims, strides, box, estr,
             CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
             CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

int spectral_take_timeouts() {
  int v = 0, zero = 0;
  if (cudaMemcpyFromSymbol(&v, g_spec_timeouts, sizeof(int)) != cudaSuccess) return -1;
  if (v != 0 && cudaMemcpyToSymbol(g_spec_timeouts, &zero, sizeof(int)) != cudaSuccess) return -1;
  return v;
}

// Dense fallback: thread (lane, warp) forms coefficients k = warp, warp + W, ...
template <int MODE>
__global__ void __launch_bounds__(256)
k_spectral_dense(SpecArgs a, int npix, int L) {
  extern __shared__ __align__(16) float sm[];
  float* db = sm;            // [L][32]
  float* vb = sm + L * 32;   // [L][32]
  __shared__ double red[32];
  const int lane = threadIdx.x, w = threadIdx.y, W = blockDim.y;
  const int pix = blockIdx.x * 32 + lane;
  const bool ok = pix < npix;
  const size_t P = (size_t)npix;
  double acc = 0.0;
  if (MODE != SPEC_TONLY) {
    for (int l = w; l < L; l += W) db[l * 32 + lane] = ok ? __ldg(a.D + (size_t)l * P + pix) : 0.0f;
    __syncthreads();
    for (int kk = w; kk < L; kk += W) {
      const float* row = a.dense + (size_t)kk * L;
      float c = 0.0f;
      for (int l = 0; l < L; ++l) c = fmaf(__ldg(row + l), db[l * 32 + lane], c);
      if (MODE == SPEC_NORM) {
        acc += fabs((double)c);
      } else if (ok) {
        float* vp = a.V + (size_t)kk * P + pix;
        const float vo = *vp;
        const float vn = a.rho * sat1(vo + a.k * c) + (1.0f - a.rho) * vo;
        *vp = vn;
        vb[kk * 32 + lane] = vn;
      } else {
        vb[kk * 32 + lane] = 0.0f;
      }
    }
    if (MODE == SPEC_NORM) {
      const double tot = block_sum(acc, red);
      if (lane == 0 && w == 0) a.partials[blockIdx.x] = tot;
      return;
    }
  } else {
    for (int kk = w; kk < L; kk += W) vb[kk * 32 + lane] = ok ? __ldg(a.V + (size_t)kk * P + pix) : 0.0f;
  }
  __syncthreads();
  if (!ok) return;
  for (int l = w; l < L; l += W) {
    float x = 0.0f;
    for (int kk = 0; kk < L; ++kk) x = fmaf(__ldg(a.dense + (size_t)kk * L + l), vb[kk * 32 + lane], x);
    a.T[(size_t)l * P + pix] = x;
  }
}

template <int L> static size_t fft_smem() {
  return (size_t)(L / 2) * 32 * sizeof(cpx<float>) + (size_t)L * 32 * sizeof(float) + (size_t)(L / 2) * sizeof(cpx<float>);
}

template <int L> static cudaError_t spec_fft(const SpecArgs& a, int npix, int mode, cudaStream_t s) {
  dim3 grid((npix + 31) / 32), block(32, L / 16);
  switch (mode) {
    case SPEC_UPDATE: k_spectral_fft<L, SPEC_UPDATE><<<grid, block, fft_smem<L>(), s>>>(a, npix); break;
    case SPEC_NORM: k_spectral_fft<L, SPEC_NORM><<<grid, block, fft_smem<L>(), s>>>(a, npix); break;
    case SPEC_TONLY: k_spectral_fft<L, SPEC_TONLY><<<grid, block, fft_smem<L>(), s>>>(a, npix); break;
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

template <int L> static cudaError_t spec_tma(const SpecArgs& a, int npix, cudaStream_t s) {
  SpecMaps maps;
  if (!spec_map(&maps.d, a.D, npix, L) || !spec_map(&maps.v, a.V, npix, L) || !spec_map(&maps.t, a.T, npix, L))
    return cudaErrorNotSupported;
  // persistent grid: as many blocks as fit on the device at once
  static int resident = 0;
  if (!resident) {
    int dev = 0, sms = 1, occ = 1;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_spectral_tma<L>, 2 * L, SpecTma<L>::SMEM) != cudaSuccess ||
        occ < 1)
      occ = 1;
    resident = (sms > 0 ? sms : 1) * occ;
  }
  const int ntiles = npix / 32;
  dim3 grid(ntiles < resident ? ntiles : resident), block(32, L / 16);
  k_spectral_tma<L><<<grid, block, SpecTma<L>::SMEM, s>>>(maps, a, ntiles);
  return cudaGetLastError();
}

// The TMA kernel serves the update pass of power-of-two L >= 16 when the
// pixel count is a multiple of 32 and the arrays are 16-byte aligned.
static bool spec_tma_ok(const SpecArgs& a, int npix, int L) {
  const auto al = [](const void* p) { return ((uintptr_t)p & 15) == 0; };
  return spectral_uses_fft(L) && npix % 32 == 0 && al(a.D) && al(a.V) && al(a.T) &&
         getenv("MUFFIN_SPECTRAL_PLAIN") == nullptr;
}

cudaError_t launch_spectral(const SpecArgs& a, int npix, int L, int mode, cudaStream_t s, int* nblocks) {
  if (nblocks) *nblocks = (npix + 31) / 32;
  if (mode == SPEC_UPDATE && spec_tma_ok(a, npix, L)) {
    switch (L) {
      case 16: return spec_tma<16>(a, npix, s);
      case 32: return spec_tma<32>(a, npix, s);
      case 64: return spec_tma<64>(a, npix, s);
      case 128: return spec_tma<128>(a, npix, s);
      case 256: return spec_tma<256>(a, npix, s);
    }
  }
  if (spectral_uses_fft(L)) {
    switch (L) {
      case 16: return spec_fft<16>(a, npix, mode, s);
      case 32: return spec_fft<32>(a, npix, mode, s);
      case 64: return spec_fft<64>(a, npix, mode, s);
      case 128: return spec_fft<128>(a, npix, mode, s);
      case 256: return spec_fft<256>(a, npix, mode, s);
    }
    return cudaErrorInvalidValue;
  }
  dim3 grid((npix + 31) / 32), block(32, 8);
  const size_t smem = (size_t)2 * L * 32 * sizeof(float);
  switch (mode) {
    case SPEC_UPDATE: k_spectral_dense<SPEC_UPDATE><<<grid, block, smem, s>>>(a, npix, L); break;
    case SPEC_NORM: k_spectral_dense<SPEC_NORM><<<grid, block, smem, s>>>(a, npix, L); break;
    case SPEC_TONLY: k_spectral_dense<SPEC_TONLY><<<grid, block, smem, s>>>(a, npix, L); break;
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

template <int L> static cudaError_t cfg_fft() {
  cudaError_t e;
  if ((e = allow_max_dyn_smem(k_spectral_tma<L>))) return e;
  if ((e = allow_max_dyn_smem(k_spectral_fft<L, SPEC_UPDATE>))) return e;
  if ((e = allow_max_dyn_smem(k_spectral_fft<L, SPEC_NORM>))) return e;
  return allow_max_dyn_smem(k_spectral_fft<L, SPEC_TONLY>);
}

cudaError_t spectral_configure(int L) {
  if (spectral_uses_fft(L)) {
    switch (L) {
      case 16: return cfg_fft<16>();
      case 32: return cfg_fft<32>();
      case 64: return cfg_fft<64>();
      case 128: return cfg_fft<128>();
      case 256: return cfg_fft<256>();
    }
    return cudaErrorInvalidValue;
  }
  cudaError_t e;
  if ((e = allow_max_dyn_smem(k_spectral_dense<SPEC_UPDATE>))) return e;
  if ((e = allow_max_dyn_smem(k_spectral_dense<SPEC_NORM>))) return e;
  return allow_max_dyn_smem(k_spectral_dense<SPEC_TONLY>);
}

}  // namespace muffin
