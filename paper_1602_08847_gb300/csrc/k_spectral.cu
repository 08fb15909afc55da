// Spectral transform W_lambda (orthonormal DCT-II along the channel axis at
// every pixel, Eq. 6) fused with the spectral dual step of Algorithm 1 (fourth
// line; Eq. 13):  V <- rho sat(V + sigma mu_lambda DCT(D)) + (1 - rho) V, and
// with the spectral adjoint of the next pass: T = W_lambda^T V = DCT^-1(V)
// (first step of the master node in Sec. 3, computed here per pixel).
//
// One block handles 32 consecutive pixels (one per lane) and all L channels;
// reads and writes of D, V and T are coalesced along the pixels.
//  * L a power of two in [16, 256]: Makhoul's O(L log L) DCT through a
//    length-L complex FFT (reorder x -> v with v[m] = x[2m], v[L-1-m] =
//    x[2m+1]; DCT[k] = Re(exp(-i pi k / 2L) FFT(v)[k]); the inverse runs the
//    same steps backwards).  Warp w is FFT thread w of all 32 transforms.
//  * other L (<= 512): the dense orthonormal DCT matrix.
#include "device.cuh"
#include "internal.h"

namespace muffin {

bool spectral_uses_fft(int L) { return L >= 16 && L <= 256 && (L & (L - 1)) == 0; }

__device__ __forceinline__ int makhoul_src(int m, int L) { return m < L / 2 ? 2 * m : 2 * (L - 1 - m) + 1; }

template <int L, int MODE>
__global__ void __launch_bounds__(4 * L)
k_spectral_fft(SpecArgs a, int npix) {
  const float* __restrict__ invs = a.invs;
  constexpr int T8 = L / 8;
  extern __shared__ __align__(16) unsigned char smraw[];
  cpx<float>* work = reinterpret_cast<cpx<float>*>(smraw);        // [L][32]
  float* vb = reinterpret_cast<float*>(work + L * 32);            // [L][32]
  cpx<float>* tw = reinterpret_cast<cpx<float>*>(vb + L * 32);
  __shared__ double red[32];
  const int lane = threadIdx.x, t = threadIdx.y;
  const int tid = t * 32 + lane, nth = 32 * T8;
  for (int i = tid; i < L; i += nth) tw[i] = reinterpret_cast<const cpx<float>*>(a.tw)[i];
  const int pix = blockIdx.x * 32 + lane;
  const bool ok = pix < npix;
  const size_t P = (size_t)npix;
  cpx<float> v[8];
  double acc = 0.0;
  if (MODE != SPEC_TONLY) {
#pragma unroll
    for (int q = 0; q < 8; ++q) {
      const int mpos = t + q * T8;
      v[q] = mk<float>(ok ? __ldg(a.D + (size_t)makhoul_src(mpos, L) * P + pix) : 0.0f, 0.0f);
    }
    __syncthreads();
    fft_regs<float, L, -1, 32>(v, work + lane, tw, t);
#pragma unroll
    for (int q = 0; q < 8; ++q) {
      const int kk = t + q * T8;
      const cpx<float> pw = reinterpret_cast<const cpx<float>*>(a.post)[kk];
      const float cdct = pw.x * v[q].x - pw.y * v[q].y;   // Re(post[k] V[k]), orthonormal scale folded in
      if (MODE == SPEC_NORM) {
        acc += fabs((double)cdct);
      } else if (ok) {
        float* vp = a.V + (size_t)kk * P + pix;
        const float vo = *vp;
        const float vt = sat1(vo + a.k * cdct);
        const float vn = a.rho * vt + (1.0f - a.rho) * vo;
        *vp = vn;
        vb[kk * 32 + lane] = vn * invs[kk];
      } else {
        vb[kk * 32 + lane] = 0.0f;
      }
    }
    if (MODE == SPEC_NORM) {
      const double tot = block_sum(acc, red);
      if (tid == 0) a.partials[blockIdx.x] = tot;
      return;
    }
  } else {
#pragma unroll
    for (int q = 0; q < 8; ++q) {
      const int kk = t + q * T8;
      vb[kk * 32 + lane] = ok ? __ldg(a.V + (size_t)kk * P + pix) * invs[kk] : 0.0f;
    }
  }
  __syncthreads();
  // inverse: W[k] = pre[k] (y[k] - i y[L-k]), y[L] = 0, then an inverse FFT
#pragma unroll
  for (int q = 0; q < 8; ++q) {
    const int kk = t + q * T8;
    const float yr = vb[kk * 32 + lane];
    const float yi = kk == 0 ? 0.0f : vb[(L - kk) * 32 + lane];
    const cpx<float> pw = reinterpret_cast<const cpx<float>*>(a.pre)[kk];
    v[q] = mul(pw, mk<float>(yr, -yi));
  }
  fft_regs<float, L, 1, 32>(v, work + lane, tw, t);
  if (ok) {
#pragma unroll
    for (int q = 0; q < 8; ++q) {
      const int mpos = t + q * T8;
      a.T[(size_t)makhoul_src(mpos, L) * P + pix] = v[q].x;
    }
  }
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
  return (size_t)L * 32 * sizeof(cpx<float>) + (size_t)L * 32 * sizeof(float) + (size_t)L * sizeof(cpx<float>);
}

template <int L> static cudaError_t spec_fft(const SpecArgs& a, int npix, int mode, cudaStream_t s) {
  dim3 grid((npix + 31) / 32), block(32, L / 8);
  switch (mode) {
    case SPEC_UPDATE: k_spectral_fft<L, SPEC_UPDATE><<<grid, block, fft_smem<L>(), s>>>(a, npix); break;
    case SPEC_NORM: k_spectral_fft<L, SPEC_NORM><<<grid, block, fft_smem<L>(), s>>>(a, npix); break;
    case SPEC_TONLY: k_spectral_fft<L, SPEC_TONLY><<<grid, block, fft_smem<L>(), s>>>(a, npix); break;
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

cudaError_t launch_spectral(const SpecArgs& a, int npix, int L, int mode, cudaStream_t s, int* nblocks) {
  if (nblocks) *nblocks = (npix + 31) / 32;
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
