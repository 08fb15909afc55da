// Per-block body of the spectral update (Eqs. 13-14 and the next pass's
// T = W_lambda^T V) for the persistent batch kernel: a block of NT threads
// handles NT / (2L) tiles of 32 pixels at once (thread group g = tid / (2L)
// takes tile tile0 + g), each as in k_spectral_fft (Makhoul's DCT through a
// half-length complex FFT, pixels on lanes).  Power-of-two L with 2L <= NT.
// D is read at L2 (__ldcg): it is written earlier in the same launch.
#pragma once
#include "device.cuh"
#include "internal.h"

namespace muffin {

__host__ __device__ __forceinline__ int makhoul_src(int m, int L) { return m < L / 2 ? 2 * m : 2 * (L - 1 - m) + 1; }

template <int L, int NT> struct SpecBlock {
  static constexpr int G = NT / (2 * L), H = L / 2;
  // per group: work [H][32] complex, vb [L][32]; then twh [H] shared by the groups
  static constexpr size_t GROUP = (size_t)H * 32 * 8 + (size_t)L * 32 * 4;
  static constexpr size_t SMEM = G * GROUP + (size_t)H * 8;
};

template <int L, int NT>
__device__ __forceinline__ void spectral_update_block(const SpecArgs& a, int npix, int tile0, int ntiles,
                                                      unsigned char* smem) {
  using B = SpecBlock<L, NT>;
  constexpr int H = L / 2, T16 = L / 16;
  const int tid = threadIdx.x, grp = tid / (2 * L), lt = tid % (2 * L);
  const int lane = lt & 31, t = lt >> 5;
  cpx<float>* work = reinterpret_cast<cpx<float>*>(smem + grp * B::GROUP);
  float* vb = reinterpret_cast<float*>(smem + grp * B::GROUP + (size_t)H * 32 * 8);
  cpx<float>* twh = reinterpret_cast<cpx<float>*>(smem + B::G * B::GROUP);
  const cpx<float>* twl = reinterpret_cast<const cpx<float>*>(a.tw);
  const cpx<float>* post = reinterpret_cast<const cpx<float>*>(a.post);
  const cpx<float>* pre = reinterpret_cast<const cpx<float>*>(a.pre);
  for (int i = tid; i < H; i += NT) twh[i] = twl[2 * i];
  const int tile = tile0 + grp;
  const int pix = tile * 32 + lane;
  const bool ok = tile < ntiles && pix < npix;
  const size_t P = (size_t)npix;
  cpx<float> z[8];
  float vold[16];
#pragma unroll
  for (int q = 0; q < 8; ++q) {
    const int m = t + q * T16;
    z[q] = ok ? mk<float>(__ldcg(a.D + (size_t)makhoul_src(2 * m, L) * P + pix),
                          __ldcg(a.D + (size_t)makhoul_src(2 * m + 1, L) * P + pix))
              : mk<float>(0.0f, 0.0f);
  }
  __syncthreads();
  fft_regs<float, H, -1, 32>(z, work + lane, twh, t);
#pragma unroll
  for (int q = 0; q < 8; ++q) {
    const int m = t + q * T16;
    vold[q] = ok ? a.V[(size_t)m * P + pix] : 0.0f;
    vold[q + 8] = ok ? a.V[(size_t)(m + H) * P + pix] : 0.0f;
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
    const cpx<float> o = mk<float>(0.5f * d.y, -0.5f * d.x);
    const cpx<float> wo = mul(twl[k], o);
    const cpx<float> v0 = add(e, wo), v1 = sub(e, wo);
    const cpx<float> p0 = post[k], p1 = post[k + H];
    const float c0 = p0.x * v0.x - p0.y * v0.y, c1 = p1.x * v1.x - p1.y * v1.y;
    const float n0 = a.rho * sat1(vold[q] + a.k * c0) + (1.0f - a.rho) * vold[q];
    const float n1 = a.rho * sat1(vold[q + 8] + a.k * c1) + (1.0f - a.rho) * vold[q + 8];
    if (ok) {
      a.V[(size_t)k * P + pix] = n0;
      a.V[(size_t)(k + H) * P + pix] = n1;
    }
    vb[k * 32 + lane] = ok ? n0 * a.invs[k] : 0.0f;
    vb[(k + H) * 32 + lane] = ok ? n1 * a.invs[k + H] : 0.0f;
  }
  __syncthreads();
#pragma unroll
  for (int q = 0; q < 8; ++q) {
    const int k = t + q * T16;
    const float ya = vb[k * 32 + lane], yb = k == 0 ? 0.0f : vb[(L - k) * 32 + lane];
    const float yc = vb[(k + H) * 32 + lane], yd = vb[(H - k) * 32 + lane];
    const cpx<float> w0 = mul(pre[k], mk<float>(ya, -yb));
    const cpx<float> w1 = mul(pre[k + H], mk<float>(yc, -yd));
    const cpx<float> A = add(w0, w1);
    const cpx<float> B = mul(sub(w0, w1), conj(twl[k]));
    z[q] = mk<float>(A.x - B.y, A.y + B.x);
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

// Dense orthonormal DCT for other L: one 32-pixel tile per block, warps take
// coefficients; smem: 2 L 32 floats.
template <int NT>
__device__ __forceinline__ void spectral_dense_block(const SpecArgs& a, int npix, int L, int tile, float* sm) {
  float* db = sm;
  float* vb = sm + L * 32;
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, W = NT / 32;
  const int pix = tile * 32 + lane;
  const bool ok = pix < npix;
  const size_t P = (size_t)npix;
  for (int l = w; l < L; l += W) db[l * 32 + lane] = ok ? __ldcg(a.D + (size_t)l * P + pix) : 0.0f;
  __syncthreads();
  for (int kk = w; kk < L; kk += W) {
    const float* row = a.dense + (size_t)kk * L;
    float c = 0.0f;
    for (int l = 0; l < L; ++l) c = fmaf(__ldg(row + l), db[l * 32 + lane], c);
    if (ok) {
      float* vp = a.V + (size_t)kk * P + pix;
      const float vo = *vp;
      const float vn = a.rho * sat1(vo + a.k * c) + (1.0f - a.rho) * vo;
      *vp = vn;
      vb[kk * 32 + lane] = vn;
    } else {
      vb[kk * 32 + lane] = 0.0f;
    }
  }
  __syncthreads();
  if (ok) {
    for (int l = w; l < L; l += W) {
      float x = 0.0f;
      for (int kk = 0; kk < L; ++kk) x = fmaf(__ldg(a.dense + (size_t)kk * L + l), vb[kk * 32 + lane], x);
      a.T[(size_t)l * P + pix] = x;
    }
  }
}

}  // namespace muffin
