// Per-block bodies of the gradient FFT kernels (Algorithm 1, first line; Eq. 8),
// shared by the one-stage kernels of k_fft.cu and the persistent batch kernel.
//   rows_fwd_block  PAIRS pairs of real rows of channel l -> half-spectrum rows
//   cols_block      C spectrum columns of channel l: FFT, multiply by K, inverse
//   rows_inv_block  PAIRS pairs of rows: inverse FFT, then the primal step
// Each takes its shared memory by pointer and expects the block's threads
// (PAIRS x N/8 or C x N/8) to call it together.
#pragma once
#include "device.cuh"
#include "internal.h"

namespace muffin {

template <int N> __host__ __device__ constexpr int rows_pairs() { return (2048 / N) < (N / 2) ? (2048 / N) : (N / 2); }
template <int N> __host__ __device__ constexpr int cols_per_cta() { return N >= 512 ? 8 : ((N / 2) < 16 ? (N / 2) : 16); }

// tw: N twiddles exp(-2 pi i m / N) in shared memory; buf: PAIRS * fft_slots<N, 1>() slots.
// Row pair f of the block (threadIdx.x / (N/8)) holds rows y0, y0 + 1 with
// y0 = 2 (bx PAIRS + f).
template <int N, int PAIRS>
__device__ __forceinline__ void rows_fwd_block(const float* __restrict__ X, cpx<float>* __restrict__ spec,
                                               const cpx<float>* tw, cpx<float>* buf, int l, int bx) {
  constexpr int T8 = N / 8, H = N / 2, NP = fft_slots<N, 1>();
  const int f = threadIdx.x / T8, t = threadIdx.x % T8;
  const int y0 = 2 * (bx * PAIRS + f);
  const float* r0 = X + ((size_t)l * N + y0) * N;
  cpx<float> v[8];
#pragma unroll
  for (int q = 0; q < 8; ++q) v[q] = mk<float>(__ldg(r0 + t + q * T8), __ldg(r0 + N + t + q * T8));
  __syncthreads();
  fft_regs<float, N, -1, 1, 1>(v, buf + f * NP, tw, t);
  __syncthreads();
#pragma unroll
  for (int q = 0; q < 8; ++q) buf[f * NP + fft_slot<1>(t + q * T8)] = v[q];
  __syncthreads();
  cpx<float>* o0 = spec + ((size_t)l * N + y0) * H;
  cpx<float>* o1 = o0 + H;
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    const int k = t + q * T8;
    const cpx<float> zk = buf[f * NP + fft_slot<1>(k)];
    if (k == 0) {
      const cpx<float> zn = buf[f * NP + fft_slot<1>(H)];
      o0[0] = mk<float>(zk.x, zn.x);
      o1[0] = mk<float>(zk.y, zn.y);
    } else {
      const cpx<float> zm = buf[f * NP + fft_slot<1>(N - k)];
      o0[k] = mk<float>(0.5f * (zk.x + zm.x), 0.5f * (zk.y - zm.y));
      o1[k] = mk<float>(0.5f * (zk.y + zm.y), 0.5f * (zm.x - zk.x));
    }
  }
}

// C columns kx = bx C + c of channel l (c = threadIdx.x % C); buf: N * C slots.
template <int N, int C>
__device__ __forceinline__ void cols_block(cpx<float>* __restrict__ spec, const float* __restrict__ Kp,
                                           const float* __restrict__ Kb, const cpx<float>* tw, cpx<float>* buf,
                                           int l, int bx) {
  constexpr int T8 = N / 8, H = N / 2;
  const int c = threadIdx.x % C, t = threadIdx.x / C;
  const int kx = bx * C + c;
  cpx<float>* base = spec + (size_t)l * N * H;
  cpx<float> v[8];
  float ka[8], kb[8];
  const float* Kl = Kp + (size_t)l * N * H;
#pragma unroll
  for (int q = 0; q < 8; ++q) {
    v[q] = base[(t + q * T8) * H + kx];
    ka[q] = __ldg(Kl + (t + q * T8) * H + kx);   // multipliers arrive during the forward FFT
    kb[q] = kx == 0 ? __ldg(Kb + (size_t)l * N + t + q * T8) : 0.0f;
  }
  __syncthreads();
  fft_regs<float, N, -1, C>(v, buf + c, tw, t);
  __syncthreads();
#pragma unroll
  for (int q = 0; q < 8; ++q) buf[(t + q * T8) * C + c] = v[q];
  __syncthreads();
#pragma unroll
  for (int q = 0; q < 8; ++q) {
    const int pos = t + q * T8;
    if (kx == 0) {
      // (DC, Nyquist) packed column: Z'(k) = a Z(k) + b conj(Z(-k))
      const cpx<float> zm = buf[((N - pos) & (N - 1)) * C + c];
      v[q] = add(scale(v[q], ka[q]), scale(conj(zm), kb[q]));
    } else {
      v[q] = scale(v[q], ka[q]);
    }
  }
  fft_regs<float, N, 1, C>(v, buf + c, tw, t);
#pragma unroll
  for (int q = 0; q < 8; ++q) base[(t + q * T8) * H + kx] = v[q];
}

// MODE 0: primal step into a.X, a.D; MODE 1: H^T H x into out.
template <int N, int PAIRS, int MODE>
__device__ __forceinline__ void rows_inv_block(const cpx<float>* __restrict__ spec, const PrimalArgs& a,
                                               float* __restrict__ out, const cpx<float>* tw, cpx<float>* buf,
                                               int l, int bx) {
  constexpr int T8 = N / 8, H = N / 2, NP = fft_slots<N, 1>();
  const int f = threadIdx.x / T8, t = threadIdx.x % T8;
  const int y0 = 2 * (bx * PAIRS + f);
  const cpx<float>* s0 = spec + ((size_t)l * N + y0) * H;
  const cpx<float>* s1 = s0 + H;
  cpx<float> v[8];
#pragma unroll
  for (int q = 0; q < 8; ++q) {
    const int pos = t + q * T8;
    if (pos == 0) {
      const cpx<float> A = s0[0], B = s1[0];
      v[q] = mk<float>(A.x, B.x);
    } else if (pos == H) {
      const cpx<float> A = s0[0], B = s1[0];
      v[q] = mk<float>(A.y, B.y);
    } else if (pos < H) {
      const cpx<float> A = s0[pos], B = s1[pos];
      v[q] = mk<float>(A.x - B.y, A.y + B.x);
    } else {
      const cpx<float> A = s0[N - pos], B = s1[N - pos];
      v[q] = mk<float>(A.x + B.y, B.x - A.y);
    }
  }
  const size_t row0 = ((size_t)l * N + y0) * N;
  // epilogue inputs of this thread's 16 pixels, loaded before the FFT so that
  // their latency hides behind it: xo = X, bo = tau (mu_s S + mu_l T - b)
  float xo[16], bo[16];
  if constexpr (MODE == 0) {
#pragma unroll
    for (int q = 0; q < 8; ++q) {
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        const size_t idx = row0 + (size_t)h * N + t + q * T8;
        xo[2 * q + h] = a.X[idx];
        float st = -__ldg(a.b + idx);
        if (a.S) st += a.mu_s * __ldg(a.S + idx);
        if (a.T) st += a.mu_l * __ldg(a.T + idx);
        bo[2 * q + h] = st;
      }
    }
  }
  __syncthreads();
  fft_regs<float, N, 1, 1, 1>(v, buf + f * NP, tw, t);
#pragma unroll
  for (int q = 0; q < 8; ++q) {
    const int x = t + q * T8;
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const size_t idx = row0 + (size_t)h * N + x;
      const float g = h == 0 ? v[q].x : v[q].y;
      if constexpr (MODE == 0) {
        const float x0 = xo[2 * q + h];
        const float xt = fmaxf(x0 - a.tau * (g + bo[2 * q + h]), 0.0f);
        a.D[idx] = 2.0f * xt - x0;
        a.X[idx] = a.rho * xt + (1.0f - a.rho) * x0;
      } else {
        out[idx] = g;
      }
    }
  }
}

}  // namespace muffin
