// W_s as a union of eight orthonormal Daubechies wavelet bases, the
// comparison dictionary of Sec. 4 (the one of the first MUFFIN version):
//   W_s x = (1/sqrt 8) [Psi_1 x; ...; Psi_8 x],
// Psi_p the J-level periodic separable 2D discrete wavelet transform with the
// Daubechies filter of p vanishing moments, coefficients of each basis in the
// Mallat layout of an N x N plane (level j transforms the top-left
// (N/2^j)^2 square; its detail quadrants are final, its low-low quadrant feeds
// level j+1).  W_s^T W_s = I (a tight frame).
//
// One analysis step along an axis of even length M:
//   lo[k] = sum_t h[t] x[(2k + t) mod M],  hi[k] = sum_t g[t] x[(2k + t) mod M],
//   g[t] = (-1)^t h[2p-1-t];
// its adjoint (= inverse, the bank is orthonormal):
//   x[i] = sum_{t = i mod 2} h[t] lo[k] + g[t] hi[k],  k = ((i - t) mod M) / 2.
// Every launch covers all channels and all eight bases (gridDim.z = 8 L);
// each thread computes a run of outputs (kRowsPerBlock rows per block in the
// row kernels, kColRun outputs per thread in the column kernels), so blocks
// live long enough to amortise their scheduling.
// The levels are short (at most a few MB per basis and channel) and the filters
// at most 16 taps: the kernels read straight from global memory through L1.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <complex>
#include <vector>

#include "device.cuh"
#include "internal.h"

namespace muffin {

constexpr int kMaxTaps = 16;

__constant__ float c_dbh[kDbBases][kMaxTaps];
__constant__ float c_dbg[kDbBases][kMaxTaps];

// ------------------------------------------------------------------ filters (host)

// H(z) = sqrt(2) ((1 + z^-1)/2)^p Q(z) with |Q(e^iw)|^2 = P(sin^2(w/2)),
// P(y) = sum_{k<p} C(p-1+k, k) y^k; each root y_k of P gives the pair of
// z roots of z^2 - 2(1 - 2y_k) z + 1, of which Q keeps the one inside the unit
// circle (minimum phase); Q(1) = 1.  Roots of P by the Weierstrass
// (Durand-Kerner) iteration.
bool daubechies_lowpass(int p, double* h) {
  using cd = std::complex<double>;
  if (p < 1 || p > kDbBases || !h) return false;
  const int deg = p - 1;
  std::vector<double> a(p);   // ascending coefficients of P
  for (int k = 0; k < p; ++k) {
    double c = 1.0;           // C(p-1+k, k)
    for (int i = 1; i <= k; ++i) c = c * (p - 1 + i) / i;
    a[k] = c;
  }
  std::vector<cd> roots(deg);
  if (deg > 0) {
    auto eval = [&](cd y) {   // monic P(y) / a[deg]
      cd v = 1.0;
      for (int k = deg - 1; k >= 0; --k) v = v * y + a[k] / a[deg];
      return v;
    };
    const cd seed(0.4, 0.9);
    cd w = 1.0;
    for (int i = 0; i < deg; ++i) { roots[i] = w; w *= seed; }
    for (int it = 0; it < 2000; ++it) {
      double move = 0.0;
      for (int i = 0; i < deg; ++i) {
        cd den = 1.0;
        for (int j = 0; j < deg; ++j) if (j != i) den *= roots[i] - roots[j];
        const cd d = eval(roots[i]) / den;
        roots[i] -= d;
        move = std::max(move, std::abs(d));
      }
      if (move < 1e-16) break;
    }
  }
  std::vector<cd> q(1, cd(1.0));
  for (int i = 0; i < deg; ++i) {
    const cd aa = 1.0 - 2.0 * roots[i];
    const cd r = std::sqrt(aa * aa - 1.0);
    const cd zk = std::abs(aa + r) < 1.0 ? aa + r : aa - r;
    std::vector<cd> nq(q.size() + 1, cd(0.0));
    for (size_t t = 0; t < q.size(); ++t) { nq[t] += q[t]; nq[t + 1] -= zk * q[t]; }
    for (auto& v : nq) v /= (1.0 - zk);
    q.swap(nq);
  }
  std::vector<double> binom(p + 1);
  for (int t = 0; t <= p; ++t) {
    double c = 1.0;
    for (int i = 1; i <= t; ++i) c = c * (p - t + i) / i;
    binom[t] = c / std::ldexp(1.0, p);
  }
  for (int t = 0; t < 2 * p; ++t) {
    cd acc = 0.0;
    for (int u = 0; u <= p; ++u) {
      const int v = t - u;
      if (v >= 0 && v < (int)q.size()) acc += binom[u] * q[v];
    }
    h[t] = std::sqrt(2.0) * acc.real();
  }
  return true;
}

cudaError_t dwt_configure() {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  static bool done[64] = {};
  if (dev < 64 && done[dev]) return cudaSuccess;
  float hf[kDbBases][kMaxTaps] = {}, gf[kDbBases][kMaxTaps] = {};
  for (int b = 0; b < kDbBases; ++b) {
    double h[kMaxTaps];
    const int p = b + 1, taps = 2 * p;
    daubechies_lowpass(p, h);
    for (int t = 0; t < taps; ++t) {
      hf[b][t] = (float)h[t];
      gf[b][t] = (float)((t & 1 ? -1.0 : 1.0) * h[taps - 1 - t]);
    }
  }
  if ((e = cudaMemcpyToSymbol(c_dbh, hf, sizeof(hf))) != cudaSuccess) return e;
  if ((e = cudaMemcpyToSymbol(c_dbg, gf, sizeof(gf))) != cudaSuccess) return e;
  if (dev < 64) done[dev] = true;
  return cudaSuccess;
}

// ------------------------------------------------------------------ kernels

constexpr float kUnionScale = 0.35355339059327373f;   // 1/sqrt(8)
constexpr int kRowsPerBlock = 8;
constexpr int kColRun = 4;

// The kernels below run one body per basis, instantiated for its filter length
// (TAPS = 2p, compile time) so that every tap loop unrolls and its loads issue
// together; the block's basis b = blockIdx.z & 7 picks the body.
#define MUFFIN_DB_DISPATCH(CALL) \
  switch (blockIdx.z & 7) {      \
    case 0: CALL(2); break;      \
    case 1: CALL(4); break;      \
    case 2: CALL(6); break;      \
    case 3: CALL(8); break;      \
    case 4: CALL(10); break;     \
    case 5: CALL(12); break;     \
    case 6: CALL(14); break;     \
    default: CALL(16); break;    \
  }

// Analysis, rows of level M: W1[z][r][k] = lo, W1[z][r][M/2 + k] = hi, for
// the level input (level 0: the shared input cube; else W2[z], the previous
// level's low-low quadrant).  grid (1, row groups, 8 L).
template <int TAPS>
__device__ __forceinline__ void dwt_rows_body(const float* __restrict__ src0, const float* __restrict__ W2,
                                              float* __restrict__ W1, int n, int M, int level0) {
  const int z = blockIdx.z, b = z & 7, l = z >> 3;
  const int H = M >> 1, m = M - 1;
  const size_t P = (size_t)n * n;
  const int r1 = min(M, (int)(blockIdx.y + 1) * kRowsPerBlock);
  for (int r = blockIdx.y * kRowsPerBlock; r < r1; ++r) {
    const float* src = (level0 ? src0 + (size_t)l * P : W2 + (size_t)z * P) + (size_t)r * n;
    float* dst = W1 + (size_t)z * P + (size_t)r * n;
    for (int k = threadIdx.x; k < H; k += blockDim.x) {
      float x[TAPS];
#pragma unroll
      for (int t = 0; t < TAPS; ++t) x[t] = __ldg(src + ((2 * k + t) & m));
      float lo = 0.f, hi = 0.f;
#pragma unroll
      for (int t = 0; t < TAPS; ++t) {
        lo = fmaf(c_dbh[b][t], x[t], lo);
        hi = fmaf(c_dbg[b][t], x[t], hi);
      }
      dst[k] = lo;
      dst[H + k] = hi;
    }
  }
}

__global__ void k_dwt_rows(const float* __restrict__ src0, const float* __restrict__ W2, float* __restrict__ W1,
                           int n, int M, int level0) {
#define CALL(T) dwt_rows_body<T>(src0, W2, W1, n, M, level0)
  MUFFIN_DB_DISPATCH(CALL)
#undef CALL
}

// Analysis, columns of level M: outputs (k, c) = lo and (M/2 + k, c) = hi of
// column c of W1[z].  The low-low quadrant feeds the next level (W2[z]) unless
// this is the last level; every final coefficient w (scaled by 1/sqrt 8)
// updates U: MODE_UPDATE U <- rho sat(U + k w) + (1 - rho) U, MODE_LINEAR U = w.
// block (32 columns, 8 outputs), kColRun outputs per thread.
template <int MODE, int TAPS>
__device__ __forceinline__ void dwt_cols_body(const float* __restrict__ W1, float* __restrict__ W2,
                                              float* __restrict__ U, int n, int M, int last, float kk, float rho) {
  const int z = blockIdx.z, b = z & 7;
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  const int H = M >> 1, m = M - 1;
  if (c >= M) return;
  const size_t P = (size_t)n * n;
  const float* col = W1 + (size_t)z * P + c;
  float* Uz = U + (size_t)z * P;
  auto put = [&](int row, float w) {
    float* u = Uz + (size_t)row * n + c;
    w *= kUnionScale;
    if (MODE == MODE_UPDATE) {
      const float uo = *u;
      *u = rho * sat1(uo + kk * w) + (1.0f - rho) * uo;
    } else {
      *u = w;
    }
  };
#pragma unroll 1
  for (int j = 0; j < kColRun; ++j) {
    const int k = (blockIdx.y * kColRun + j) * blockDim.y + threadIdx.y;
    if (k >= H) break;
    float x[TAPS];
#pragma unroll
    for (int t = 0; t < TAPS; ++t) x[t] = __ldg(col + (size_t)((2 * k + t) & m) * n);
    float lo = 0.f, hi = 0.f;
#pragma unroll
    for (int t = 0; t < TAPS; ++t) {
      lo = fmaf(c_dbh[b][t], x[t], lo);
      hi = fmaf(c_dbg[b][t], x[t], hi);
    }
    if (c < H && !last) W2[(size_t)z * P + (size_t)k * n + c] = lo;
    else put(k, lo);
    put(H + k, hi);
  }
}

template <int MODE>
__global__ void k_dwt_cols(const float* __restrict__ W1, float* __restrict__ W2, float* __restrict__ U, int n,
                           int M, int last, float kk, float rho) {
#define CALL(T) dwt_cols_body<MODE, T>(W1, W2, U, n, M, last, kk, rho)
  MUFFIN_DB_DISPATCH(CALL)
#undef CALL
}

// Adjoint, columns of level M: W1[z][i][c] from the low half (rows < M/2:
// the low-low quadrant from W2[z], or from U at the coarsest level, next to the
// U quadrant for c >= M/2) and the high half (U rows >= M/2).
template <int TAPS>
__device__ __forceinline__ void idwt_cols_body(const float* __restrict__ U, const float* __restrict__ W2,
                                               float* __restrict__ W1, int n, int M, int coarsest) {
  const int z = blockIdx.z, b = z & 7;
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  const int H = M >> 1, m = M - 1;
  if (c >= M) return;
  const size_t P = (size_t)n * n;
  const float* lo = ((c < H && !coarsest) ? W2 : U) + (size_t)z * P + c;
  const float* hi = U + (size_t)z * P + (size_t)H * n + c;
#pragma unroll 1
  for (int j = 0; j < kColRun; ++j) {
    const int i = (blockIdx.y * kColRun + j) * blockDim.y + threadIdx.y;
    if (i >= M) break;
    const int par = i & 1;
    float a[TAPS / 2], d[TAPS / 2];
#pragma unroll
    for (int s2 = 0; s2 < TAPS / 2; ++s2) {
      const size_t kk = (size_t)(((i - par - 2 * s2) & m) >> 1) * n;
      a[s2] = __ldg(lo + kk);
      d[s2] = __ldg(hi + kk);
    }
    float acc = 0.f;
#pragma unroll
    for (int s2 = 0; s2 < TAPS / 2; ++s2) {
      acc = fmaf(c_dbh[b][par + 2 * s2], a[s2], acc);
      acc = fmaf(c_dbg[b][par + 2 * s2], d[s2], acc);
    }
    W1[(size_t)z * P + (size_t)i * n + c] = acc;
  }
}

__global__ void k_idwt_cols(const float* __restrict__ U, const float* __restrict__ W2, float* __restrict__ W1,
                            int n, int M, int coarsest) {
#define CALL(T) idwt_cols_body<T>(U, W2, W1, n, M, coarsest)
  MUFFIN_DB_DISPATCH(CALL)
#undef CALL
}

// Adjoint, rows of level M: out[z][r][i] from W1[z][r][k] (low) and W1[z][r][M/2 + k] (high).
template <int TAPS>
__device__ __forceinline__ void idwt_rows_body(const float* __restrict__ W1, float* __restrict__ out, int n, int M) {
  const int z = blockIdx.z, b = z & 7;
  const int H = M >> 1, m = M - 1;
  const size_t P = (size_t)n * n;
  const int r1 = min(M, (int)(blockIdx.y + 1) * kRowsPerBlock);
  for (int r = blockIdx.y * kRowsPerBlock; r < r1; ++r) {
    const float* src = W1 + (size_t)z * P + (size_t)r * n;
    float* dst = out + (size_t)z * P + (size_t)r * n;
    for (int i = threadIdx.x; i < M; i += blockDim.x) {
      const int par = i & 1;
      float a[TAPS / 2], d[TAPS / 2];
#pragma unroll
      for (int s2 = 0; s2 < TAPS / 2; ++s2) {
        const int kk = ((i - par - 2 * s2) & m) >> 1;
        a[s2] = __ldg(src + kk);
        d[s2] = __ldg(src + H + kk);
      }
      float acc = 0.f;
#pragma unroll
      for (int s2 = 0; s2 < TAPS / 2; ++s2) {
        acc = fmaf(c_dbh[b][par + 2 * s2], a[s2], acc);
        acc = fmaf(c_dbg[b][par + 2 * s2], d[s2], acc);
      }
      dst[i] = acc;
    }
  }
}

__global__ void k_idwt_rows(const float* __restrict__ W1, float* __restrict__ out, int n, int M) {
#define CALL(T) idwt_rows_body<T>(W1, out, n, M)
  MUFFIN_DB_DISPATCH(CALL)
#undef CALL
}

// Finest level of the adjoint, rows, for all eight bases at once: S[l][r][i] =
// (1/sqrt 8) sum_b (row synthesis of W1[l][b] at (r, i)), bases summed in
// order, so the per-basis images are never stored.  grid (1, row groups, L).
template <int TAPS>
__device__ __forceinline__ float idwt_row_value(const float* __restrict__ src, int b, int i, int H, int m) {
  const int par = i & 1;
  float a[TAPS / 2], d[TAPS / 2];
#pragma unroll
  for (int s2 = 0; s2 < TAPS / 2; ++s2) {
    const int kk = ((i - par - 2 * s2) & m) >> 1;
    a[s2] = __ldg(src + kk);
    d[s2] = __ldg(src + H + kk);
  }
  float acc = 0.f;
#pragma unroll
  for (int s2 = 0; s2 < TAPS / 2; ++s2) {
    acc = fmaf(c_dbh[b][par + 2 * s2], a[s2], acc);
    acc = fmaf(c_dbg[b][par + 2 * s2], d[s2], acc);
  }
  return acc;
}

__global__ void k_idwt_rows_sum(const float* __restrict__ W1, float* __restrict__ S, int n) {
  const int l = blockIdx.z, M = n, H = M >> 1, m = M - 1;
  const size_t P = (size_t)n * n;
  const int r1 = min(M, (int)(blockIdx.y + 1) * kRowsPerBlock);
  for (int r = blockIdx.y * kRowsPerBlock; r < r1; ++r) {
    const float* src = W1 + (size_t)l * kDbBases * P + (size_t)r * n;
    for (int i = threadIdx.x; i < M; i += blockDim.x) {
      float acc = idwt_row_value<2>(src, 0, i, H, m);
      acc += idwt_row_value<4>(src + P, 1, i, H, m);
      acc += idwt_row_value<6>(src + 2 * P, 2, i, H, m);
      acc += idwt_row_value<8>(src + 3 * P, 3, i, H, m);
      acc += idwt_row_value<10>(src + 4 * P, 4, i, H, m);
      acc += idwt_row_value<12>(src + 5 * P, 5, i, H, m);
      acc += idwt_row_value<14>(src + 6 * P, 6, i, H, m);
      acc += idwt_row_value<16>(src + 7 * P, 7, i, H, m);
      S[(size_t)l * P + (size_t)r * n + i] = kUnionScale * acc;
    }
  }
}

__global__ void k_abs_sum(const float* __restrict__ x, size_t n, double* __restrict__ partials) {
  __shared__ double red[32];
  double acc = 0.0;
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
    acc += fabs((double)x[i]);
  const double t = block_sum(acc, red);
  if (threadIdx.x == 0) partials[blockIdx.x] = t;
}

// ------------------------------------------------------------------ launchers

cudaError_t launch_dwt_analysis(const Geom& g, const DwtArgs& a, int mode, cudaStream_t s) {
  const int n = g.n, Z = kDbBases * g.L;
  for (int j = 0; j < g.J; ++j) {
    const int M = n >> j, H = M >> 1;
    k_dwt_rows<<<dim3(1, (M + kRowsPerBlock - 1) / kRowsPerBlock, Z), 128, 0, s>>>(a.src, a.W2, a.W1, n, M, j == 0);
    const dim3 grid((M + 31) / 32, (H + 8 * kColRun - 1) / (8 * kColRun), Z), block(32, 8);
    const int last = j == g.J - 1;
    if (mode == MODE_UPDATE) k_dwt_cols<MODE_UPDATE><<<grid, block, 0, s>>>(a.W1, a.W2, a.U, n, M, last, a.k, a.rho);
    else k_dwt_cols<MODE_LINEAR><<<grid, block, 0, s>>>(a.W1, a.W2, a.U, n, M, last, 1.f, 1.f);
  }
  return cudaGetLastError();
}

cudaError_t launch_dwt_adjoint(const Geom& g, const DwtArgs& a, cudaStream_t s) {
  const int n = g.n, Z = kDbBases * g.L;
  for (int j = g.J - 1; j >= 0; --j) {
    const int M = n >> j;
    k_idwt_cols<<<dim3((M + 31) / 32, (M + 8 * kColRun - 1) / (8 * kColRun), Z), dim3(32, 8), 0, s>>>(
        a.U, a.W2, a.W1, n, M, j == g.J - 1);
    if (j > 0) k_idwt_rows<<<dim3(1, (M + kRowsPerBlock - 1) / kRowsPerBlock, Z), 128, 0, s>>>(a.W1, a.W2, n, M);
    else k_idwt_rows_sum<<<dim3(1, (M + kRowsPerBlock - 1) / kRowsPerBlock, g.L), 256, 0, s>>>(a.W1, a.S, n);
  }
  return cudaGetLastError();
}

cudaError_t launch_abs_sum(const float* x, size_t n, double* partials, int* nparts, cudaStream_t s) {
  const int blocks = (int)std::min<size_t>((n + 255) / 256, 1024);
  k_abs_sum<<<blocks, 256, 0, s>>>(x, n, partials);
  if (nparts) *nparts = blocks;
  return cudaGetLastError();
}

}  // namespace muffin

extern "C" int muffin_daubechies_filter(int p, double* h_out) {
  return muffin::daubechies_lowpass(p, h_out) ? 0 : -1;
}
