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
// Every launch covers all channels and all eight bases (gridDim.z = 8 L).
// The analysis runs one kernel per level, its row and column passes fused
// through shared memory (a block owns a slab of columns for all rows).  The
// adjoint runs a column and a row kernel per level, each thread computing a
// run of outputs (kColRun per thread, kRowsPerBlock rows per block) so that
// blocks live long enough to amortise their scheduling; the filters have at
// most 16 taps and those kernels read straight from global memory through L1.
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

// Analysis of one whole level, rows and columns fused through shared memory.
// A block owns a slab of SC consecutive columns k0 .. k0 + SC - 1 of the
// row-transformed plane (all lo columns or all hi columns, H % SC == 0):
// it computes them for all M rows into shared memory (row filter, inputs read
// through L1), then filters each of its columns: the low-low quadrant feeds
// the next level (written to `ll`, which the caller alternates between two
// scratch planes so that no level overwrites the plane it reads), every final
// coefficient updates U as in dwt_cols_body.  grid (M / SC, 1, 8 L), shared
// memory M * SC floats.
template <int MODE, int TAPS>
__device__ __forceinline__ void dwt_level_body(const float* __restrict__ src0, const float* __restrict__ llin,
                                               float* __restrict__ ll, float* __restrict__ U, int n, int M, int SC,
                                               int level0, int last, float kk, float rho, float* __restrict__ sY) {
  const int z = blockIdx.z, b = z & 7, l = z >> 3;
  const int H = M >> 1, m = M - 1;
  const size_t P = (size_t)n * n;
  const int k0 = blockIdx.x * SC;
  const bool hic = k0 >= H;                    // slab of high-pass (detail) columns
  const int kb = hic ? k0 - H : k0;
  const float* src = level0 ? src0 + (size_t)l * P : llin + (size_t)z * P;
  const int lsc = __ffs(SC) - 1;
  // the basis' filters in registers (constant-memory reads per tap would cost an issue slot each)
  float hf[TAPS], gf[TAPS];
#pragma unroll
  for (int t = 0; t < TAPS; ++t) {
    hf[t] = c_dbh[b][t];
    gf[t] = c_dbg[b][t];
  }
  for (int idx = threadIdx.x; idx < M * SC; idx += blockDim.x) {
    const int r = idx >> lsc, j = idx & (SC - 1);
    const float* row = src + (size_t)r * n;
    const int base = 2 * (kb + j);
    // taps in aligned pairs: (2k + t) is even for even t and M is even, so x[t + 1] follows x[t]
    float x[TAPS];
#pragma unroll
    for (int t = 0; t < TAPS; t += 2) {
      const float2 v = __ldg(reinterpret_cast<const float2*>(row + ((base + t) & m)));
      x[t] = v.x;
      x[t + 1] = v.y;
    }
    float acc = 0.f;
#pragma unroll
    for (int t = 0; t < TAPS; ++t) acc = fmaf(hic ? gf[t] : hf[t], x[t], acc);
    sY[idx] = acc;
  }
  __syncthreads();
  float* Uz = U + (size_t)z * P;
  auto put = [&](int row, int c, float w) {
    float* u = Uz + (size_t)row * n + c;
    w *= kUnionScale;
    if (MODE == MODE_UPDATE) {
      const float uo = *u;
      *u = rho * sat1(uo + kk * w) + (1.0f - rho) * uo;
    } else {
      *u = w;
    }
  };
  for (int idx = threadIdx.x; idx < H * SC; idx += blockDim.x) {
    const int q = idx >> lsc, j = idx & (SC - 1), c = k0 + j;
    float x[TAPS];
#pragma unroll
    for (int t = 0; t < TAPS; ++t) x[t] = sY[(((2 * q + t) & m) << lsc) + j];
    float lo = 0.f, hi = 0.f;
#pragma unroll
    for (int t = 0; t < TAPS; ++t) {
      lo = fmaf(hf[t], x[t], lo);
      hi = fmaf(gf[t], x[t], hi);
    }
    if (!hic && !last) ll[(size_t)z * P + (size_t)q * n + c] = lo;
    else put(q, c, lo);
    put(H + q, c, hi);
  }
}

template <int MODE>
__global__ void __launch_bounds__(256)
k_dwt_level(const float* __restrict__ src0, const float* __restrict__ llin, float* __restrict__ ll,
            float* __restrict__ U, int n, int M, int SC, int level0, int last, float kk, float rho) {
  extern __shared__ float sY[];
#define CALL(T) dwt_level_body<MODE, T>(src0, llin, ll, U, n, M, SC, level0, last, kk, rho, sY)
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
  // output rows i of this thread all have the parity of threadIdx.y (blockDim.y is even): its taps in registers
  const int par = threadIdx.y & 1;
  float he[TAPS / 2], ge[TAPS / 2];
#pragma unroll
  for (int s2 = 0; s2 < TAPS / 2; ++s2) {
    he[s2] = c_dbh[b][par + 2 * s2];
    ge[s2] = c_dbg[b][par + 2 * s2];
  }
#pragma unroll 1
  for (int j = 0; j < kColRun; ++j) {
    const int i = (blockIdx.y * kColRun + j) * blockDim.y + threadIdx.y;
    if (i >= M) break;
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
      acc = fmaf(he[s2], a[s2], acc);
      acc = fmaf(ge[s2], d[s2], acc);
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
// The first half of the block computes the even outputs i = 2u, the second
// half the odd ones, so that each thread's taps sit in registers and the
// loads of a warp are consecutive.
template <int TAPS>
__device__ __forceinline__ void idwt_rows_body(const float* __restrict__ W1, float* __restrict__ out, int n, int M) {
  const int z = blockIdx.z, b = z & 7;
  const int H = M >> 1;
  const size_t P = (size_t)n * n;
  const int half = blockDim.x >> 1, par = threadIdx.x >= half, u0 = threadIdx.x - par * half;
  float he[TAPS / 2], ge[TAPS / 2];
#pragma unroll
  for (int s2 = 0; s2 < TAPS / 2; ++s2) {
    he[s2] = c_dbh[b][par + 2 * s2];
    ge[s2] = c_dbg[b][par + 2 * s2];
  }
  const int r1 = min(M, (int)(blockIdx.y + 1) * kRowsPerBlock);
  for (int r = blockIdx.y * kRowsPerBlock; r < r1; ++r) {
    const float* src = W1 + (size_t)z * P + (size_t)r * n;
    float* dst = out + (size_t)z * P + (size_t)r * n;
    for (int u = u0; u < H; u += half) {
      float a[TAPS / 2], d[TAPS / 2];
#pragma unroll
      for (int s2 = 0; s2 < TAPS / 2; ++s2) {
        const int kk = (u - s2) & (H - 1);   // ((2u + par - par - 2 s2) mod M) / 2
        a[s2] = __ldg(src + kk);
        d[s2] = __ldg(src + H + kk);
      }
      float acc = 0.f;
#pragma unroll
      for (int s2 = 0; s2 < TAPS / 2; ++s2) {
        acc = fmaf(he[s2], a[s2], acc);
        acc = fmaf(ge[s2], d[s2], acc);
      }
      dst[2 * u + par] = acc;
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
__device__ __forceinline__ float idwt_row_value(const float* __restrict__ src, int b, int u, int par, int H) {
  float a[TAPS / 2], d[TAPS / 2];
#pragma unroll
  for (int s2 = 0; s2 < TAPS / 2; ++s2) {
    const int kk = (u - s2) & (H - 1);
    a[s2] = __ldg(src + kk);
    d[s2] = __ldg(src + H + kk);
  }
  float acc = 0.f;
#pragma unroll
  for (int s2 = 0; s2 < TAPS / 2; ++s2) {
    acc = fmaf(c_dbh[b][par + 2 * s2], a[s2], acc);   // par is the same across a warp: one broadcast read
    acc = fmaf(c_dbg[b][par + 2 * s2], d[s2], acc);
  }
  return acc;
}

// Output i = 2u + par: the first half of the block takes the even outputs, the second the odd ones.
__global__ void k_idwt_rows_sum(const float* __restrict__ W1, float* __restrict__ S, int n) {
  const int l = blockIdx.z, M = n, H = M >> 1;
  const size_t P = (size_t)n * n;
  const int half = blockDim.x >> 1, par = threadIdx.x >= half, u0 = threadIdx.x - par * half;
  const int r1 = min(M, (int)(blockIdx.y + 1) * kRowsPerBlock);
  for (int r = blockIdx.y * kRowsPerBlock; r < r1; ++r) {
    const float* src = W1 + (size_t)l * kDbBases * P + (size_t)r * n;
    for (int u = u0; u < H; u += half) {
      float acc = idwt_row_value<2>(src, 0, u, par, H);
      acc += idwt_row_value<4>(src + P, 1, u, par, H);
      acc += idwt_row_value<6>(src + 2 * P, 2, u, par, H);
      acc += idwt_row_value<8>(src + 3 * P, 3, u, par, H);
      acc += idwt_row_value<10>(src + 4 * P, 4, u, par, H);
      acc += idwt_row_value<12>(src + 5 * P, 5, u, par, H);
      acc += idwt_row_value<14>(src + 6 * P, 6, u, par, H);
      acc += idwt_row_value<16>(src + 7 * P, 7, u, par, H);
      S[(size_t)l * P + (size_t)r * n + 2 * u + par] = kUnionScale * acc;
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

// Columns per slab of the fused analysis: at most 32, at most 8192 / M (32 KB
// of shared memory), at most H.
static int dwt_slab(int M) {
  int sc = 32;
  while (sc > 1 && (sc > M / 2 || sc * M > 8192)) sc >>= 1;
  return sc;
}

cudaError_t launch_dwt_analysis(const Geom& g, const DwtArgs& a, int mode, cudaStream_t s) {
  const int n = g.n, Z = kDbBases * g.L;
  for (int j = 0; j < g.J; ++j) {
    const int M = n >> j, sc = dwt_slab(M);
    // level j reads the low-low plane level j - 1 wrote and writes its own to the other scratch plane
    const float* llin = (j & 1) ? a.W1 : a.W2;
    float* ll = (j & 1) ? a.W2 : a.W1;
    const dim3 grid(M / sc, 1, Z);
    const size_t sm = (size_t)M * sc * sizeof(float);
    const int last = j == g.J - 1;
    if (mode == MODE_UPDATE)
      k_dwt_level<MODE_UPDATE><<<grid, 256, sm, s>>>(a.src, llin, ll, a.U, n, M, sc, j == 0, last, a.k, a.rho);
    else
      k_dwt_level<MODE_LINEAR><<<grid, 256, sm, s>>>(a.src, llin, ll, a.U, n, M, sc, j == 0, last, 1.f, 1.f);
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
