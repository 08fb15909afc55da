// Isotropic undecimated wavelet transform W_s (B3 spline, a trous, periodic)
// and its exact adjoint, fused with the spatial dual step of Algorithm 1
// (third line; Eq. 11):  U <- rho sat(U + sigma mu_s W_s D) + (1 - rho) U,
// and with the spatial adjoint of the next pass (Eq. 9): S = W_s^T U.
//
// Generation 1: c_{j+1} = H_j c_j, w_j = c_j - c_{j+1}.
// Generation 2: c_{j+1} = H_j c_j, w_j = c_j - H_j c_{j+1}.
// H_j is the separable filter [1,4,6,4,1]/16 (x) itself with taps 2^j apart.
// The adjoint runs from the coarse end: r = u_J, then for j = J-1..0
//   gen 1: r <- u_j + H_j (r - u_j);   gen 2: r <- u_j + H_j (r - H_j u_j).
//
// Levels j < j1 ("fine") are computed on 64 x 64 output tiles held in shared
// memory with the halo the recursion needs.  At dilation 2^j with j >= j1 the
// filter only couples pixels of the same residue class modulo s = 2^j1, so
// levels j >= j1 ("coarse") run one class sub-image ((N/s) x (N/s), periodic)
// per block, with the planes U_j (j >= j1) stored class-permuted so that
// those blocks read and write contiguous memory.  The coarse block updates
// U_j1..U_J and, still holding them, computes r_j1 of the adjoint for the
// next pass.
#include "device.cuh"
#include "internal.h"

namespace muffin {

constexpr int kTile = 64;

__device__ __forceinline__ float hconv(const float* p, int d) {
  return 0.0625f * (p[-2 * d] + p[2 * d]) + 0.25f * (p[-d] + p[d]) + 0.375f * p[0];
}

template <int MODE>
__device__ __forceinline__ void dual_update(float* u, float w, float k, float rho, double& acc) {
  if (MODE == MODE_UPDATE) {
    const float uo = *u;
    const float ut = sat1(uo + k * w);
    *u = rho * ut + (1.0f - rho) * uo;
  } else if (MODE == MODE_LINEAR) {
    *u = w;
  } else if (MODE == MODE_NORM) {
    acc += fabs((double)w);
  }
}

// Row pass over a square region: dst rows = rows of the src region (halo es),
// dst cols = cols of the region with halo ed = es - 2d.
template <int SD, int HM>
__device__ __forceinline__ void row_pass(const float* __restrict__ src, float* __restrict__ dst, int es, int ed, int d) {
  for (int r = HM - es + (int)threadIdx.y; r < HM + kTile + es; r += blockDim.y)
    for (int c = HM - ed + (int)threadIdx.x; c < HM + kTile + ed; c += blockDim.x)
      dst[r * SD + c] = hconv(src + r * SD + c, d);
}

// ------------------------------------------------------------------ fine analysis
template <int GEN, int J1, int MODE>
__global__ void __launch_bounds__(512)
k_fine_analysis(int n, int J, IuwtArgs a) {
  constexpr int HM = halo_max(GEN, J1), SD = kTile + 2 * HM;
  extern __shared__ __align__(16) float sm[];
  __shared__ double red[32];
  float* A = sm;
  float* Tm = sm + SD * SD;
  float* B = sm + 2 * SD * SD;   // generation 2 only
  const int l = blockIdx.z, ty0 = blockIdx.y * kTile, tx0 = blockIdx.x * kTile;
  const size_t P = (size_t)n * n;
  const int m = n - 1;
  double acc = 0.0;
  {
    const int e = halo_c(GEN, J1, 0);
    const float* src = a.D + (size_t)l * P;
    for (int r = HM - e + (int)threadIdx.y; r < HM + kTile + e; r += blockDim.y) {
      const int gy = (ty0 - HM + r) & m;
      for (int c = HM - e + (int)threadIdx.x; c < HM + kTile + e; c += blockDim.x)
        A[r * SD + c] = __ldg(src + (size_t)gy * n + ((tx0 - HM + c) & m));
    }
  }
  __syncthreads();
#pragma unroll
  for (int j = 0; j < J1; ++j) {
    const int d = 1 << j;
    const int ein = halo_c(GEN, J1, j), eout = halo_c(GEN, J1, j + 1);
    float* Uj = a.U + ((size_t)l * (J + 1) + j) * P;
    row_pass<SD, HM>(A, Tm, ein, eout, d);
    __syncthreads();
    if (GEN == 1) {
      for (int r = HM - eout + (int)threadIdx.y; r < HM + kTile + eout; r += blockDim.y)
        for (int c = HM - eout + (int)threadIdx.x; c < HM + kTile + eout; c += blockDim.x) {
          const int i = r * SD + c;
          const float v = hconv(Tm + i, d * SD);
          if (r >= HM && r < HM + kTile && c >= HM && c < HM + kTile) {
            const size_t gi = (size_t)(ty0 + r - HM) * n + (tx0 + c - HM);
            dual_update<MODE>(Uj + gi, A[i] - v, a.k, a.rho, acc);
          }
          A[i] = v;
        }
      __syncthreads();
    } else {
      for (int r = HM - eout + (int)threadIdx.y; r < HM + kTile + eout; r += blockDim.y)
        for (int c = HM - eout + (int)threadIdx.x; c < HM + kTile + eout; c += blockDim.x) {
          const int i = r * SD + c;
          B[i] = hconv(Tm + i, d * SD);
        }
      __syncthreads();
      row_pass<SD, HM>(B, Tm, eout, 0, d);
      __syncthreads();
      for (int r = HM + (int)threadIdx.y; r < HM + kTile; r += blockDim.y)
        for (int c = HM + (int)threadIdx.x; c < HM + kTile; c += blockDim.x) {
          const int i = r * SD + c;
          const size_t gi = (size_t)(ty0 + r - HM) * n + (tx0 + c - HM);
          dual_update<MODE>(Uj + gi, A[i] - hconv(Tm + i, d * SD), a.k, a.rho, acc);
        }
      __syncthreads();
      float* t = A; A = B; B = t;
    }
  }
  // c_{j1} on the tile: last plane (J == j1) or hand-off to the coarse levels
  for (int r = HM + (int)threadIdx.y; r < HM + kTile; r += blockDim.y)
    for (int c = HM + (int)threadIdx.x; c < HM + kTile; c += blockDim.x) {
      const int gy = ty0 + r - HM, gx = tx0 + c - HM;
      const int ci = class_index(gy, gx, n, J1);
      const float cv = A[r * SD + c];
      if (J == J1) {
        dual_update<MODE>(a.U + ((size_t)l * (J + 1) + J) * P + ci, cv, a.k, a.rho, acc);
      } else {
        a.cr[(size_t)l * P + ci] = cv;
      }
    }
  if (MODE == MODE_NORM) {
    const double tot = block_sum(acc, red);
    if (threadIdx.x == 0 && threadIdx.y == 0)
      a.partials[((size_t)blockIdx.z * gridDim.y + blockIdx.y) * gridDim.x + blockIdx.x] = tot;
  }
}

// ------------------------------------------------------------------ fine adjoint
// rin: r_{j1} per channel (class-permuted, stride 2^j1), channel stride rin_stride.
template <int GEN, int J1>
__global__ void __launch_bounds__(512)
k_fine_adjoint(int n, int J, const float* __restrict__ rin, size_t rin_stride, IuwtArgs a) {
  constexpr int HM = halo_max(GEN, J1), SD = kTile + 2 * HM;
  extern __shared__ __align__(16) float sm[];
  float* R = sm;
  float* Ub = sm + SD * SD;
  float* Tm = sm + 2 * SD * SD;
  const int l = blockIdx.z, ty0 = blockIdx.y * kTile, tx0 = blockIdx.x * kTile;
  const size_t P = (size_t)n * n;
  const int m = n - 1;
  {
    const int e = halo_r(J1);
    const float* src = rin + (size_t)l * rin_stride;
    for (int r = HM - e + (int)threadIdx.y; r < HM + kTile + e; r += blockDim.y) {
      const int gy = (ty0 - HM + r) & m;
      for (int c = HM - e + (int)threadIdx.x; c < HM + kTile + e; c += blockDim.x)
        R[r * SD + c] = __ldg(src + class_index(gy, (tx0 - HM + c) & m, n, J1));
    }
  }
#pragma unroll
  for (int j = J1 - 1; j >= 0; --j) {
    const int d = 1 << j;
    const int er = halo_r(j + 1), eu = halo_u(GEN, j), enew = halo_r(j);
    const float* Uj = a.U + ((size_t)l * (J + 1) + j) * P;
    for (int r = HM - eu + (int)threadIdx.y; r < HM + kTile + eu; r += blockDim.y) {
      const int gy = (ty0 - HM + r) & m;
      for (int c = HM - eu + (int)threadIdx.x; c < HM + kTile + eu; c += blockDim.x)
        Ub[r * SD + c] = __ldg(Uj + (size_t)gy * n + ((tx0 - HM + c) & m));
    }
    __syncthreads();
    if (GEN == 1) {
      for (int r = HM - er + (int)threadIdx.y; r < HM + kTile + er; r += blockDim.y)
        for (int c = HM - er + (int)threadIdx.x; c < HM + kTile + er; c += blockDim.x) R[r * SD + c] -= Ub[r * SD + c];
    } else {
      row_pass<SD, HM>(Ub, Tm, eu, er, d);
      __syncthreads();
      for (int r = HM - er + (int)threadIdx.y; r < HM + kTile + er; r += blockDim.y)
        for (int c = HM - er + (int)threadIdx.x; c < HM + kTile + er; c += blockDim.x) {
          const int i = r * SD + c;
          R[i] -= hconv(Tm + i, d * SD);
        }
    }
    __syncthreads();
    row_pass<SD, HM>(R, Tm, er, enew, d);
    __syncthreads();
    for (int r = HM - enew + (int)threadIdx.y; r < HM + kTile + enew; r += blockDim.y)
      for (int c = HM - enew + (int)threadIdx.x; c < HM + kTile + enew; c += blockDim.x) {
        const int i = r * SD + c;
        Ub[i] += hconv(Tm + i, d * SD);
      }
    __syncthreads();
    float* t = R; R = Ub; Ub = t;
  }
  for (int r = HM + (int)threadIdx.y; r < HM + kTile; r += blockDim.y)
    for (int c = HM + (int)threadIdx.x; c < HM + kTile; c += blockDim.x)
      a.S[(size_t)l * P + (size_t)(ty0 + r - HM) * n + (tx0 + c - HM)] = R[r * SD + c];
}

// ------------------------------------------------------------------ coarse levels (class sub-images)
__device__ __forceinline__ void row_full(const float* __restrict__ src, float* __restrict__ dst, int M, int lgm, int d,
                                         int tid, int nth) {
  const int mm = M - 1;
  for (int i = tid; i < M * M; i += nth) {
    const int y = i >> lgm, x = i & mm;
    const float* row = src + (y << lgm);
    dst[i] = 0.0625f * (row[(x - 2 * d) & mm] + row[(x + 2 * d) & mm]) + 0.25f * (row[(x - d) & mm] + row[(x + d) & mm]) +
             0.375f * row[x];
  }
}

__device__ __forceinline__ float col_at(const float* __restrict__ t, int i, int M, int lgm, int d) {
  const int mm = M - 1;
  const int y = i >> lgm, x = i & mm;
  return 0.0625f * (t[(((y - 2 * d) & mm) << lgm) + x] + t[(((y + 2 * d) & mm) << lgm) + x]) +
         0.25f * (t[(((y - d) & mm) << lgm) + x] + t[(((y + d) & mm) << lgm) + x]) + 0.375f * t[i];
}

template <int GEN, int MODE>
__global__ void __launch_bounds__(1024)
k_coarse(int n, int J, int j1, const float* c_in, float* r_out, float* U, float k, float rho, double* partials) {
  extern __shared__ __align__(16) float sm[];
  __shared__ double red[32];
  const int M = n >> j1, lgm = __ffs(M) - 1, MM = M * M;
  float* A = sm;
  float* Tm = sm + MM;
  float* B = sm + 2 * MM;   // generation 2 only
  const int tid = threadIdx.x, nth = blockDim.x;
  const int cls = blockIdx.x, l = blockIdx.y;
  const size_t P = (size_t)n * n;
  const size_t sub = (size_t)cls * MM;
  auto plane = [&](int j) { return U + ((size_t)l * (J + 1) + j) * P + sub; };
  double acc = 0.0;
  if (MODE != MODE_ADJ) {
    const float* src = c_in + (size_t)l * P + sub;
    for (int i = tid; i < MM; i += nth) A[i] = src[i];
    __syncthreads();
    for (int j = j1; j < J; ++j) {
      const int d = 1 << (j - j1);
      float* Uj = plane(j);
      row_full(A, Tm, M, lgm, d, tid, nth);
      __syncthreads();
      if (GEN == 1) {
        for (int i = tid; i < MM; i += nth) {
          const float v = col_at(Tm, i, M, lgm, d);
          dual_update<MODE>(Uj + i, A[i] - v, k, rho, acc);
          A[i] = v;
        }
        __syncthreads();
      } else {
        for (int i = tid; i < MM; i += nth) B[i] = col_at(Tm, i, M, lgm, d);
        __syncthreads();
        row_full(B, Tm, M, lgm, d, tid, nth);
        __syncthreads();
        for (int i = tid; i < MM; i += nth) dual_update<MODE>(Uj + i, A[i] - col_at(Tm, i, M, lgm, d), k, rho, acc);
        __syncthreads();
        float* t = A; A = B; B = t;
      }
    }
    float* UJ = plane(J);
    for (int i = tid; i < MM; i += nth) {
      dual_update<MODE>(UJ + i, A[i], k, rho, acc);
      if (MODE == MODE_UPDATE) A[i] = UJ[i];
    }
    if (MODE == MODE_NORM) {
      const double tot = block_sum(acc, red);
      if (tid == 0) partials[(size_t)blockIdx.y * gridDim.x + blockIdx.x] = tot;
      return;
    }
  } else {
    const float* UJ = plane(J);
    for (int i = tid; i < MM; i += nth) A[i] = UJ[i];
  }
  __syncthreads();
  // adjoint from the coarse end down to r_{j1}
  for (int j = J - 1; j >= j1; --j) {
    const int d = 1 << (j - j1);
    const float* Uj = plane(j);
    if (GEN == 1) {
      for (int i = tid; i < MM; i += nth) A[i] -= Uj[i];
      __syncthreads();
      row_full(A, Tm, M, lgm, d, tid, nth);
      __syncthreads();
      for (int i = tid; i < MM; i += nth) A[i] = Uj[i] + col_at(Tm, i, M, lgm, d);
      __syncthreads();
    } else {
      for (int i = tid; i < MM; i += nth) B[i] = Uj[i];
      __syncthreads();
      row_full(B, Tm, M, lgm, d, tid, nth);
      __syncthreads();
      for (int i = tid; i < MM; i += nth) A[i] -= col_at(Tm, i, M, lgm, d);
      __syncthreads();
      row_full(A, Tm, M, lgm, d, tid, nth);
      __syncthreads();
      for (int i = tid; i < MM; i += nth) A[i] = B[i] + col_at(Tm, i, M, lgm, d);
      __syncthreads();
    }
  }
  float* dst = r_out + (size_t)l * P + sub;
  for (int i = tid; i < MM; i += nth) dst[i] = A[i];
}

// ------------------------------------------------------------------ J = 0 (W_s = I)
template <int MODE>
__global__ void k_u0_pointwise(const float* __restrict__ D, float* __restrict__ U, size_t total, float k, float rho,
                               double* partials) {
  __shared__ double red[32];
  double acc = 0.0;
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < total; i += (size_t)gridDim.x * blockDim.x)
    dual_update<MODE>(U + i, D[i], k, rho, acc);
  if (MODE == MODE_NORM) {
    const double tot = block_sum(acc, red);
    if (threadIdx.x == 0) partials[blockIdx.x] = tot;
  }
}

// ------------------------------------------------------------------ launchers
size_t fine_smem_bytes(const Geom& g, int adjoint) {
  const int hm = halo_max(g.gen, g.j1);
  const size_t sd = kTile + 2 * hm;
  const int planes = adjoint ? 3 : (g.gen == 1 ? 2 : 3);
  return planes * sd * sd * sizeof(float);
}

size_t coarse_smem_bytes(const Geom& g) {
  const size_t M = (size_t)(g.n >> g.j1);
  return (g.gen == 1 ? 2 : 3) * M * M * sizeof(float);
}

template <int GEN, int J1, int MODE> static cudaError_t fine_an(const Geom& g, const IuwtArgs& a, cudaStream_t s) {
  dim3 grid(g.n / kTile, g.n / kTile, g.L);
  k_fine_analysis<GEN, J1, MODE><<<grid, dim3(32, 16), fine_smem_bytes(g, 0), s>>>(g.n, g.J, a);
  return cudaGetLastError();
}

template <int GEN, int J1> static cudaError_t fine_an_mode(const Geom& g, const IuwtArgs& a, int mode, cudaStream_t s) {
  switch (mode) {
    case MODE_UPDATE: return fine_an<GEN, J1, MODE_UPDATE>(g, a, s);
    case MODE_LINEAR: return fine_an<GEN, J1, MODE_LINEAR>(g, a, s);
    case MODE_NORM: return fine_an<GEN, J1, MODE_NORM>(g, a, s);
  }
  return cudaErrorInvalidValue;
}

cudaError_t launch_fine_analysis(const Geom& g, const IuwtArgs& a, int mode, cudaStream_t s, int* nblocks) {
  if (g.J == 0) {
    const size_t total = (size_t)g.L * g.n * g.n;
    int blocks = (int)((total + 255) / 256);
    if (blocks > 4096) blocks = 4096;
    if (nblocks) *nblocks = blocks;
    switch (mode) {
      case MODE_UPDATE: k_u0_pointwise<MODE_UPDATE><<<blocks, 256, 0, s>>>(a.D, a.U, total, a.k, a.rho, a.partials); break;
      case MODE_LINEAR: k_u0_pointwise<MODE_LINEAR><<<blocks, 256, 0, s>>>(a.D, a.U, total, a.k, a.rho, a.partials); break;
      case MODE_NORM: k_u0_pointwise<MODE_NORM><<<blocks, 256, 0, s>>>(a.D, a.U, total, a.k, a.rho, a.partials); break;
      default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
  }
  if (nblocks) *nblocks = (g.n / kTile) * (g.n / kTile) * g.L;
  const int key = g.gen * 10 + g.j1;
  switch (key) {
    case 11: return fine_an_mode<1, 1>(g, a, mode, s);
    case 12: return fine_an_mode<1, 2>(g, a, mode, s);
    case 13: return fine_an_mode<1, 3>(g, a, mode, s);
    case 21: return fine_an_mode<2, 1>(g, a, mode, s);
    case 22: return fine_an_mode<2, 2>(g, a, mode, s);
    case 23: return fine_an_mode<2, 3>(g, a, mode, s);
  }
  return cudaErrorInvalidValue;
}

template <int GEN, int J1> static cudaError_t fine_adj(const Geom& g, const IuwtArgs& a, cudaStream_t s) {
  dim3 grid(g.n / kTile, g.n / kTile, g.L);
  const size_t P = (size_t)g.n * g.n;
  const bool from_u = (g.J == g.j1);
  const float* rin = from_u ? a.U + (size_t)g.J * P : a.rin;
  const size_t stride = from_u ? (size_t)(g.J + 1) * P : P;
  k_fine_adjoint<GEN, J1><<<grid, dim3(32, 16), fine_smem_bytes(g, 1), s>>>(g.n, g.J, rin, stride, a);
  return cudaGetLastError();
}

cudaError_t launch_fine_adjoint(const Geom& g, const IuwtArgs& a, cudaStream_t s) {
  switch (g.gen * 10 + g.j1) {
    case 11: return fine_adj<1, 1>(g, a, s);
    case 12: return fine_adj<1, 2>(g, a, s);
    case 13: return fine_adj<1, 3>(g, a, s);
    case 21: return fine_adj<2, 1>(g, a, s);
    case 22: return fine_adj<2, 2>(g, a, s);
    case 23: return fine_adj<2, 3>(g, a, s);
  }
  return cudaErrorInvalidValue;
}

template <int GEN, int MODE>
static cudaError_t coarse_n(const Geom& g, const float* c_in, float* r_out, float* U, float k, float rho,
                            double* partials, cudaStream_t s) {
  const int M = g.n >> g.j1;
  const int s2 = 1 << (2 * g.j1);
  int th = M * M < 1024 ? M * M : 1024;
  th = (th + 31) / 32 * 32;
  k_coarse<GEN, MODE><<<dim3(s2, g.L), th, coarse_smem_bytes(g), s>>>(g.n, g.J, g.j1, c_in, r_out, U, k, rho,
                                                                      partials);
  return cudaGetLastError();
}

cudaError_t launch_coarse(const Geom& g, const float* c_in, float* r_out, float* U, float k, float rho, int mode,
                          double* partials, cudaStream_t s, int* nblocks) {
  if (nblocks) *nblocks = (1 << (2 * g.j1)) * g.L;
#define CO(GEN)                                                                                            \
  switch (mode) {                                                                                          \
    case MODE_UPDATE: return coarse_n<GEN, MODE_UPDATE>(g, c_in, r_out, U, k, rho, partials, s);           \
    case MODE_LINEAR: return coarse_n<GEN, MODE_LINEAR>(g, c_in, r_out, U, k, rho, partials, s);           \
    case MODE_NORM: return coarse_n<GEN, MODE_NORM>(g, c_in, r_out, U, k, rho, partials, s);               \
    case MODE_ADJ: return coarse_n<GEN, MODE_ADJ>(g, c_in, r_out, U, k, rho, partials, s);                 \
  }
  if (g.gen == 1) { CO(1) } else { CO(2) }
#undef CO
  return cudaErrorInvalidValue;
}

template <int GEN> static cudaError_t cfg_gen(const Geom& g) {
  cudaError_t e;
#define SET(fn) if ((e = allow_max_dyn_smem(fn))) return e;
  if (g.J > 0 && g.j1 > 0) {
    switch (g.j1) {
      case 1: SET((k_fine_analysis<GEN, 1, 0>)) SET((k_fine_analysis<GEN, 1, 1>)) SET((k_fine_analysis<GEN, 1, 2>))
              SET((k_fine_adjoint<GEN, 1>)) break;
      case 2: SET((k_fine_analysis<GEN, 2, 0>)) SET((k_fine_analysis<GEN, 2, 1>)) SET((k_fine_analysis<GEN, 2, 2>))
              SET((k_fine_adjoint<GEN, 2>)) break;
      case 3: SET((k_fine_analysis<GEN, 3, 0>)) SET((k_fine_analysis<GEN, 3, 1>)) SET((k_fine_analysis<GEN, 3, 2>))
              SET((k_fine_adjoint<GEN, 3>)) break;
    }
  }
  if (g.J > g.j1) {
    SET((k_coarse<GEN, 0>)) SET((k_coarse<GEN, 1>)) SET((k_coarse<GEN, 2>)) SET((k_coarse<GEN, 3>))
  }
#undef SET
  return cudaSuccess;
}

cudaError_t iuwt_configure(const Geom& g) { return g.gen == 1 ? cfg_gen<1>(g) : cfg_gen<2>(g); }

}  // namespace muffin
