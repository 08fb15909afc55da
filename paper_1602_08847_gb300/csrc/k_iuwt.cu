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
// Levels j < j1 ("fine") run on 64 x 64 output tiles held in shared memory
// with the halo their recursion needs.  At dilation 2^j with j >= j1 the
// filter only couples pixels of one residue class modulo s = 2^j1, so levels
// j >= j1 ("coarse") run on class sub-images ((N/s) x (N/s), periodic), with
// the planes U_j (j >= j1) stored class-permuted so that those blocks stream
// contiguous memory.  A coarse sub-image is split over a thread-block cluster
// (1-8 blocks, one band of rows each) that keeps every coarse plane of U
// resident in shared memory; the vertical passes read their halo rows from
// the neighbouring blocks' shared memory.  It updates U_j1..U_J and, still
// holding them, computes r_j1 of the adjoint for the next pass.
//
// Every separable level is two passes over shared memory, each a sliding
// window of 8 outputs per thread held in registers: pass 1 filters along
// columns of the natural layout and writes its result transposed; pass 2
// filters along the transposed copy.  Both passes read consecutive addresses
// across a warp, and the transposed writes use odd pitches, so neither has
// bank conflicts.
#include <cooperative_groups.h>
#include <cstdlib>

#include "device.cuh"
#include "internal.h"

namespace cg = cooperative_groups;

namespace muffin {

constexpr int kTile = 64;     // fine output tile
constexpr int kQ = 8;         // outputs per thread along a window
constexpr int kFineThreads = 512;
constexpr int kCoarseThreads = 512;   // upper bound; the launch uses coarse_threads()

__device__ __forceinline__ float b3(float a, float b, float c, float d, float e) {
  return 0.0625f * (a + e) + 0.25f * (b + d) + 0.375f * c;
}

// out[i] = sum_k h_k src[(i + (k - 2) D) * stride], i < kQ.  src points at output 0.
template <int D>
__device__ __forceinline__ void win(const float* __restrict__ src, int stride, float (&out)[kQ]) {
  if constexpr (D <= 4) {
    float w[kQ + 4 * D];
#pragma unroll
    for (int t = 0; t < kQ + 4 * D; ++t) w[t] = src[(t - 2 * D) * stride];
#pragma unroll
    for (int i = 0; i < kQ; ++i) out[i] = b3(w[i], w[i + D], w[i + 2 * D], w[i + 3 * D], w[i + 4 * D]);
  } else {
#pragma unroll
    for (int i = 0; i < kQ; ++i) {
      const float* p = src + i * stride;
      out[i] = b3(p[-2 * D * stride], p[-D * stride], p[0], p[D * stride], p[2 * D * stride]);
    }
  }
}

// Same on the difference src - sub (both read at the same offsets).
template <int D>
__device__ __forceinline__ void win_diff(const float* __restrict__ src, const float* __restrict__ sub, int stride,
                                         float (&out)[kQ]) {
  if constexpr (D <= 4) {
    float w[kQ + 4 * D];
#pragma unroll
    for (int t = 0; t < kQ + 4 * D; ++t) w[t] = src[(t - 2 * D) * stride] - sub[(t - 2 * D) * stride];
#pragma unroll
    for (int i = 0; i < kQ; ++i) out[i] = b3(w[i], w[i + D], w[i + 2 * D], w[i + 3 * D], w[i + 4 * D]);
  } else {
#pragma unroll
    for (int i = 0; i < kQ; ++i) {
      const float* p = src + i * stride;
      const float* q = sub + i * stride;
      out[i] = b3(p[-2 * D * stride] - q[-2 * D * stride], p[-D * stride] - q[-D * stride], p[0] - q[0],
                  p[D * stride] - q[D * stride], p[2 * D * stride] - q[2 * D * stride]);
    }
  }
}

// Same along a periodic axis of length mm + 1: element t at base[((c0 + t) & mm) * stride].
template <int D>
__device__ __forceinline__ void win_per(const float* __restrict__ base, int stride, int c0, int mm, float (&out)[kQ]) {
  if constexpr (D <= 4) {
    float w[kQ + 4 * D];
#pragma unroll
    for (int t = 0; t < kQ + 4 * D; ++t) w[t] = base[((c0 + t - 2 * D) & mm) * stride];
#pragma unroll
    for (int i = 0; i < kQ; ++i) out[i] = b3(w[i], w[i + D], w[i + 2 * D], w[i + 3 * D], w[i + 4 * D]);
  } else {
#pragma unroll
    for (int i = 0; i < kQ; ++i) {
      const int c = c0 + i;
      out[i] = b3(base[((c - 2 * D) & mm) * stride], base[((c - D) & mm) * stride], base[(c & mm) * stride],
                  base[((c + D) & mm) * stride], base[((c + 2 * D) & mm) * stride]);
    }
  }
}

template <int MODE>
__device__ __forceinline__ void dual_update(float* u, float w, float k, float rho, double& acc) {
  if constexpr (MODE == MODE_UPDATE) {
    const float uo = *u;
    *u = rho * sat1(uo + k * w) + (1.0f - rho) * uo;
  } else if constexpr (MODE == MODE_LINEAR) {
    *u = w;
  } else if constexpr (MODE == MODE_NORM) {
    acc += fabs((double)w);
  }
}

// Update from a prefetched old value uo.
template <int MODE>
__device__ __forceinline__ void dual_update_pf(float* u, float uo, float w, float k, float rho, double& acc) {
  if constexpr (MODE == MODE_UPDATE) {
    *u = rho * sat1(uo + k * w) + (1.0f - rho) * uo;
  } else if constexpr (MODE == MODE_LINEAR) {
    *u = w;
  } else if constexpr (MODE == MODE_NORM) {
    acc += fabs((double)w);
  }
}

// ================================================================== fine levels (halo tiles)
template <int GEN, int J1> struct FineGeo {
  static constexpr int HM = halo_max(GEN, J1);
  static constexpr int SD = kTile + 2 * HM;      // region side
  static constexpr int PA = SD + 1;              // pitch of natural-layout buffers (odd)
  static constexpr int RA = SD;                  // rows allocated
  static constexpr int PT = SD + 1;              // pitch of the transposed buffer (odd)
  static constexpr int PI = kTile + 1;           // pitch of the interior buffer
  static constexpr int NA = RA * PA, NT = RA * PT, NI = kTile * PI;
};

// pass 1: vertical filter of X over rows of region eo, columns of region ei -> T (transposed)
// The last window of a row or column is moved back to end on the region's
// edge (regions are at least kQ wide), so no window reads or writes past the
// buffers; outputs it shares with the previous window are written once.
template <int HM, int PA, int PT, int D>
__device__ __forceinline__ void fine_pass1(const float* __restrict__ X, float* __restrict__ T, int ei, int eo) {
  const int ncol = kTile + 2 * ei, nseg = (kTile + 2 * eo + kQ - 1) / kQ, rend = HM + kTile + eo;
  for (int it = threadIdx.x; it < ncol * nseg; it += blockDim.x) {
    const int c = HM - ei + it % ncol, r0o = HM - eo + (it / ncol) * kQ;
    const int r0 = r0o + kQ <= rend ? r0o : rend - kQ;
    float o[kQ];
    win<D>(X + r0 * PA + c, PA, o);
#pragma unroll
    for (int i = 0; i < kQ; ++i)
      if (r0 + i >= r0o) T[c * PT + r0 + i] = o[i];
  }
}

// pass 1 on the difference X - Y (gen-1 adjoint: H_j (r - u_j) without storing r - u_j)
template <int HM, int PA, int PT, int D>
__device__ __forceinline__ void fine_pass1_diff(const float* __restrict__ X, const float* __restrict__ Y,
                                                float* __restrict__ T, int ei, int eo) {
  const int ncol = kTile + 2 * ei, nseg = (kTile + 2 * eo + kQ - 1) / kQ, rend = HM + kTile + eo;
  for (int it = threadIdx.x; it < ncol * nseg; it += blockDim.x) {
    const int c = HM - ei + it % ncol, r0o = HM - eo + (it / ncol) * kQ;
    const int r0 = r0o + kQ <= rend ? r0o : rend - kQ;
    float o[kQ];
    win_diff<D>(X + r0 * PA + c, Y + r0 * PA + c, PA, o);
#pragma unroll
    for (int i = 0; i < kQ; ++i)
      if (r0 + i >= r0o) T[c * PT + r0 + i] = o[i];
  }
}

// pass 2: horizontal filter through T over rows of region er, columns of region ec
template <int HM, int PT, int D, typename F>
__device__ __forceinline__ void fine_pass2(const float* __restrict__ T, int er, int ec, F&& epi) {
  const int nrow = kTile + 2 * er, ncs = (kTile + 2 * ec + kQ - 1) / kQ, cend = HM + kTile + ec;
  for (int it = threadIdx.x; it < nrow * ncs; it += blockDim.x) {
    const int r = HM - er + it % nrow, c0o = HM - ec + (it / nrow) * kQ;
    const int c0 = c0o + kQ <= cend ? c0o : cend - kQ;
    float o[kQ];
    win<D>(T + c0 * PT + r, PT, o);
#pragma unroll
    for (int i = 0; i < kQ; ++i)
      if (c0 + i >= c0o) epi(r, c0 + i, o[i]);
  }
}

// Asynchronous 4-byte copy global -> shared (cp.async): a thread issues all
// of its copies before waiting once, so all of them are in flight together and
// none passes through registers.
__device__ __forceinline__ void cp_async4(float* dst, const float* src) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"((uint32_t)__cvta_generic_to_shared(dst)), "l"(src)
               : "memory");
}
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_all;" ::: "memory"); }

// Load the square region of side 64 + 2E around the tile (periodic wrap) of a
// natural-layout plane into X: warps take rows, lanes take columns.  The
// wrapped column offsets of a lane are the same on every row, so they are
// formed once; the rows are unrolled so that all of a thread's loads are in
// flight together.
template <int HM, int PA, int E, int NTH>
__device__ __forceinline__ void load_region(float* __restrict__ X, const float* __restrict__ plane, int n, int ty0,
                                            int tx0) {
  constexpr int SIDE = kTile + 2 * E, NQ = (SIDE + 31) / 32, NW = NTH / 32, RPW = (SIDE + NW - 1) / NW;
  const int m = n - 1, lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  int cofs[NQ];
#pragma unroll
  for (int q = 0; q < NQ; ++q) cofs[q] = (tx0 - E + lane + 32 * q) & m;
  float* xb = X + (HM - E) * PA + HM - E + lane;
#pragma unroll
  for (int k = 0; k < RPW; ++k) {
    const int r = w + k * NW;
    if (r < SIDE) {
      const float* srow = plane + (size_t)((ty0 - E + r) & m) * n;
#pragma unroll
      for (int q = 0; q < NQ; ++q)
        if (lane + 32 * q < SIDE) xb[r * PA + 32 * q] = __ldg(srow + cofs[q]);
    }
  }
}

// Same from a class-permuted plane (stride 2^lgs): element (gy, gx) sits at
// ((gy & s1) s + (gx & s1)) mc^2 + (gy >> lgs) mc + (gx >> lgs), a row part
// plus a column part.
template <int HM, int PA, int E, int NTH>
__device__ __forceinline__ void load_region_class(float* __restrict__ X, const float* __restrict__ plane, int n,
                                                  int lgs, int ty0, int tx0) {
  constexpr int SIDE = kTile + 2 * E, NQ = (SIDE + 31) / 32, NW = NTH / 32, RPW = (SIDE + NW - 1) / NW;
  const int m = n - 1, lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const int s1 = (1 << lgs) - 1, mc = n >> lgs;
  const size_t mc2 = (size_t)mc * mc;
  size_t cofs[NQ];
#pragma unroll
  for (int q = 0; q < NQ; ++q) {
    const int gx = (tx0 - E + lane + 32 * q) & m;
    cofs[q] = (size_t)(gx & s1) * mc2 + (gx >> lgs);
  }
  float* xb = X + (HM - E) * PA + HM - E + lane;
#pragma unroll
  for (int k = 0; k < RPW; ++k) {
    const int r = w + k * NW;
    if (r < SIDE) {
      const int gy = (ty0 - E + r) & m;
      const float* srow = plane + ((size_t)(gy & s1) << lgs) * mc2 + (size_t)(gy >> lgs) * mc;
#pragma unroll
      for (int q = 0; q < NQ; ++q)
        if (lane + 32 * q < SIDE) xb[r * PA + 32 * q] = __ldg(srow + cofs[q]);
    }
  }
}

// Square region of side S (compile time, <= 128) centred on the tile: warps
// take rows, lanes take columns, f(r, c) with region-relative r, c.
template <int S, typename F>
__device__ __forceinline__ void region_for(F&& f) {
  const int lane = threadIdx.x & 31, nw = blockDim.x >> 5;
  for (int r = threadIdx.x >> 5; r < S; r += nw) {
#pragma unroll
    for (int q = 0; q < (S + 31) / 32; ++q) {
      const int c = lane + 32 * q;
      if (c < S) f(r, c);
    }
  }
}

// Interior pixel k (k < 4096 / NT) of this thread: row, column inside the 64 x 64 tile.
template <int NT> __device__ __forceinline__ int int_row(int k) { return (int)threadIdx.x / kTile + (NT / kTile) * k; }
__device__ __forceinline__ int int_col() { return (int)threadIdx.x % kTile; }

template <int GEN, int J1, int MODE, int J0, int NTH = kFineThreads>
__device__ __forceinline__ void fine_analysis_level(float*& A, float*& B, float* T, float* Bi, float (&up)[J1 + 1][8],
                                                    const IuwtArgs& a, int n, int J, int l, int ty0, int tx0,
                                                    double& acc) {
  using G = FineGeo<GEN, J1>;
  constexpr int HM = G::HM, PA = G::PA, PT = G::PT, PI = G::PI, D = 1 << J0;
  constexpr int ei = halo_c(GEN, J1, J0), eo = halo_c(GEN, J1, J0 + 1);
  fine_pass1<HM, PA, PT, D>(A, T, ei, eo);
  __syncthreads();
  if constexpr (GEN == 1) {
    fine_pass2<HM, PT, D>(T, eo, eo, [&](int r, int c, float v) {
      if (r >= HM && r < HM + kTile && c >= HM && c < HM + kTile) Bi[(r - HM) * PI + (c - HM)] = v;
      else A[r * PA + c] = v;
    });
  } else {
    fine_pass2<HM, PT, D>(T, eo, eo, [&](int r, int c, float v) { B[r * PA + c] = v; });
    __syncthreads();
    fine_pass1<HM, PA, PT, D>(B, T, eo, 0);
    __syncthreads();
    fine_pass2<HM, PT, D>(T, 0, 0, [&](int r, int c, float v) { Bi[(r - HM) * PI + (c - HM)] = v; });
  }
  __syncthreads();
  const size_t P = (size_t)n * n;
  float* Uj = a.U + ((size_t)l * (J + 1) + J0) * P;
  const int ci = int_col();
#pragma unroll
  for (int k = 0; k < 8; ++k) {
    const int ri = int_row<NTH>(k);
    const int i = (HM + ri) * PA + HM + ci;
    const float v = Bi[ri * PI + ci];
    dual_update_pf<MODE>(Uj + (size_t)(ty0 + ri) * n + (tx0 + ci), up[J0][k], A[i] - v, a.k, a.rho, acc);
    if constexpr (GEN == 1) A[i] = v;
  }
  __syncthreads();
  if constexpr (GEN == 2) { float* t = A; A = B; B = t; }
  if constexpr (J0 + 1 < J1) fine_analysis_level<GEN, J1, MODE, J0 + 1>(A, B, T, Bi, up, a, n, J, l, ty0, tx0, acc);
}

template <int GEN, int J1, int MODE>
__global__ void __launch_bounds__(kFineThreads, 2)
k_fine_analysis(int n, int J, IuwtArgs a) {
  constexpr int NTH = kFineThreads;
  using G = FineGeo<GEN, J1>;
  constexpr int HM = G::HM, PA = G::PA;
  extern __shared__ __align__(16) float sm[];
  __shared__ double red[32];
  float* A = sm;
  float* T = A + G::NA;
  float* Bi = T + G::NT;
  float* B = Bi + G::NI;   // generation 2 only
  const int l = blockIdx.z, ty0 = blockIdx.y * kTile, tx0 = blockIdx.x * kTile;
  const size_t P = (size_t)n * n;
  double acc = 0.0;
  // prefetch the tile's dual values; their latency hides behind the filtering
  float up[J1 + 1][8];
  const int ci = int_col();
#pragma unroll
  for (int k = 0; k < 8; ++k) {
    const int ri = int_row<NTH>(k);
#pragma unroll
    for (int j = 0; j <= J1; ++j) up[j][k] = 0.0f;
    if constexpr (MODE == MODE_UPDATE) {
#pragma unroll
      for (int j = 0; j < J1; ++j) up[j][k] = __ldg(a.U + ((size_t)l * (J + 1) + j) * P + (size_t)(ty0 + ri) * n + tx0 + ci);
      if (J == J1)
        up[J1][k] = __ldg(a.U + ((size_t)l * (J + 1) + J) * P + class_index(ty0 + ri, tx0 + ci, n, J1));
    }
  }
  load_region<HM, PA, HM, NTH>(A, a.D + (size_t)l * P, n, ty0, tx0);
  __syncthreads();
  if constexpr (J1 > 0) fine_analysis_level<GEN, J1, MODE, 0>(A, B, T, Bi, up, a, n, J, l, ty0, tx0, acc);
  // c_{j1} on the tile: last plane (J == j1) or hand-off to the coarse levels
#pragma unroll
  for (int k = 0; k < 8; ++k) {
    const int ri = int_row<NTH>(k);
    const int gy = ty0 + ri, gx = tx0 + ci;
    const int cidx = class_index(gy, gx, n, J1);
    const float cv = A[(HM + ri) * PA + HM + ci];
    if (J == J1) dual_update_pf<MODE>(a.U + ((size_t)l * (J + 1) + J) * P + cidx, up[J1][k], cv, a.k, a.rho, acc);
    else a.cr[(size_t)l * P + cidx] = cv;
  }
  if constexpr (MODE == MODE_NORM) {
    const double tot = block_sum(acc, red);
    if (threadIdx.x == 0) a.partials[((size_t)blockIdx.z * gridDim.y + blockIdx.y) * gridDim.x + blockIdx.x] = tot;
  }
}

// ------------------------------------------------------------------ fine adjoint
template <int GEN, int J1, int J0, int NTH>
__device__ __forceinline__ void fine_adjoint_level(float*& R, float*& Ub, float* T, const IuwtArgs& a, int n, int J,
                                                   int l, int ty0, int tx0) {
  using G = FineGeo<GEN, J1>;
  constexpr int HM = G::HM, PA = G::PA, PT = G::PT, D = 1 << J0;
  constexpr int er = halo_r(J0 + 1), en = halo_r(J0), eu = halo_u(GEN, J0);
  // prefetch u_{J0-1} for the next level into registers while this level filters:
  // thread (warp w, lane) takes rows w + NW k and columns lane + 32 q of that region
  constexpr int eun = J0 > 0 ? halo_u(GEN, J0 - 1) : 0;
  constexpr int sidn = kTile + 2 * eun, NW = NTH / 32;
  constexpr int NR = J0 > 0 ? (sidn + NW - 1) / NW : 1, NQ = J0 > 0 ? (sidn + 31) / 32 : 1;
  float pf[NR][NQ];
  const int lane = threadIdx.x & 31, wrp = threadIdx.x >> 5;
  const int m = n - 1;
  if constexpr (J0 > 0) {
    const float* Un = a.U + ((size_t)l * (J + 1) + J0 - 1) * (size_t)n * n;
    int cofs[NQ];
#pragma unroll
    for (int q = 0; q < NQ; ++q) cofs[q] = (tx0 - eun + lane + 32 * q) & m;
#pragma unroll
    for (int k = 0; k < NR; ++k) {
      const int r = wrp + NW * k;
      const float* srow = Un + (size_t)((ty0 - eun + r) & m) * n;
#pragma unroll
      for (int q = 0; q < NQ; ++q) {
        const int c = lane + 32 * q;
        pf[k][q] = (r < sidn && c < sidn) ? __ldg(srow + cofs[q]) : 0.0f;
      }
    }
  }
  if constexpr (GEN == 1) {
    fine_pass1_diff<HM, PA, PT, D>(R, Ub, T, er, en);     // H_j (r - u_j), first pass
  } else {
    fine_pass1<HM, PA, PT, D>(Ub, T, eu, er);
    __syncthreads();
    fine_pass2<HM, PT, D>(T, er, er, [&](int r, int c, float v) { R[r * PA + c] -= v; });
    __syncthreads();
    fine_pass1<HM, PA, PT, D>(R, T, er, en);
  }
  __syncthreads();
  fine_pass2<HM, PT, D>(T, en, en, [&](int r, int c, float v) { Ub[r * PA + c] += v; });
  __syncthreads();
  { float* t = R; R = Ub; Ub = t; }
  if constexpr (J0 > 0) {
#pragma unroll
    for (int k = 0; k < NR; ++k) {
      const int r = wrp + NW * k;
      float* drow = Ub + (HM - eun + r) * PA + HM - eun;
#pragma unroll
      for (int q = 0; q < NQ; ++q) {
        const int c = lane + 32 * q;
        if (r < sidn && c < sidn) drow[c] = pf[k][q];
      }
    }
    __syncthreads();
    fine_adjoint_level<GEN, J1, J0 - 1, NTH>(R, Ub, T, a, n, J, l, ty0, tx0);
  }
}

// rin: r_{j1} per channel (class-permuted, stride 2^j1), channel stride rin_stride.
// NTH threads: 1024 when the block's shared memory leaves room for one block per SM.
template <int GEN, int J1, int NTH>
__global__ void __launch_bounds__(NTH)
k_fine_adjoint(int n, int J, const float* __restrict__ rin, size_t rin_stride, IuwtArgs a) {
  using G = FineGeo<GEN, J1>;
  constexpr int HM = G::HM, PA = G::PA;
  extern __shared__ __align__(16) float sm[];
  float* R = sm;
  float* Ub = R + G::NA;
  float* T = Ub + G::NA;
  const int l = blockIdx.z, ty0 = blockIdx.y * kTile, tx0 = blockIdx.x * kTile;
  const size_t P = (size_t)n * n;
  load_region_class<HM, PA, halo_r(J1), NTH>(R, rin + (size_t)l * rin_stride, n, J1, ty0, tx0);
  load_region<HM, PA, halo_u(GEN, J1 - 1), NTH>(Ub, a.U + ((size_t)l * (J + 1) + J1 - 1) * P, n, ty0, tx0);
  __syncthreads();
  fine_adjoint_level<GEN, J1, J1 - 1, NTH>(R, Ub, T, a, n, J, l, ty0, tx0);
  const int ci = int_col();
#pragma unroll
  for (int k = 0; k < 4096 / NTH; ++k) {
    const int ri = int_row<NTH>(k);
    a.S[(size_t)l * P + (size_t)(ty0 + ri) * n + tx0 + ci] = R[(HM + ri) * PA + HM + ci];
  }
}

// ================================================================== coarse levels, cluster-resident
// Index arithmetic here uses only shifts and masks (M and the band height are
// powers of two): an integer division per element would cost more issue
// slots than the filtering itself.
struct CoarseGeo {
  int M, RPC, HR, PA, PT, nU, lgM, lgR;
  size_t NA, NT, NU;   // floats of one A/B buffer, of T, of one U plane
};

__host__ __device__ inline int ilog2i(int v) {
  int r = 0;
  while ((1 << r) < v) ++r;
  return r;
}

__host__ __device__ inline CoarseGeo coarse_geo(int n, int J, int j1, int cs) {
  CoarseGeo g;
  g.M = n >> j1;
  g.RPC = g.M / cs;
  const int dmax = J - 1 - j1 >= 0 ? (1 << (J - 1 - j1)) : 0;
  g.HR = 2 * dmax;
  g.PA = g.M + 1;
  g.PT = g.RPC + 1;
  g.nU = J - j1 + 1;
  g.lgM = ilog2i(g.M);
  g.lgR = ilog2i(g.RPC);
  g.NA = (size_t)(g.RPC + 2 * g.HR) * g.PA;
  g.NT = (size_t)g.M * g.PT;
  g.NU = (size_t)g.RPC * g.PA;
  return g;
}

size_t coarse_cl_smem_bytes(int n, int J, int gen, int j1, int cs) {
  const CoarseGeo g = coarse_geo(n, J, j1, cs);
  return ((gen == 2 ? 2 : 1) * g.NA + g.NT + g.nU * g.NU) * sizeof(float);
}

// For every element (r, c) of this block's band (RPC x M): f(r, c).  Thread
// tid keeps column tid mod M and walks rows (blockDim.x is a multiple of M).
template <typename F>
__device__ __forceinline__ void band_for(const CoarseGeo& g, F&& f) {
  const int c = threadIdx.x & (g.M - 1), rstep = blockDim.x >> g.lgM;
#pragma unroll 4
  for (int r = threadIdx.x >> g.lgM; r < g.RPC; r += rstep) f(r, c);
}

// Copy the 2d rows above and below this block's band from the blocks that own
// them.  Remote (distributed shared memory) loads are issued in batches of 8
// into registers before any store: a store between them would serialise the
// loads, since local and remote shared pointers may alias.
__device__ __forceinline__ void halo_exchange(cg::cluster_group& cl, float* X, int d, const CoarseGeo& g, int rank) {
  if (g.RPC == g.M) {
    // one block holds the whole sub-image: the halo rows are its own rows, wrapped
    __syncthreads();
    const int h2 = 2 * d, mm = g.M - 1, c = threadIdx.x & mm, step = blockDim.x >> g.lgM;
    for (int hh = threadIdx.x >> g.lgM; hh < 2 * h2; hh += step) {
      const int srow = (hh < h2 ? hh - h2 : g.M + hh - h2) & mm;
      const int erow = hh < h2 ? g.HR - h2 + hh : g.HR + g.M + hh - h2;
      X[erow * g.PA + c] = X[(g.HR + srow) * g.PA + c];
    }
    __syncthreads();
    return;
  }
  cl.sync();
  const int h2 = 2 * d, row0 = rank * g.RPC, mm = g.M - 1;
  const int c = threadIdx.x & mm, step = blockDim.x >> g.lgM, nrows = 2 * h2;
  for (int hb = threadIdx.x >> g.lgM; hb < nrows; hb += 8 * step) {
    float v[8];
    int er[8];
#pragma unroll
    for (int b = 0; b < 8; ++b) {
      const int hh = hb + b * step;
      er[b] = -1;
      v[b] = 0.0f;
      if (hh < nrows) {
        int srow;
        if (hh < h2) { srow = row0 - h2 + hh; er[b] = g.HR - h2 + hh; }
        else { srow = row0 + g.RPC + hh - h2; er[b] = g.HR + g.RPC + hh - h2; }
        srow &= mm;
        const int owner = srow >> g.lgR, lr = srow & (g.RPC - 1);
        v[b] = cl.map_shared_rank(X, owner)[(g.HR + lr) * g.PA + c];
      }
    }
#pragma unroll
    for (int b = 0; b < 8; ++b)
      if (er[b] >= 0) X[er[b] * g.PA + c] = v[b];
  }
  cl.sync();
}

// Stream one band (RPC x M, row-major with stride M) from global memory into a
// pitched shared buffer by asynchronous copies (cp_async_wait() and a barrier
// before it is read), so the bands of every plane are in flight together.
__device__ __forceinline__ void band_load(float* __restrict__ dst, int pitch, const float* __restrict__ src,
                                          const CoarseGeo& g) {
  const int c = threadIdx.x & (g.M - 1), rstep = blockDim.x >> g.lgM;
  for (int r = threadIdx.x >> g.lgM; r < g.RPC; r += rstep) cp_async4(dst + r * pitch + c, src + (r << g.lgM) + c);
}

// Both passes of one level at dilation D over the band of X (halo rows
// already in place); epi(r, c0, o) receives 8 outputs of row r from column c0.
template <int D, typename F>
__device__ __forceinline__ void coarse_level(const float* __restrict__ X, float* __restrict__ T, const CoarseGeo& g,
                                             F&& epi) {
  const int mm = g.M - 1;
  {
    const int c = threadIdx.x & mm, step = blockDim.x >> g.lgM, nseg = g.RPC >> 3;
    for (int seg = threadIdx.x >> g.lgM; seg < nseg; seg += step) {
      float o[kQ];
      win<D>(X + (g.HR + seg * kQ) * g.PA + c, g.PA, o);
      float* q = T + c * g.PT + seg * kQ;
#pragma unroll
      for (int i = 0; i < kQ; ++i) q[i] = o[i];
    }
  }
  __syncthreads();
  {
    const int r = threadIdx.x & (g.RPC - 1), step = blockDim.x >> g.lgR, ncs = g.M >> 3;
    for (int cs = threadIdx.x >> g.lgR; cs < ncs; cs += step) {
      const int c0 = cs * kQ;
      float o[kQ];
      if (c0 >= 2 * D && c0 + kQ + 2 * D <= g.M) win<D>(T + c0 * g.PT + r, g.PT, o);
      else win_per<D>(T + r, g.PT, c0, mm, o);
      epi(r, c0, o);
    }
  }
  __syncthreads();
}

// halo exchange of X for dilation d, then both passes with epilogue epi
template <typename F>
__device__ __forceinline__ void coarse_filter(cg::cluster_group& cl, float* X, float* T, int d, const CoarseGeo& g,
                                              int rank, F&& epi) {
  halo_exchange(cl, X, d, g, rank);
  switch (d) {
    case 1: coarse_level<1>(X, T, g, epi); break;
    case 2: coarse_level<2>(X, T, g, epi); break;
    case 4: coarse_level<4>(X, T, g, epi); break;
    case 8: coarse_level<8>(X, T, g, epi); break;
    case 16: coarse_level<16>(X, T, g, epi); break;
    case 32: coarse_level<32>(X, T, g, epi); break;
    case 64: coarse_level<64>(X, T, g, epi); break;
    default: coarse_level<128>(X, T, g, epi); break;
  }
}

// MT > 0: a single-block instance for class sub-images of MT x MT (cs = 1),
// whose geometry is known at compile time, so that every shared-memory stencil
// address is a base plus immediate offsets.
template <int GEN, int MODE, int MT = 0>
__global__ void __launch_bounds__(kCoarseThreads)
k_coarse_cl(int n, int J, int j1, int cs, const float* __restrict__ c_in, float* __restrict__ r_out,
            float* __restrict__ U, float k, float rho, double* __restrict__ partials) {
  cg::cluster_group cl = cg::this_cluster();
  const int rank = (int)cl.block_rank();
  CoarseGeo g = coarse_geo(n, J, j1, cs);
  if constexpr (MT > 0) {
    constexpr int lg = MT == 32 ? 5 : MT == 64 ? 6 : 7;
    g.M = MT; g.RPC = MT; g.PA = MT + 1; g.PT = MT + 1; g.lgM = lg; g.lgR = lg;
    g.NA = (size_t)(MT + 2 * g.HR) * (MT + 1);
    g.NT = (size_t)MT * (MT + 1);
    g.NU = (size_t)MT * (MT + 1);
    cs = 1;
  }
  extern __shared__ __align__(16) float sm[];
  __shared__ double red[32];
  float* A = sm;
  float* B = A + g.NA;                          // generation 2 only
  float* T = A + (GEN == 2 ? 2 : 1) * g.NA;
  float* Us = T + g.NT;
  const int cls = blockIdx.x / cs, l = blockIdx.y;
  const size_t P = (size_t)n * n;
  const size_t sub = (size_t)cls * g.M * g.M + (size_t)rank * g.RPC * g.M;
  const int PA = g.PA, HR = g.HR;
  auto gplane = [&](int j) { return U + ((size_t)l * (J + 1) + j) * P + sub; };
  auto us = [&](int j) { return Us + (size_t)(j - j1) * g.NU; };
  // --- loads: the band of c_j1 and every coarse plane of U, all in flight at once
  if constexpr (MODE != MODE_ADJ) {
    band_load(A + HR * PA, PA, c_in + (size_t)l * P + sub, g);
  }
  if constexpr (MODE == MODE_UPDATE || MODE == MODE_ADJ) {
    for (int j = j1; j <= J; ++j) band_load(us(j), PA, gplane(j), g);
  }
  cp_async_wait();
  __syncthreads();
  double acc = 0.0;
  if constexpr (MODE != MODE_ADJ) {
    for (int j = j1; j < J; ++j) {
      const int d = 1 << (j - j1);
      float* Uj = us(j);
      if constexpr (GEN == 1) {
        coarse_filter(cl, A, T, d, g, rank, [&](int r, int c0, const float (&o)[kQ]) {
          float* ar = A + (HR + r) * PA + c0;
          float* ur = Uj + r * PA + c0;
#pragma unroll
          for (int i = 0; i < kQ; ++i) {
            dual_update<MODE>(ur + i, ar[i] - o[i], k, rho, acc);
            ar[i] = o[i];
          }
        });
      } else {
        coarse_filter(cl, A, T, d, g, rank, [&](int r, int c0, const float (&o)[kQ]) {
          float* br = B + (HR + r) * PA + c0;
#pragma unroll
          for (int i = 0; i < kQ; ++i) br[i] = o[i];
        });
        coarse_filter(cl, B, T, d, g, rank, [&](int r, int c0, const float (&o)[kQ]) {
          const float* ar = A + (HR + r) * PA + c0;
          float* ur = Uj + r * PA + c0;
#pragma unroll
          for (int i = 0; i < kQ; ++i) dual_update<MODE>(ur + i, ar[i] - o[i], k, rho, acc);
        });
        float* t = A; A = B; B = t;
      }
    }
    float* UJ = us(J);
    band_for(g, [&](int r, int c) {
      float* ap = A + (HR + r) * PA + c;
      dual_update<MODE>(UJ + r * PA + c, *ap, k, rho, acc);
      if constexpr (MODE == MODE_UPDATE) *ap = UJ[r * PA + c];
    });
    if constexpr (MODE == MODE_NORM) {
      const double tot = block_sum(acc, red);
      if (threadIdx.x == 0) partials[(size_t)blockIdx.y * gridDim.x + blockIdx.x] = tot;
      if (cs > 1) cl.sync();
      return;
    }
  } else {
    const float* UJ = us(J);
    band_for(g, [&](int r, int c) { A[(HR + r) * PA + c] = UJ[r * PA + c]; });
  }
  __syncthreads();
  // --- adjoint from the coarse end down to r_j1
  for (int j = J - 1; j >= j1; --j) {
    const int d = 1 << (j - j1);
    const float* Uj = us(j);
    auto finish = [&](int r, int c0, const float (&o)[kQ]) {
      float* ar = A + (HR + r) * PA + c0;
      const float* ur = Uj + r * PA + c0;
#pragma unroll
      for (int i = 0; i < kQ; ++i) ar[i] = ur[i] + o[i];
    };
    if constexpr (GEN == 1) {
      band_for(g, [&](int r, int c) { A[(HR + r) * PA + c] -= Uj[r * PA + c]; });
      coarse_filter(cl, A, T, d, g, rank, finish);
    } else {
      band_for(g, [&](int r, int c) { B[(HR + r) * PA + c] = Uj[r * PA + c]; });
      coarse_filter(cl, B, T, d, g, rank, [&](int r, int c0, const float (&o)[kQ]) {
        float* ar = A + (HR + r) * PA + c0;
#pragma unroll
        for (int i = 0; i < kQ; ++i) ar[i] -= o[i];
      });
      coarse_filter(cl, A, T, d, g, rank, finish);
    }
  }
  // --- stores: r_j1 band, and the updated coarse planes
  {
    float* dst = r_out + (size_t)l * P + sub;
    band_for(g, [&](int r, int c) { dst[(r << g.lgM) + c] = A[(HR + r) * PA + c]; });
  }
  if constexpr (MODE == MODE_UPDATE || MODE == MODE_LINEAR) {
    for (int j = j1; j <= J; ++j) {
      float* dst = gplane(j);
      const float* src = us(j);
      band_for(g, [&](int r, int c) { dst[(r << g.lgM) + c] = src[r * PA + c]; });
    }
  }
  if (cs > 1) cl.sync();   // no block leaves while a neighbour may still read its shared memory
}

// ================================================================== coarse levels, streaming fallback
// One block per class sub-image with two (three) planes in shared memory; the
// dual planes stream from global memory.  Used when no cluster split fits.
__device__ __forceinline__ void row_full(const float* __restrict__ src, float* __restrict__ dst, int M, int lgm, int d,
                                         int tid, int nth) {
  const int mm = M - 1;
  for (int i = tid; i < M * M; i += nth) {
    const int y = i >> lgm, x = i & mm;
    const float* row = src + (y << lgm);
    dst[i] = b3(row[(x - 2 * d) & mm], row[(x - d) & mm], row[x], row[(x + d) & mm], row[(x + 2 * d) & mm]);
  }
}

__device__ __forceinline__ float col_at(const float* __restrict__ t, int i, int M, int lgm, int d) {
  const int mm = M - 1;
  const int y = i >> lgm, x = i & mm;
  return b3(t[(((y - 2 * d) & mm) << lgm) + x], t[(((y - d) & mm) << lgm) + x], t[i], t[(((y + d) & mm) << lgm) + x],
            t[(((y + 2 * d) & mm) << lgm) + x]);
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
  if constexpr (MODE != MODE_ADJ) {
    const float* src = c_in + (size_t)l * P + sub;
    for (int i = tid; i < MM; i += nth) A[i] = src[i];
    __syncthreads();
    for (int j = j1; j < J; ++j) {
      const int d = 1 << (j - j1);
      float* Uj = plane(j);
      row_full(A, Tm, M, lgm, d, tid, nth);
      __syncthreads();
      if constexpr (GEN == 1) {
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
      if constexpr (MODE == MODE_UPDATE) A[i] = UJ[i];
    }
    if constexpr (MODE == MODE_NORM) {
      const double tot = block_sum(acc, red);
      if (tid == 0) partials[(size_t)blockIdx.y * gridDim.x + blockIdx.x] = tot;
      return;
    }
  } else {
    const float* UJ = plane(J);
    for (int i = tid; i < MM; i += nth) A[i] = UJ[i];
  }
  __syncthreads();
  for (int j = J - 1; j >= j1; --j) {
    const int d = 1 << (j - j1);
    const float* Uj = plane(j);
    if constexpr (GEN == 1) {
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

// ================================================================== J = 0 (W_s = I)
template <int MODE>
__global__ void k_u0_pointwise(const float* __restrict__ D, float* __restrict__ U, size_t total, float k, float rho,
                               double* partials) {
  __shared__ double red[32];
  double acc = 0.0;
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < total; i += (size_t)gridDim.x * blockDim.x)
    dual_update<MODE>(U + i, D[i], k, rho, acc);
  if constexpr (MODE == MODE_NORM) {
    const double tot = block_sum(acc, red);
    if (threadIdx.x == 0) partials[blockIdx.x] = tot;
  }
}

// ================================================================== host side
size_t fine_smem_bytes(int gen, int j1, int adjoint) {
  const int hm = halo_max(gen, j1);
  const size_t sd = kTile + 2 * hm, pa = sd + 1, ra = sd, pt = sd + 1, ni = (size_t)kTile * (kTile + 1);
  const size_t na = ra * pa, nt = ra * pt;
  const size_t floats = adjoint ? 2 * na + nt : (gen == 1 ? na + nt + ni : 2 * na + nt + ni);
  return floats * sizeof(float);
}

size_t coarse_stream_smem_bytes(int n, int gen, int j1) {
  const size_t M = (size_t)(n >> j1);
  return (gen == 1 ? 2 : 3) * M * M * sizeof(float);
}

int coarse_cluster_size(int n, int J, int gen, int j1, size_t budget) {
  const int M = n >> j1;
  for (int cs = 1; cs <= 8; cs *= 2) {
    const int rpc = M / cs;
    if (rpc < kQ || rpc % kQ != 0) break;
    if (coarse_cl_smem_bytes(n, J, gen, j1, cs) <= budget) return cs;
  }
  return 0;
}

size_t fine_smem_bytes(const Geom& g, int adjoint) { return fine_smem_bytes(g.gen, g.j1, adjoint); }

size_t coarse_smem_bytes(const Geom& g) {
  return g.cs > 0 ? coarse_cl_smem_bytes(g.n, g.J, g.gen, g.j1, g.cs) : coarse_stream_smem_bytes(g.n, g.gen, g.j1);
}

template <int GEN, int J1, int MODE> static cudaError_t fine_an(const Geom& g, const IuwtArgs& a, cudaStream_t s) {
  dim3 grid(g.n / kTile, g.n / kTile, g.L);
  k_fine_analysis<GEN, J1, MODE><<<grid, kFineThreads, fine_smem_bytes(g, 0), s>>>(g.n, g.J, a);
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
  if (g.vec && mode == MODE_UPDATE && iuwt_vec_fine_ok(g)) return launch_fine_analysis_vec(g, a, s);
  switch (g.gen * 10 + g.j1) {
    case 11: return fine_an_mode<1, 1>(g, a, mode, s);
    case 12: return fine_an_mode<1, 2>(g, a, mode, s);
    case 13: return fine_an_mode<1, 3>(g, a, mode, s);
    case 21: return fine_an_mode<2, 1>(g, a, mode, s);
    case 22: return fine_an_mode<2, 2>(g, a, mode, s);
    case 23: return fine_an_mode<2, 3>(g, a, mode, s);
  }
  return cudaErrorInvalidValue;
}

// The adjoint tile takes 1024 threads when its shared memory fits one block per SM only.
static bool fine_adj_wide(int gen, int j1) { return fine_smem_bytes(gen, j1, 1) > 113 * 1024; }

template <int GEN, int J1> static cudaError_t fine_adj(const Geom& g, const IuwtArgs& a, cudaStream_t s) {
  dim3 grid(g.n / kTile, g.n / kTile, g.L);
  const size_t P = (size_t)g.n * g.n;
  const bool from_u = (g.J == g.j1);
  const float* rin = from_u ? a.U + (size_t)g.J * P : a.rin;
  const size_t stride = from_u ? (size_t)(g.J + 1) * P : P;
  if (fine_adj_wide(GEN, J1))
    k_fine_adjoint<GEN, J1, 1024><<<grid, 1024, fine_smem_bytes(g, 1), s>>>(g.n, g.J, rin, stride, a);
  else
    k_fine_adjoint<GEN, J1, kFineThreads><<<grid, kFineThreads, fine_smem_bytes(g, 1), s>>>(g.n, g.J, rin, stride, a);
  return cudaGetLastError();
}

cudaError_t launch_fine_adjoint(const Geom& g, const IuwtArgs& a, cudaStream_t s) {
  if (g.vec && iuwt_vec_fine_ok(g)) return launch_fine_adjoint_vec(g, a, s);
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

// Threads per coarse cluster block: one pass-1 item (8 outputs) per thread.
static int coarse_threads(const Geom& g) {
  const int m = g.n >> g.j1, rpc = m / (g.cs > 0 ? g.cs : 1);
  int t = m * rpc / kQ;
  if (t < 64) t = 64;
  if (t > kCoarseThreads) t = kCoarseThreads;
  return t < m ? m : t;
}

template <int GEN, int MODE>
static cudaError_t coarse_n(const Geom& g, const float* c_in, float* r_out, float* U, float k, float rho,
                            double* partials, cudaStream_t s) {
  const int s2 = 1 << (2 * g.j1);
  if (g.cs > 0) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(s2 * g.cs, g.L);
    cfg.blockDim = dim3(coarse_threads(g));
    cfg.dynamicSmemBytes = coarse_cl_smem_bytes(g.n, g.J, g.gen, g.j1, g.cs);
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = g.cs;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    if (g.cs == 1 && (g.n >> g.j1) == 64)
      return cudaLaunchKernelEx(&cfg, k_coarse_cl<GEN, MODE, 64>, g.n, g.J, g.j1, g.cs, c_in, r_out, U, k, rho,
                                partials);
    return cudaLaunchKernelEx(&cfg, k_coarse_cl<GEN, MODE>, g.n, g.J, g.j1, g.cs, c_in, r_out, U, k, rho, partials);
  }
  const int M = g.n >> g.j1;
  int th = M * M < 1024 ? M * M : 1024;
  th = (th + 31) / 32 * 32;
  k_coarse<GEN, MODE><<<dim3(s2, g.L), th, coarse_stream_smem_bytes(g.n, g.gen, g.j1), s>>>(g.n, g.J, g.j1, c_in, r_out,
                                                                                            U, k, rho, partials);
  return cudaGetLastError();
}

cudaError_t launch_coarse(const Geom& g, const float* c_in, float* r_out, float* U, float k, float rho, int mode,
                          double* partials, cudaStream_t s, int* nblocks) {
  if (g.vec && mode == MODE_UPDATE && iuwt_vec_coarse_ok(g)) {
    if (nblocks) *nblocks = (1 << (2 * g.j1)) * g.L;
    return launch_coarse_vec(g, c_in, r_out, U, k, rho, s);
  }
  if (nblocks) *nblocks = (1 << (2 * g.j1)) * g.L * (g.cs > 0 ? g.cs : 1);
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

// Number of clusters of size cs that can be resident on this device (0: cannot run).
template <int GEN> static int cluster_fit(const Geom& g, int cs) {
  Geom gc = g;
  gc.cs = cs;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((1 << (2 * g.j1)) * cs, g.L);
  cfg.blockDim = dim3(coarse_threads(gc));
  cfg.dynamicSmemBytes = coarse_cl_smem_bytes(g.n, g.J, g.gen, g.j1, cs);
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = cs;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  int ncl = 0;
  if (cudaOccupancyMaxActiveClusters(&ncl, k_coarse_cl<GEN, MODE_UPDATE>, &cfg) != cudaSuccess) {
    cudaGetLastError();
    return 0;
  }
  return ncl;
}

template <int GEN> static cudaError_t cfg_gen(Geom& g) {
  cudaError_t e;
#define SET(fn) if ((e = allow_max_dyn_smem(fn))) return e;
  if (g.J > 0 && g.j1 > 0) {
    switch (g.j1) {
      case 1: SET((k_fine_analysis<GEN, 1, 0>)) SET((k_fine_analysis<GEN, 1, 1>)) SET((k_fine_analysis<GEN, 1, 2>))
              SET((k_fine_adjoint<GEN, 1, 512>)) SET((k_fine_adjoint<GEN, 1, 1024>)) break;
      case 2: SET((k_fine_analysis<GEN, 2, 0>)) SET((k_fine_analysis<GEN, 2, 1>)) SET((k_fine_analysis<GEN, 2, 2>))
              SET((k_fine_adjoint<GEN, 2, 512>)) SET((k_fine_adjoint<GEN, 2, 1024>)) break;
      case 3: SET((k_fine_analysis<GEN, 3, 0>)) SET((k_fine_analysis<GEN, 3, 1>)) SET((k_fine_analysis<GEN, 3, 2>))
              SET((k_fine_adjoint<GEN, 3, 512>)) SET((k_fine_adjoint<GEN, 3, 1024>)) break;
    }
  }
  g.cs = 0;
  if (g.J > g.j1) {
    SET((k_coarse<GEN, 0>)) SET((k_coarse<GEN, 1>)) SET((k_coarse<GEN, 2>)) SET((k_coarse<GEN, 3>))
    SET((k_coarse_cl<GEN, 0>)) SET((k_coarse_cl<GEN, 1>)) SET((k_coarse_cl<GEN, 2>)) SET((k_coarse_cl<GEN, 3>))
    SET((k_coarse_cl<GEN, 0, 64>)) SET((k_coarse_cl<GEN, 1, 64>)) SET((k_coarse_cl<GEN, 2, 64>))
    SET((k_coarse_cl<GEN, 3, 64>))
    // cluster split: the smallest whose blocks fit three, two, then one per SM; MUFFIN_COARSE_CLUSTER
    // (1, 2, 4 or 8) forces a size for tuning when it fits
    if (const char* env = getenv("MUFFIN_COARSE_CLUSTER")) {
      const int cs = atoi(env);
      if (cs >= 1 && cs <= 8 && (cs & (cs - 1)) == 0 && (g.n >> g.j1) / cs >= kQ &&
          coarse_cl_smem_bytes(g.n, g.J, g.gen, g.j1, cs) <= 220 * 1024 && cluster_fit<GEN>(g, cs) > 0)
        g.cs = cs;
    }
    for (size_t budget : {(size_t)110 * 1024, (size_t)220 * 1024}) {
      if (g.cs) break;
      for (int cs = coarse_cluster_size(g.n, g.J, g.gen, g.j1, budget); cs > 0 && cs <= 8; cs *= 2) {
        const int rpc = (g.n >> g.j1) / cs;
        if (rpc < kQ || rpc % kQ != 0) break;
        if (coarse_cl_smem_bytes(g.n, g.J, g.gen, g.j1, cs) <= budget && cluster_fit<GEN>(g, cs) > 0) {
          g.cs = cs;
          break;
        }
      }
      if (g.cs) break;
    }
    if (g.cs == 0 && coarse_stream_smem_bytes(g.n, g.gen, g.j1) > 220 * 1024) return cudaErrorInvalidConfiguration;
  }
#undef SET
  return cudaSuccess;
}

cudaError_t iuwt_configure(Geom& g) {
  // MUFFIN_IUWT_GENERAL: the general kernels for every generation (comparisons)
  g.vec = (g.gen == 1 && getenv("MUFFIN_IUWT_GENERAL") == nullptr) ? 1 : 0;
  // MUFFIN_FINE_THREADS / MUFFIN_COARSE_THREADS (256 or 512) fix the block sizes the autotuner would choose
  if (const char* v = getenv("MUFFIN_FINE_THREADS")) g.fnt = atoi(v) == 512 ? 512 : 256;
  if (const char* v = getenv("MUFFIN_COARSE_THREADS")) g.cnt = atoi(v) == 512 ? 512 : 256;
  if (g.vec) {
    const cudaError_t e = iuwt_vec_configure();
    if (e != cudaSuccess) return e;
  }
  return g.gen == 1 ? cfg_gen<1>(g) : cfg_gen<2>(g);
}

}  // namespace muffin
