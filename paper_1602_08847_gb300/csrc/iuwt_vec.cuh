// Vectorised kernels of the generation-1 IUWT on the hot path (Eqs. 9 and 11):
// the fine-level analysis with the spatial dual update, the fine-level
// adjoint, and the coarse levels on one class sub-image per block.
//
// Same arithmetic as the general kernels (k_iuwt.cu), organised for issue
// slots: every separable pass moves float4 chunks (four adjacent columns).
//   vertical pass  one thread walks a chain of output rows o, o + D, o + 2D,
//                  ... of one chunk column with a five-row window in
//                  registers: one 128-bit shared load per four outputs;
//   horizontal pass one thread walks a run of output chunks of one row with
//                  a window of chunks in registers (the five taps of each of
//                  the four lanes are register picks fixed at compile time).
// Both passes read and write shared memory with row pitches = 4 (mod 8)
// floats, so the eight 16-byte accesses of a quarter warp fall into distinct
// bank groups.  The taps are summed unnormalised, (a + e) + 4 (b + d) + 6 c,
// and the 1/256 of the two passes is applied once in the epilogue.
// Global loads and stores of the natural-layout planes are 128-bit.
#pragma once
#include "device.cuh"

namespace muffin {
namespace vec {

constexpr int kT = 64;          // output tile side (fine kernels)
// Threads per block: NT is a template parameter of every kernel (256 or 512).

// Outputs per work item of a vertical pass (chains of RO / D rows over NCH
// chunk columns) and of a horizontal pass (rows of NCO chunks), chosen for NT
// threads: the least per-thread work, counted as rounds of items times
// (outputs + window loads), ties to the longer run (fewer window reloads).
__host__ __device__ constexpr int choose_seg(int NT, int NCH, int RO, int D) {
  int best = 1, best_cost = 1 << 30;
  const int chain = (RO + D - 1) / D;
  for (int seg = 2; seg <= 11 && seg <= chain; ++seg) {
    const int items = NCH * D * ((chain + seg - 1) / seg);
    const int cost = ((items + NT - 1) / NT) * (2 * seg + 4);
    if (cost <= best_cost) { best_cost = cost; best = seg; }
  }
  return best;
}
__host__ __device__ constexpr int choose_segc(int NT, int NR, int NCO, int D) {
  int best = 1, best_cost = 1 << 30;
  const int kr = (2 * D + 3) / 4;
  for (int seg = 2; seg <= 11 && seg <= NCO; ++seg) {
    const int items = NR * ((NCO + seg - 1) / seg);
    const int cost = ((items + NT - 1) / NT) * (2 * seg + 2 * kr);
    if (cost <= best_cost) { best_cost = cost; best = seg; }
  }
  return best;
}

__host__ __device__ constexpr int ceil4(int v) { return (v + 3) & ~3; }

__device__ __forceinline__ float4 ld4(const float* p) { return *reinterpret_cast<const float4*>(p); }
__device__ __forceinline__ void st4(float* p, float4 v) { *reinterpret_cast<float4*>(p) = v; }
// Global loads at L2 (ld.global.cg): coherent with what other blocks of the same
// launch wrote before a grid barrier (the persistent batch kernel), and these
// streams gain nothing from L1.
__device__ __forceinline__ float4 ldg4(const float* p) { return __ldcg(reinterpret_cast<const float4*>(p)); }
__device__ __forceinline__ float4 sub4(float4 a, float4 b) { return make_float4(a.x - b.x, a.y - b.y, a.z - b.z, a.w - b.w); }
__device__ __forceinline__ float comp(const float4& v, int e) { return e == 0 ? v.x : e == 1 ? v.y : e == 2 ? v.z : v.w; }
__device__ __forceinline__ float& compr(float4& v, int e) { return e == 0 ? v.x : e == 1 ? v.y : e == 2 ? v.z : v.w; }

// unnormalised B3 taps: 16 x [1, 4, 6, 4, 1] / 16
__device__ __forceinline__ float b3u(float a, float b, float c, float d, float e) {
  return fmaf(6.0f, c, fmaf(4.0f, b + d, a + e));
}
__device__ __forceinline__ float4 b3u4(const float4& a, const float4& b, const float4& c, const float4& d,
                                       const float4& e) {
  return make_float4(b3u(a.x, b.x, c.x, d.x, e.x), b3u(a.y, b.y, c.y, d.y, e.y), b3u(a.z, b.z, c.z, d.z, e.z),
                     b3u(a.w, b.w, c.w, d.w, e.w));
}

// ------------------------------------------------------------------ vertical pass
// Output row o (0 <= o < RO) of chunk column c (0 <= c < NCH) is the unnormalised
// B3 sum of input rows o, o + D, ..., o + 4D (the input origin sits 2D rows above
// the output origin).  DIFF: the input is in - sub (both read at the same place).
// A work item is a chain segment: chunk column c (fastest across threads),
// residue rho = o mod D, SEG outputs.
template <int NT, int D, int NCH, int RO, int SEG, int PI, int PO, bool DIFF>
__device__ __forceinline__ void vpass(const float* __restrict__ in, const float* __restrict__ sub,
                                      float* __restrict__ out) {
  constexpr int CHAIN = (RO + D - 1) / D;
  constexpr int NSEG = (CHAIN + SEG - 1) / SEG;
  constexpr int NITEMS = NCH * D * NSEG;
  constexpr int RIN = RO + 4 * D;
  for (int it = threadIdx.x; it < NITEMS; it += NT) {
    const int c = it % NCH;
    const int rest = it / NCH;
    const int rho = rest % D;
    const int s = rest / D;
    const int o0 = rho + D * SEG * s;
    float4 w[SEG + 4];
#pragma unroll
    for (int t = 0; t < SEG + 4; ++t) {
      const int row = o0 + D * t;
      if (row < RIN) {
        w[t] = ld4(in + row * PI + 4 * c);
        if constexpr (DIFF) w[t] = sub4(w[t], ld4(sub + row * PI + 4 * c));
      }
    }
#pragma unroll
    for (int i = 0; i < SEG; ++i) {
      const int o = o0 + D * i;
      if (o < RO) st4(out + o * PO + 4 * c, b3u4(w[i], w[i + 1], w[i + 2], w[i + 3], w[i + 4]));
    }
  }
}

// Unnormalised B3 sums of the four lanes of the chunk at window index k0:
// lane e takes input columns 4 k0 + e + t D, t = -2..2 (register picks fixed
// at compile time).
template <int D, int NW>
__device__ __forceinline__ float4 hsum(const float4 (&w)[NW], int k0) {
  float4 o;
#pragma unroll
  for (int e = 0; e < 4; ++e) {
    float tap[5];
#pragma unroll
    for (int t = 0; t < 5; ++t) {
      const int off = e + (t - 2) * D;                         // column offset from chunk start
      const int dk = off >= 0 ? off / 4 : -((-off + 3) / 4);   // floor(off / 4)
      tap[t] = comp(w[k0 + dk], off - 4 * dk);
    }
    compr(o, e) = b3u(tap[0], tap[1], tap[2], tap[3], tap[4]);
  }
  return o;
}

// ------------------------------------------------------------------ horizontal pass
// Output chunk k (0 <= k < NCO) of row r (0 <= r < NR): lane e is the
// unnormalised B3 sum of input columns 4 (k + KO) + e + t D, t = -2..2, where
// KO is the input chunk of output chunk 0 (input chunk index 0 = in).
// epi(r, k, raw) receives the float4 of raw sums.  A work item is a run of SEGC
// output chunks of one row (rows fastest across threads).
template <int NT, int D, int NR, int NCO, int SEGC, int KO, int PI, typename F>
__device__ __forceinline__ void hpass(const float* __restrict__ in, F&& epi) {
  constexpr int KR = (2 * D + 3) / 4;          // input chunks needed on each side
  constexpr int NSEG = (NCO + SEGC - 1) / SEGC;
  constexpr int NITEMS = NR * NSEG;
  constexpr int NW = SEGC + 2 * KR;
  for (int it = threadIdx.x; it < NITEMS; it += NT) {
    const int r = it % NR;
    const int s = it / NR;
    const int k0 = s * SEGC;
    const float* row = in + r * PI + 4 * (k0 + KO - KR);
    float4 w[NW];
#pragma unroll
    for (int q = 0; q < NW; ++q)
      if (k0 + q - KR < NCO + KR) w[q] = ld4(row + 4 * q);
#pragma unroll
    for (int i = 0; i < SEGC; ++i)
      if (k0 + i < NCO) epi(r, k0 + i, hsum<D>(w, i + KR));
  }
}

// Same along a periodic row of NCH chunks (coarse sub-images): input chunk
// (k + q) mod NCH.
template <int NT, int D, int NR, int NCH, int SEGC, int PI, typename F>
__device__ __forceinline__ void hpass_per(const float* __restrict__ in, F&& epi) {
  constexpr int KR = (2 * D + 3) / 4;
  constexpr int NSEG = NCH / SEGC;
  static_assert(NCH % SEGC == 0, "periodic rows split into whole runs");
  constexpr int NITEMS = NR * NSEG;
  constexpr int NW = SEGC + 2 * KR;
  for (int it = threadIdx.x; it < NITEMS; it += NT) {
    const int r = it % NR;
    const int s = it / NR;
    const int k0 = s * SEGC;
    const float* row = in + r * PI;
    float4 w[NW];
#pragma unroll
    for (int q = 0; q < NW; ++q) w[q] = ld4(row + 4 * ((k0 + q - KR + NCH) % NCH));
#pragma unroll
    for (int i = 0; i < SEGC; ++i) epi(r, k0 + i, hsum<D>(w, i + KR));
  }
}

__device__ __forceinline__ float dual1(float uo, float w, float k, float rho) {
  return rho * sat1(fmaf(k, w, uo)) + (1.0f - rho) * uo;
}
__device__ __forceinline__ float4 dual4(float4 uo, float4 w, float k, float rho) {
  return make_float4(dual1(uo.x, w.x, k, rho), dual1(uo.y, w.y, k, rho), dual1(uo.z, w.z, k, rho),
                     dual1(uo.w, w.w, k, rho));
}

// Region of a natural-layout plane around the tile (periodic wrap): rows
// ty0 - HY .. ty0 + 64 + HY - 1, columns tx0 - HX .. tx0 + 64 + HX - 1 (HX a
// multiple of 4), as float4 chunks, into dst (pitch P).  Loads then stores,
// NPT chunks per thread in flight.
template <int NT, int HY, int HX, int P>
struct Region {
  static constexpr int ROWS = kT + 2 * HY, NCH = (kT + 2 * HX) / 4, N4 = ROWS * NCH;
  static constexpr int NPT = (N4 + NT - 1) / NT;
  float4 v[NPT];
  __device__ __forceinline__ void load(const float* __restrict__ plane, int n, int ty0, int tx0) {
    const int m = n - 1;
#pragma unroll
    for (int q = 0; q < NPT; ++q) {
      const int i = threadIdx.x + q * NT;
      if (i < N4) {
        const int r = i / NCH, c = i % NCH;
        const int gy = (ty0 - HY + r) & m, gx = (tx0 - HX + 4 * c) & m;
        v[q] = ldg4(plane + (size_t)gy * n + gx);
      }
    }
  }
  // store at region row r, chunk c -> dst[(r + R0) * P + 4 (c + C0)]
  template <int R0, int C0>
  __device__ __forceinline__ void store(float* __restrict__ dst) const {
#pragma unroll
    for (int q = 0; q < NPT; ++q) {
      const int i = threadIdx.x + q * NT;
      if (i < N4) {
        const int r = i / NCH, c = i % NCH;
        st4(dst + (r + R0) * P + 4 * (c + C0), v[q]);
      }
    }
  }
};

// ------------------------------------------------------------------ L2 prefetch for the next wave
// (pf_line, pf_bulk, pf_next: device.cuh)
// Lines of the region rows ty0 - HY .. ty0 + 63 + HY, columns tx0 - HX ..
// tx0 + 63 + HX (periodic) of a natural-layout plane.
template <int NT, int HY, int HX>
__device__ __forceinline__ void pf_region(const float* __restrict__ plane, int n, int ty0, int tx0) {
  constexpr int ROWS = kT + 2 * HY, LINES = 2 + 2 * ((HX + 31) / 32);   // tx0 is a multiple of 64
  const int m = n - 1, q0 = (tx0 - HX) >> 5;
  for (int i = threadIdx.x; i < ROWS * LINES; i += NT) {
    const int r = i / LINES, q = i % LINES;
    pf_line(plane + (size_t)((ty0 - HY + r) & m) * n + ((32 * (q0 + q)) & m));
  }
}

// ================================================================== fine analysis (generation 1)
// Levels j < J1 on a 64 x 64 tile; c_j is needed on a halo HC(j) rows /
// HX(j) columns (a multiple of 4) around the tile.  A holds c_j in place
// (origin: the level-0 region), T the vertical pass, W the detail plane w_j on
// the tile.  U_j of the tile is prefetched at the start of level j.
template <int J1> struct FineA {
  __host__ __device__ static constexpr int HC(int j) { return (1 << (J1 + 1)) - (1 << (j + 1)); }
  __host__ __device__ static constexpr int HX(int j) { return ceil4(HC(j)); }
  static constexpr int RA = kT + 2 * HC(0);
  static constexpr int CA = kT + 2 * HX(0);
  static constexpr int PA = CA + 4;                 // = 4 (mod 8)
  static constexpr int PW = kT + 4;
  static constexpr int NA = RA * PA, NW = kT * PW;
  static constexpr size_t SMEM = (size_t)(2 * NA + NW) * sizeof(float);
};

template <int NT, int J1, int J0>
__device__ __forceinline__ void fine_an_level(float* __restrict__ A, float* __restrict__ T, float* __restrict__ W,
                                              float* __restrict__ Uj, int n, int ty0, int tx0, float k, float rho) {
  using G = FineA<J1>;
  constexpr int D = 1 << J0, PA = G::PA, PW = G::PW;
  constexpr int HCi = G::HC(J0), HCo = G::HC(J0 + 1), HXi = G::HX(J0), HXo = G::HX(J0 + 1);
  constexpr int RO = kT + 2 * HCo, NCHI = (kT + 2 * HXi) / 4, NCO = (kT + 2 * HXo) / 4;
  constexpr int R0 = G::HC(0) - HCo;                // region row of output row 0
  constexpr int C0 = (G::HX(0) - HXo) / 4;          // region chunk of output chunk 0
  // this thread's four chunks of U_j on the tile; they arrive during the passes
  constexpr int NU = kT * kT / 4 / NT;
  float4 uo[NU];
#pragma unroll
  for (int q = 0; q < NU; ++q) {
    const int i = threadIdx.x + q * NT, r = i >> 4, c = i & 15;
    uo[q] = ldg4(Uj + (size_t)(ty0 + r) * n + tx0 + 4 * c);
  }
  constexpr int SEGV = choose_seg(NT, NCHI, RO, D);
  vpass<NT, D, NCHI, RO, SEGV, PA, PA, false>(A + (G::HC(0) - HCi) * PA + (G::HX(0) - HXi),
                                          nullptr, T + R0 * PA + (G::HX(0) - HXi));
  __syncthreads();
  constexpr int SEGC = choose_segc(NT, RO, NCO, D);
  constexpr float inv = 1.0f / 256.0f;
  hpass<NT, D, RO, NCO, SEGC, (HXi - HXo) / 4, PA>(
      T + R0 * PA + (G::HX(0) - HXi), [&](int r, int kc, float4 raw) {
        float* a = A + (R0 + r) * PA + 4 * (C0 + kc);
        const float4 cj = ld4(a);
        const float4 cn = make_float4(raw.x * inv, raw.y * inv, raw.z * inv, raw.w * inv);
        const int tr = r - HCo, tc = kc - HXo / 4;    // tile coordinates
        if (tr >= 0 && tr < kT && tc >= 0 && tc < kT / 4) st4(W + tr * PW + 4 * tc, sub4(cj, cn));
        st4(a, cn);
      });
  __syncthreads();
#pragma unroll
  for (int q = 0; q < NU; ++q) {
    const int i = threadIdx.x + q * NT, r = i >> 4, c = i & 15;
    const float4 w = ld4(W + r * PW + 4 * c);
    float4* dst = reinterpret_cast<float4*>(Uj + (size_t)(ty0 + r) * n + tx0 + 4 * c);
    *dst = dual4(uo[q], w, k, rho);
  }
  if constexpr (J0 + 1 < J1) fine_an_level<NT, J1, J0 + 1>(A, T, W, Uj + (size_t)n * n, n, ty0, tx0, k, rho);
}

// One 64 x 64 tile (origin ty0, tx0) of channel l; sm: FineA<J1>::SMEM bytes.
// U: [L][J+1][n][n]; planes j >= J1 class-permuted.
template <int NT, int J1>
__device__ __forceinline__ void fine_analysis_tile(float* __restrict__ sm, int n, int J, const float* __restrict__ D,
                                                   float* __restrict__ U, float* __restrict__ cr, float k, float rho,
                                                   int l, int ty0, int tx0) {
  using G = FineA<J1>;
  float* A = sm;
  float* T = A + G::NA;
  float* W = T + G::NA;
  const size_t P = (size_t)n * n;
  {
    Region<NT, G::HC(0), G::HX(0), G::PA> reg;
    reg.load(D + (size_t)l * P, n, ty0, tx0);
    reg.template store<0, 0>(A);
  }
  __syncthreads();
  fine_an_level<NT, J1, 0>(A, T, W, U + (size_t)l * (J + 1) * P, n, ty0, tx0, k, rho);
  // c_J1 on the tile -> class-permuted (stride S = 2^J1): one float4 = 4 sub-columns of one class
  constexpr int S = 1 << J1, NSUB = kT / S / 4;   // float4 per class per tile row
  const int mc = n >> J1;
  const size_t mc2 = (size_t)mc * mc;
  float* dst = J == J1 ? U + ((size_t)l * (J + 1) + J) * P : cr + (size_t)l * P;
  for (int i = threadIdx.x; i < kT * S * NSUB; i += NT) {
    // at S = 8 the rows are taken in the order 0, 2, 1, 3 of each group of four:
    // the two rows of a warp then sit 2 pitches apart, which halves the bank
    // conflicts of the strided reads (4-way -> 2-way)
    const int cx = i % S, rest = i / S, m4 = rest % NSUB, rr = rest / NSUB;
    const int r = S == 8 ? (rr & ~3) | ((rr & 1) << 1) | ((rr >> 1) & 1) : rr;
    const float* a = A + (G::HC(0) + r) * G::PA + G::HX(0) + cx + S * 4 * m4;
    float4 v = make_float4(a[0], a[S], a[2 * S], a[3 * S]);
    const int gy = ty0 + r;
    float* p = dst + (size_t)((gy & (S - 1)) * S + cx) * mc2 + (size_t)(gy >> J1) * mc + (tx0 >> J1) + 4 * m4;
    if (J == J1) v = dual4(ld4(p), v, k, rho);
    st4(p, v);
  }
}

// grid (n/64, n/64, L); ahead: resident blocks (0: no L2 prefetch)
template <int NT, int J1>
__global__ void __launch_bounds__(NT, 2)
k_fine_analysis_v(int n, int J, const float* __restrict__ D, float* __restrict__ U, float* __restrict__ cr,
                  float k, float rho, int ahead) {
  extern __shared__ __align__(16) float sm[];
  const int nx = pf_next(ahead);
  if (nx >= 0) {
    const int tx = nx % gridDim.x, ty = (nx / gridDim.x) % gridDim.y, l = nx / (gridDim.x * gridDim.y);
    const size_t P = (size_t)n * n;
    pf_region<NT, FineA<J1>::HC(0), FineA<J1>::HX(0)>(D + (size_t)l * P, n, ty * kT, tx * kT);
    for (int j = 0; j < J1; ++j) pf_region<NT, 0, 0>(U + ((size_t)l * (J + 1) + j) * P, n, ty * kT, tx * kT);
  }
  fine_analysis_tile<NT, J1>(sm, n, J, D, U, cr, k, rho, blockIdx.z, blockIdx.y * kT, blockIdx.x * kT);
}

// ================================================================== fine adjoint (generation 1)
// r_J1 (class-permuted) on halo HR(J1) around the tile, then for j = J1-1 .. 0:
// r_j = u_j + H_j (r_{j+1} - u_j) on halo HR(j); S = r_0 on the tile.
template <int J1> struct FineT {
  __host__ __device__ static constexpr int HR(int j) { return (1 << (j + 1)) - 2; }
  __host__ __device__ static constexpr int HX(int j) { return ceil4(HR(j)); }
  static constexpr int RA = kT + 2 * HR(J1);
  static constexpr int CA = kT + 2 * HX(J1);
  static constexpr int PA = CA + 4;
  static constexpr int RT = kT + 2 * HR(J1 - 1);
  static constexpr int NA = RA * PA, NT = RT * PA;
  static constexpr size_t SMEM = (size_t)(2 * NA + NT) * sizeof(float);
};

template <int NT, int J1, int J0>
__device__ __forceinline__ void fine_adj_level(float* __restrict__ R, float* __restrict__ Ub, float* __restrict__ T,
                                               const float* __restrict__ Uc, int n, int ty0, int tx0) {
  using G = FineT<J1>;
  constexpr int D = 1 << J0, PA = G::PA;
  constexpr int HRi = G::HR(J0 + 1), HRo = G::HR(J0), HXi = G::HX(J0 + 1), HXo = G::HX(J0);
  constexpr int RO = kT + 2 * HRo, NCHI = (kT + 2 * HXi) / 4, NCO = (kT + 2 * HXo) / 4;
  constexpr int RI0 = G::HR(J1) - HRi, R0 = G::HR(J1) - HRo;
  constexpr int CI0 = (G::HX(J1) - HXi) / 4, C0 = (G::HX(J1) - HXo) / 4;
  // u_{J0-1} on the region of r_J0, loaded while this level filters
  constexpr int HRn = J0 > 0 ? G::HR(J0) : 0, HXn = J0 > 0 ? G::HX(J0) : 0;
  Region<NT, HRn, HXn, PA> nxt;
  if constexpr (J0 > 0) nxt.load(Uc - (size_t)n * n, n, ty0, tx0);
  constexpr int SEGV = choose_seg(NT, NCHI, RO, D);
  vpass<NT, D, NCHI, RO, SEGV, PA, PA, true>(R + RI0 * PA + 4 * CI0, Ub + RI0 * PA + 4 * CI0, T + 4 * CI0);
  __syncthreads();
  constexpr int SEGC = choose_segc(NT, RO, NCO, D);
  constexpr float inv = 1.0f / 256.0f;
  hpass<NT, D, RO, NCO, SEGC, C0 - CI0, PA>(T + 4 * CI0, [&](int r, int kc, float4 raw) {
    const int off = (R0 + r) * PA + 4 * (C0 + kc);
    const float4 u = ld4(Ub + off);
    st4(R + off, make_float4(fmaf(raw.x, inv, u.x), fmaf(raw.y, inv, u.y), fmaf(raw.z, inv, u.z),
                             fmaf(raw.w, inv, u.w)));
  });
  __syncthreads();
  if constexpr (J0 > 0) {
    nxt.template store<G::HR(J1) - HRn, (G::HX(J1) - HXn) / 4>(Ub);
    __syncthreads();
    fine_adj_level<NT, J1, J0 - 1>(R, Ub, T, Uc - (size_t)n * n, n, ty0, tx0);
  }
}

// One tile of channel l; rin: r_J1 per channel (class-permuted, stride 2^J1),
// channel stride rin_stride; sm: FineT<J1>::SMEM bytes.
template <int NT, int J1>
__device__ __forceinline__ void fine_adjoint_tile(float* __restrict__ sm, int n, int J, const float* __restrict__ rin,
                                                  size_t rin_stride, const float* __restrict__ U,
                                                  float* __restrict__ S, int l, int ty0, int tx0) {
  using G = FineT<J1>;
  float* R = sm;
  float* Ub = R + G::NA;
  float* T = Ub + G::NA;
  const size_t P = (size_t)n * n;
  const float* Uc = U + ((size_t)l * (J + 1) + J1 - 1) * P;   // u_{J1-1}
  {
    Region<NT, G::HR(J1), G::HX(J1), G::PA> ub;
    ub.load(Uc, n, ty0, tx0);
    // r_J1 region from the class-permuted plane, read two sub-columns (8 bytes)
    // at a time and scattered into R.  Lane (cx, p) of a warp takes class cx
    // and sub-column pairs p, p + PL, ... of the warp's rows (rows wid,
    // wid + NW, ...): per row one address computation; a warp's load is eight
    // 32-byte runs.  Lanes in the upper half of p write the odd sub-column
    // first, which puts the two halves of the warp on different banks.
    constexpr int SC = 1 << J1, HXR = G::HX(J1), NSC = (kT + 2 * HXR) / SC, NP = NSC / 2;
    constexpr int PL = 32 / SC, NPP = (NP + PL - 1) / PL;
    constexpr int NW = NT / 32, RPW = (G::RA + NW - 1) / NW;
    const int mc = n >> J1, mm = mc - 1, m = n - 1;
    const size_t mc2 = (size_t)mc * mc;
    const float* rl = rin + (size_t)l * rin_stride;
    const int sc0 = (tx0 >> J1) - HXR / SC;
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const int cx = lane % SC, p = lane / SC;
    float2 rv[RPW][NPP];
#pragma unroll
    for (int rr = 0; rr < RPW; ++rr) {     // every load in flight before the first store
      const int r = wid + rr * NW;
      if (r < G::RA) {
        const int gy = (ty0 - G::HR(J1) + r) & m;
        const float* row = rl + (size_t)((gy & (SC - 1)) * SC + cx) * mc2 + (size_t)(gy >> J1) * mc;
#pragma unroll
        for (int h = 0; h < NPP; ++h) {
          const int p2 = p + h * PL;
          if (p2 < NP) rv[rr][h] = __ldcg(reinterpret_cast<const float2*>(row + ((sc0 + 2 * p2) & mm)));
        }
      }
    }
    const bool odd_first = p >= PL / 2;
#pragma unroll
    for (int rr = 0; rr < RPW; ++rr) {
      const int r = wid + rr * NW;
      if (r < G::RA) {
#pragma unroll
        for (int h = 0; h < NPP; ++h) {
          const int p2 = p + h * PL;
          if (p2 < NP) {
            float* d = R + r * G::PA + cx + SC * 2 * p2;
            const float2 v = rv[rr][h];
            d[odd_first ? SC : 0] = odd_first ? v.y : v.x;
            d[odd_first ? 0 : SC] = odd_first ? v.x : v.y;
          }
        }
      }
    }
    ub.template store<0, 0>(Ub);
  }
  __syncthreads();
  fine_adj_level<NT, J1, J1 - 1>(R, Ub, T, Uc, n, ty0, tx0);
  for (int i = threadIdx.x; i < kT * kT / 4; i += NT) {
    const int r = i >> 4, c = i & 15;
    st4(S + (size_t)l * P + (size_t)(ty0 + r) * n + tx0 + 4 * c,
        ld4(R + (G::HR(J1) + r) * G::PA + G::HX(J1) + 4 * c));
  }
}

// u_{J0-1} on halo HR(J0) for J0 = J1-1 .. 1: what the levels load as they go.
template <int NT, int J1, int J0>
__device__ __forceinline__ void pf_adj_planes(const float* __restrict__ Ul, size_t P, int n, int ty0, int tx0) {
  if constexpr (J0 >= 1) {
    pf_region<NT, FineT<J1>::HR(J0), FineT<J1>::HX(J0)>(Ul + (size_t)(J0 - 1) * P, n, ty0, tx0);
    pf_adj_planes<NT, J1, J0 - 1>(Ul, P, n, ty0, tx0);
  }
}

template <int NT, int J1>
__global__ void __launch_bounds__(NT, 2)
k_fine_adjoint_v(int n, int J, const float* __restrict__ rin, size_t rin_stride, const float* __restrict__ U,
                 float* __restrict__ S, int ahead) {
  extern __shared__ __align__(16) float sm[];
  const int nx = pf_next(ahead);
  if (nx >= 0) {
    using G = FineT<J1>;
    const int tx0 = (nx % gridDim.x) * kT, ty0 = ((nx / gridDim.x) % gridDim.y) * kT, l = nx / (gridDim.x * gridDim.y);
    const size_t P = (size_t)n * n;
    pf_region<NT, G::HR(J1), G::HX(J1)>(U + ((size_t)l * (J + 1) + J1 - 1) * P, n, ty0, tx0);
    pf_adj_planes<NT, J1, J1 - 1>(U + (size_t)l * (J + 1) * P, P, n, ty0, tx0);
    // r_J1, class-permuted: per region row and class, the run of sub-columns (two lines at most)
    constexpr int SC = 1 << J1, HXR = G::HX(J1), NSC = (kT + 2 * HXR) / SC;
    const int m = n - 1, mc = n >> J1, mm = mc - 1;
    const size_t mc2 = (size_t)mc * mc;
    const float* rl = rin + (size_t)l * rin_stride;
    const int sc0 = (tx0 >> J1) - HXR / SC;
    for (int i = threadIdx.x; i < G::RA * SC * 2; i += NT) {
      const int e = i & 1, cx = (i >> 1) % SC, r = (i >> 1) / SC;
      const int gy = (ty0 - G::HR(J1) + r) & m;
      pf_line(rl + (size_t)((gy & (SC - 1)) * SC + cx) * mc2 + (size_t)(gy >> J1) * mc + ((sc0 + e * (NSC - 1)) & mm));
    }
  }
  fine_adjoint_tile<NT, J1>(sm, n, J, rin, rin_stride, U, S, blockIdx.z, blockIdx.y * kT, blockIdx.x * kT);
}

// ================================================================== coarse levels, one sub-image per block
// Class sub-image M x M (periodic), levels j1 .. J-1 at sub-dilation d =
// 2^(j - j1) (NL = J - j1 levels) and the coarse plane, all resident: A holds
// c (then r) with HR wrapped halo rows above and below, T the vertical pass,
// Us the NL + 1 dual planes.  Updates U_j1..U_J and leaves r_j1 for the next
// pass's fine adjoint.
template <int M, int NL> struct CoarseV {
  static constexpr int HR = 2 << (NL - 1 < 0 ? 0 : NL - 1);   // 2 dmax
  static constexpr int P = M + 4;
  static constexpr int NA = (M + 2 * HR) * P, NT = M * P, NU = M * P;
  static constexpr size_t SMEM = (size_t)(NA + NT + (NL + 1) * NU) * sizeof(float);
};

// Chunks per work item of a periodic horizontal pass: a divisor of NCH.
__host__ __device__ constexpr int coarse_segp(int NT, int M, int NCH, int d) {
  int best = 1, best_cost = 1 << 30;
  const int kr = (2 * d + 3) / 4;
  for (int seg = 1; seg <= 8 && seg <= NCH; seg *= 2) {
    const int items = M * (NCH / seg);
    const int cost = ((items + NT - 1) / NT) * (2 * seg + 2 * kr);
    if (cost <= best_cost) { best_cost = cost; best = seg; }
  }
  return best;
}

template <int NT, int M, int PP>
__device__ __forceinline__ void wrap_rows(float* __restrict__ A, int h, int HR) {
  // rows -h..-1 <- M-h..M-1, rows M..M+h-1 <- 0..h-1 (A points at row 0)
  constexpr int NCH = M / 4;
  for (int i = threadIdx.x; i < 2 * h * NCH; i += NT) {
    const int c = i % NCH, rr = i / NCH;
    const int dst = rr < h ? rr - h : M + rr - h;
    const int src = rr < h ? M + rr - h : rr - h;
    st4(A + dst * PP + 4 * c, ld4(A + src * PP + 4 * c));
  }
}

template <int NT, int M, int NL, int LV>
__device__ __forceinline__ void coarse_an(float* __restrict__ A, float* __restrict__ T, float* __restrict__ Us,
                                          float k, float rho) {
  using G = CoarseV<M, NL>;
  constexpr int d = 1 << LV, P = G::P, NCH = M / 4;
  constexpr float inv = 1.0f / 256.0f;
  wrap_rows<NT, M, P>(A, 2 * d, G::HR);
  __syncthreads();
  vpass<NT, d, NCH, M, choose_seg(NT, NCH, M, d), P, P, false>(A - 2 * d * P, nullptr, T);
  __syncthreads();
  float* Uj = Us + LV * G::NU;
  hpass_per<NT, d, M, NCH, coarse_segp(NT, M, NCH, d), P>(T, [&](int r, int kc, float4 raw) {
    float* a = A + r * P + 4 * kc;
    const float4 cn = make_float4(raw.x * inv, raw.y * inv, raw.z * inv, raw.w * inv);
    float* up = Uj + r * P + 4 * kc;
    st4(up, dual4(ld4(up), sub4(ld4(a), cn), k, rho));
    st4(a, cn);
  });
  __syncthreads();
  if constexpr (LV + 1 < NL) coarse_an<NT, M, NL, LV + 1>(A, T, Us, k, rho);
}

// On entry A holds r_{LV+1} - u_LV (the difference is formed in the previous
// level's epilogue, not in a separate pass); leaves r_LV - u_{LV-1} (LV > 0)
// or r_LV (LV = 0) in A.
template <int NT, int M, int NL, int LV>
__device__ __forceinline__ void coarse_adj(float* __restrict__ A, float* __restrict__ T, const float* __restrict__ Us) {
  using G = CoarseV<M, NL>;
  constexpr int d = 1 << LV, P = G::P, NCH = M / 4;
  constexpr float inv = 1.0f / 256.0f;
  const float* Uj = Us + LV * G::NU;
  wrap_rows<NT, M, P>(A, 2 * d, G::HR);
  __syncthreads();
  vpass<NT, d, NCH, M, choose_seg(NT, NCH, M, d), P, P, false>(A - 2 * d * P, nullptr, T);
  __syncthreads();
  hpass_per<NT, d, M, NCH, coarse_segp(NT, M, NCH, d), P>(T, [&](int r, int kc, float4 raw) {
    const float4 u = ld4(Uj + r * P + 4 * kc);
    const float4 rj = make_float4(fmaf(raw.x, inv, u.x), fmaf(raw.y, inv, u.y), fmaf(raw.z, inv, u.z),
                                  fmaf(raw.w, inv, u.w));
    if constexpr (LV > 0)
      st4(A + r * P + 4 * kc, sub4(rj, ld4(Uj - G::NU + r * P + 4 * kc)));
    else
      st4(A + r * P + 4 * kc, rj);
  });
  __syncthreads();
  if constexpr (LV > 0) coarse_adj<NT, M, NL, LV - 1>(A, T, Us);
}

// Class sub-image cls of channel l; sm: CoarseV<M, NL>::SMEM bytes.
template <int NT, int M, int NL>
__device__ __forceinline__ void coarse_sub(float* __restrict__ sm, int n, int J, int j1,
                                           const float* __restrict__ c_in, float* __restrict__ r_out,
                                           float* __restrict__ U, float k, float rho, int cls, int l) {
  using G = CoarseV<M, NL>;
  constexpr int P = G::P, NCH = M / 4;
  float* A = sm + G::HR * P;       // row 0 of the sub-image
  float* T = sm + G::NA;
  float* Us = T + G::NT;
  const size_t Pl = (size_t)n * n, sub = (size_t)cls * M * M;
  const float* src = c_in + (size_t)l * Pl + sub;
  float* Ul = U + ((size_t)l * (J + 1) + j1) * Pl + sub;
  // the sub-image of c_j1 and of every coarse dual plane (coalesced float4),
  // all of a thread's loads in flight before its first store
  constexpr int NQ = (M * NCH + NT - 1) / NT;
  float4 va[NQ], vu[NQ][NL + 1];
#pragma unroll
  for (int q = 0; q < NQ; ++q) {
    const int i = threadIdx.x + q * NT;
    if (i < M * NCH) {
      const int c = i % NCH, r = i / NCH;
      va[q] = ldg4(src + r * M + 4 * c);
#pragma unroll
      for (int j = 0; j <= NL; ++j) vu[q][j] = ldg4(Ul + (size_t)j * Pl + r * M + 4 * c);
    }
  }
#pragma unroll
  for (int q = 0; q < NQ; ++q) {
    const int i = threadIdx.x + q * NT;
    if (i < M * NCH) {
      const int c = i % NCH, r = i / NCH;
      st4(A + r * P + 4 * c, va[q]);
#pragma unroll
      for (int j = 0; j <= NL; ++j) st4(Us + j * G::NU + r * P + 4 * c, vu[q][j]);
    }
  }
  __syncthreads();
  coarse_an<NT, M, NL, 0>(A, T, Us, k, rho);
  // coarse plane: U_J <- update with c_J; r_J = U_J, and A <- r_J - u_{J-1}
  {
    float* UJ = Us + NL * G::NU;
    for (int i = threadIdx.x; i < M * NCH; i += NT) {
      const int c = i % NCH, r = i / NCH;
      const float4 nv = dual4(ld4(UJ + r * P + 4 * c), ld4(A + r * P + 4 * c), k, rho);
      st4(UJ + r * P + 4 * c, nv);
      st4(A + r * P + 4 * c, sub4(nv, ld4(UJ - G::NU + r * P + 4 * c)));
    }
  }
  __syncthreads();
  coarse_adj<NT, M, NL, NL - 1>(A, T, Us);
  float* dst = r_out + (size_t)l * Pl + sub;
  for (int i = threadIdx.x; i < M * NCH; i += NT) {
    const int c = i % NCH, r = i / NCH;
    st4(dst + r * M + 4 * c, ld4(A + r * P + 4 * c));
#pragma unroll
    for (int j = 0; j <= NL; ++j)
      reinterpret_cast<float4*>(Ul + (size_t)j * Pl + r * M)[c] = ld4(Us + j * G::NU + r * P + 4 * c);
  }
}

// grid (4^j1, L): block = one class sub-image of one channel.
template <int NT, int M, int NL>
__global__ void __launch_bounds__(NT, 2)
k_coarse_v(int n, int J, int j1, const float* __restrict__ c_in, float* __restrict__ r_out, float* __restrict__ U,
           float k, float rho, int ahead) {
  extern __shared__ __align__(16) float sm[];
  const int nx = pf_next(ahead);
  if (nx >= 0) {
    const int cls = nx % gridDim.x, l = nx / gridDim.x;
    const size_t Pl = (size_t)n * n, sub = (size_t)cls * M * M;
    // c_j1 and U_j1..U_J of the sub-image: NL + 2 contiguous runs of M^2 floats,
    // one bulk prefetch each
    if (threadIdx.x < NL + 2) {
      const int pl = threadIdx.x;
      const float* base = pl == 0 ? c_in + (size_t)l * Pl : U + ((size_t)l * (J + 1) + j1 + pl - 1) * Pl;
      pf_bulk(base + sub, 4u * M * M);
    }
  }
  coarse_sub<NT, M, NL>(sm, n, J, j1, c_in, r_out, U, k, rho, blockIdx.x, blockIdx.y);
}

// ------------------------------------------------------------------ coarse levels, dual planes streamed
// Same levels on sub-images too large to hold every dual plane in shared
// memory (M = 128): only A (c, then r, with wrapped halo rows) and T stay
// resident; U_j is read from and written to global memory where it is used,
// and the adjoint reads back the U_j this block has just written (from L2).
template <int M, int NL> struct CoarseS {
  static constexpr int HR = 2 << (NL - 1 < 0 ? 0 : NL - 1);
  static constexpr int P = M + 4;
  static constexpr int NA = (M + 2 * HR) * P, NT = M * P;
  static constexpr size_t SMEM = (size_t)(NA + NT) * sizeof(float);
};

template <int NT, int M, int NL, int LV>
__device__ __forceinline__ void coarse_an_s(float* __restrict__ A, float* __restrict__ T, float* __restrict__ Ug,
                                            size_t Pl, float k, float rho) {
  using G = CoarseS<M, NL>;
  constexpr int d = 1 << LV, P = G::P, NCH = M / 4;
  constexpr float inv = 1.0f / 256.0f;
  wrap_rows<NT, M, P>(A, 2 * d, G::HR);
  __syncthreads();
  vpass<NT, d, NCH, M, choose_seg(NT, NCH, M, d), P, P, false>(A - 2 * d * P, nullptr, T);
  __syncthreads();
  float* Uj = Ug + (size_t)LV * Pl;
  hpass_per<NT, d, M, NCH, coarse_segp(NT, M, NCH, d), P>(T, [&](int r, int kc, float4 raw) {
    float* a = A + r * P + 4 * kc;
    const float4 cn = make_float4(raw.x * inv, raw.y * inv, raw.z * inv, raw.w * inv);
    float* up = Uj + (size_t)r * M + 4 * kc;
    st4(up, dual4(ld4(up), sub4(ld4(a), cn), k, rho));
    st4(a, cn);
  });
  __syncthreads();
  if constexpr (LV + 1 < NL) coarse_an_s<NT, M, NL, LV + 1>(A, T, Ug, Pl, k, rho);
}

template <int NT, int M, int NL, int LV>
__device__ __forceinline__ void coarse_adj_s(float* __restrict__ A, float* __restrict__ T,
                                             const float* __restrict__ Ug, size_t Pl) {
  using G = CoarseS<M, NL>;
  constexpr int d = 1 << LV, P = G::P, NCH = M / 4;
  constexpr float inv = 1.0f / 256.0f;
  // U_j was written by this block earlier in the launch: plain (coherent) loads
  const float* Uj = Ug + (size_t)LV * Pl;
  for (int i = threadIdx.x; i < M * NCH; i += NT) {      // A <- r - u_j
    const int c = i % NCH, r = i / NCH;
    st4(A + r * P + 4 * c, sub4(ld4(A + r * P + 4 * c), ld4(Uj + (size_t)r * M + 4 * c)));
  }
  __syncthreads();
  wrap_rows<NT, M, P>(A, 2 * d, G::HR);
  __syncthreads();
  vpass<NT, d, NCH, M, choose_seg(NT, NCH, M, d), P, P, false>(A - 2 * d * P, nullptr, T);
  __syncthreads();
  hpass_per<NT, d, M, NCH, coarse_segp(NT, M, NCH, d), P>(T, [&](int r, int kc, float4 raw) {
    const float4 u = ld4(Uj + (size_t)r * M + 4 * kc);
    st4(A + r * P + 4 * kc, make_float4(fmaf(raw.x, inv, u.x), fmaf(raw.y, inv, u.y), fmaf(raw.z, inv, u.z),
                                        fmaf(raw.w, inv, u.w)));
  });
  __syncthreads();
  if constexpr (LV > 0) coarse_adj_s<NT, M, NL, LV - 1>(A, T, Ug, Pl);
}

// Class sub-image cls of channel l; sm: CoarseS<M, NL>::SMEM bytes.
template <int NT, int M, int NL>
__device__ __forceinline__ void coarse_sub_s(float* __restrict__ sm, int n, int J, int j1,
                                             const float* __restrict__ c_in, float* __restrict__ r_out,
                                             float* __restrict__ U, float k, float rho, int cls, int l) {
  using G = CoarseS<M, NL>;
  constexpr int P = G::P, NCH = M / 4;
  float* A = sm + G::HR * P;
  float* T = sm + G::NA;
  const size_t Pl = (size_t)n * n, sub = (size_t)cls * M * M;
  const float* src = c_in + (size_t)l * Pl + sub;
  float* Ug = U + ((size_t)l * (J + 1) + j1) * Pl + sub;
  constexpr int NQ = (M * NCH + NT - 1) / NT;
  float4 va[NQ];
#pragma unroll
  for (int q = 0; q < NQ; ++q) {
    const int i = threadIdx.x + q * NT;
    if (i < M * NCH) va[q] = ldg4(src + (i / NCH) * M + 4 * (i % NCH));
  }
#pragma unroll
  for (int q = 0; q < NQ; ++q) {
    const int i = threadIdx.x + q * NT;
    if (i < M * NCH) st4(A + (i / NCH) * P + 4 * (i % NCH), va[q]);
  }
  __syncthreads();
  coarse_an_s<NT, M, NL, 0>(A, T, Ug, Pl, k, rho);
  {
    float* UJ = Ug + (size_t)NL * Pl;
    for (int i = threadIdx.x; i < M * NCH; i += NT) {
      const int c = i % NCH, r = i / NCH;
      float* up = UJ + (size_t)r * M + 4 * c;
      const float4 nv = dual4(ld4(up), ld4(A + r * P + 4 * c), k, rho);
      st4(up, nv);
      st4(A + r * P + 4 * c, nv);
    }
  }
  __syncthreads();
  coarse_adj_s<NT, M, NL, NL - 1>(A, T, Ug, Pl);
  float* dst = r_out + (size_t)l * Pl + sub;
  for (int i = threadIdx.x; i < M * NCH; i += NT) {
    const int c = i % NCH, r = i / NCH;
    st4(dst + r * M + 4 * c, ld4(A + r * P + 4 * c));
  }
}

template <int NT, int M, int NL>
__global__ void __launch_bounds__(NT, 1)
k_coarse_s(int n, int J, int j1, const float* __restrict__ c_in, float* __restrict__ r_out, float* __restrict__ U,
           float k, float rho) {
  extern __shared__ __align__(16) float sm[];
  coarse_sub_s<NT, M, NL>(sm, n, J, j1, c_in, r_out, U, k, rho, blockIdx.x, blockIdx.y);
}

}  // namespace vec

}  // namespace muffin
