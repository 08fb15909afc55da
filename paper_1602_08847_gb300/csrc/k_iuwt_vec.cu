// Host launchers of the vectorised generation-1 IUWT kernels (iuwt_vec.cuh).
#include <cstdlib>

#include "internal.h"
#include "iuwt_vec.cuh"

namespace muffin {

// ------------------------------------------------------------------ host side
bool iuwt_vec_fine_ok(const Geom& g) { return g.gen == 1 && g.n >= 64 && g.j1 >= 1 && g.j1 <= 3 && g.J >= g.j1; }

bool iuwt_vec_coarse_ok(const Geom& g) {
  const int M = g.n >> g.j1, NL = g.J - g.j1;
  return g.gen == 1 && g.j1 >= 1 && (M == 32 || M == 64 || M == 128) && NL >= 1 && NL <= 3;
}

// Threads per block of the fine and of the coarse kernels: g.fnt / g.cnt,
// 256 (two blocks per SM) or 512, chosen by the set-up autotuner.

template <int NT>
static cudaError_t fine_an_vec(const Geom& g, const IuwtArgs& a, cudaStream_t s) {
  dim3 grid(g.n / vec::kT, g.n / vec::kT, g.L);
#define FA(JJ)                                                                                          \
  vec::k_fine_analysis_v<NT, JJ><<<grid, NT, vec::FineA<JJ>::SMEM, s>>>(                                \
      g.n, g.J, a.D, a.U, a.cr, a.k, a.rho, resident_blocks(vec::k_fine_analysis_v<NT, JJ>, NT, vec::FineA<JJ>::SMEM))
  switch (g.j1) {
    case 1: FA(1); break;
    case 2: FA(2); break;
    case 3: FA(3); break;
    default: return cudaErrorInvalidValue;
  }
#undef FA
  return cudaGetLastError();
}

cudaError_t launch_fine_analysis_vec(const Geom& g, const IuwtArgs& a, cudaStream_t s) {
  return g.fnt == 512 ? fine_an_vec<512>(g, a, s) : fine_an_vec<256>(g, a, s);
}

template <int NT>
static cudaError_t fine_adj_vec(const Geom& g, const IuwtArgs& a, cudaStream_t s) {
  dim3 grid(g.n / vec::kT, g.n / vec::kT, g.L);
  const size_t P = (size_t)g.n * g.n;
  const bool from_u = (g.J == g.j1);
  const float* rin = from_u ? a.U + (size_t)g.J * P : a.rin;
  const size_t stride = from_u ? (size_t)(g.J + 1) * P : P;
#define FT(JJ)                                                                                     \
  vec::k_fine_adjoint_v<NT, JJ><<<grid, NT, vec::FineT<JJ>::SMEM, s>>>(                            \
      g.n, g.J, rin, stride, a.U, a.S, resident_blocks(vec::k_fine_adjoint_v<NT, JJ>, NT, vec::FineT<JJ>::SMEM))
  switch (g.j1) {
    case 1: FT(1); break;
    case 2: FT(2); break;
    case 3: FT(3); break;
    default: return cudaErrorInvalidValue;
  }
#undef FT
  return cudaGetLastError();
}

cudaError_t launch_fine_adjoint_vec(const Geom& g, const IuwtArgs& a, cudaStream_t s) {
  return g.fnt == 512 ? fine_adj_vec<512>(g, a, s) : fine_adj_vec<256>(g, a, s);
}

template <int NT>
static cudaError_t coarse_vec(const Geom& g, const float* c_in, float* r_out, float* U, float k, float rho,
                              cudaStream_t s) {
  dim3 grid(1 << (2 * g.j1), g.L);
  const int M = g.n >> g.j1, NL = g.J - g.j1;
#define CV(MM, LL)                                                                                             \
  if (M == MM && NL == LL) {                                                                                   \
    vec::k_coarse_v<NT, MM, LL><<<grid, NT, vec::CoarseV<MM, LL>::SMEM, s>>>(                              \
        g.n, g.J, g.j1, c_in, r_out, U, k, rho,                                                            \
        resident_blocks(vec::k_coarse_v<NT, MM, LL>, NT, vec::CoarseV<MM, LL>::SMEM));                             \
    return cudaGetLastError();                                                                                 \
  }
  CV(32, 1) CV(32, 2) CV(32, 3) CV(64, 1) CV(64, 2) CV(64, 3)
#undef CV
  // 128 x 128 sub-images: dual planes streamed through L2, one block per SM
#define CS(LL)                                                                                              \
  if (M == 128 && NL == LL) {                                                                               \
    vec::k_coarse_s<512, 128, LL><<<grid, 512, vec::CoarseS<128, LL>::SMEM, s>>>(g.n, g.J, g.j1, c_in, r_out, U, \
                                                                                k, rho);                   \
    return cudaGetLastError();                                                                              \
  }
  CS(1) CS(2) CS(3)
#undef CS
  return cudaErrorInvalidValue;
}

cudaError_t launch_coarse_vec(const Geom& g, const float* c_in, float* r_out, float* U, float k, float rho,
                              cudaStream_t s) {
  return g.cnt == 512 ? coarse_vec<512>(g, c_in, r_out, U, k, rho, s)
                                   : coarse_vec<256>(g, c_in, r_out, U, k, rho, s);
}

template <int NT> static cudaError_t vec_configure_nt() {
  cudaError_t e;
#define SET(fn) if ((e = allow_max_dyn_smem(fn))) return e;
  SET((vec::k_fine_analysis_v<NT, 1>)) SET((vec::k_fine_analysis_v<NT, 2>)) SET((vec::k_fine_analysis_v<NT, 3>))
  SET((vec::k_fine_adjoint_v<NT, 1>)) SET((vec::k_fine_adjoint_v<NT, 2>)) SET((vec::k_fine_adjoint_v<NT, 3>))
  SET((vec::k_coarse_v<NT, 32, 1>)) SET((vec::k_coarse_v<NT, 32, 2>)) SET((vec::k_coarse_v<NT, 32, 3>))
  SET((vec::k_coarse_v<NT, 64, 1>)) SET((vec::k_coarse_v<NT, 64, 2>)) SET((vec::k_coarse_v<NT, 64, 3>))
#undef SET
  return cudaSuccess;
}

cudaError_t iuwt_vec_configure() {
  cudaError_t e = vec_configure_nt<256>();
  if (e == cudaSuccess) e = vec_configure_nt<512>();
  if (e == cudaSuccess) e = allow_max_dyn_smem(vec::k_coarse_s<512, 128, 1>);
  if (e == cudaSuccess) e = allow_max_dyn_smem(vec::k_coarse_s<512, 128, 2>);
  if (e == cudaSuccess) e = allow_max_dyn_smem(vec::k_coarse_s<512, 128, 3>);
  return e;
}

}  // namespace muffin
