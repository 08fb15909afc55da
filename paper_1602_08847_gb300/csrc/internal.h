// Host-side launchers of the MUFFIN kernels (internal to libmuffin).
#pragma once
#include <cuda_runtime.h>
#include <stddef.h>
#include <stdint.h>

#include <cstdlib>
#include <map>
#include <mutex>

namespace muffin {

// Geometry of one cube as the kernels see it.
struct Geom {
  int n;        // image side N (power of two, 16..1024)
  int L;        // channels
  int J;        // IUWT detail scales
  int gen;      // IUWT generation (1 or 2)
  int j1;       // fine levels computed on halo tiles; levels >= j1 run class-permuted
  int cs;       // blocks per cluster of the coarse kernel (0: single-block streaming kernel)
  int dict = 0; // W_s: 0 IUWT, 1 union of eight Daubechies bases (k_dwt.cu)
  int vec = 1;  // generation 1: the vectorised pass kernels (k_iuwt_vec.cu) where the geometry allows
  int fnt = 256;  // threads per block of the vectorised fine kernels (256 or 512)
  int cnt = 256;  // threads per block of the vectorised resident coarse kernel (256 or 512)
};

// ---- FFT path (k_fft.cu) ----
// Per-channel H_l^T H_l x_l (weights and 1/N^2 folded into Kp, Kb) followed
// by the primal step of Algorithm 1, or, in power mode, only H^T H x -> out.
cudaError_t launch_rows_fwd(const float* X, float* spec, int n, int L, const float* twf, cudaStream_t s);
// Blocks of the pipelined column filter that gave up a bounded wait since the
// last call (resets the count); -1 on a CUDA error.
int fft_take_timeouts();
cudaError_t launch_cols_filter(float* spec, const float* Kp, const float* Kb, int n, int L, const float* twf,
                               cudaStream_t s);
struct PrimalArgs {
  const float* b; const float* S; const float* T;
  float* X; float* D;
  float tau, mu_s, mu_l, rho;
};
cudaError_t launch_rows_inv_primal(const float* spec, const PrimalArgs& a, int n, int L, const float* twf,
                                   cudaStream_t s);
cudaError_t launch_rows_inv_plain(const float* spec, float* out, int n, int L, const float* twf, cudaStream_t s);

// FP64 full-complex 2-D FFT helpers for setup and the objective.
// mode_in: 0 complex input z; 1 real float input with ifftshift; 2 real float input.
cudaError_t launch_c2c_rows64(const void* in, int mode_in, void* z, int n, int L, int dir, const void* twd,
                              cudaStream_t s);
cudaError_t launch_c2c_cols64(void* z, int n, int L, int dir, const void* twd, cudaStream_t s);
cudaError_t launch_build_K(const void* hhat, const double* w, float* Kp, float* Kb, int n, int L, cudaStream_t s);
cudaError_t launch_mul_conj(const void* hhat, void* z, int n, int L, cudaStream_t s);
cudaError_t launch_real_to_float(const void* z, const double* w, float* out, int n, int L, cudaStream_t s);
// sum_l w_l / (2 N^2) sum_k |hhat z - yhat|^2 over column tiles -> partials
cudaError_t launch_cols64_fidelity(void* z, const void* hhat, const void* yhat, const double* w, int n, int L,
                                   const void* twd, double* partials, int* nparts, cudaStream_t s);
cudaError_t launch_max_abs2(const void* hhat, const double* w, int n, int L, double* partials, int* nparts,
                            cudaStream_t s);

// ---- IUWT (k_iuwt.cu) ----
enum IuwtMode { MODE_UPDATE = 0, MODE_LINEAR = 1, MODE_NORM = 2, MODE_ADJ = 3 };
struct IuwtArgs {
  const float* D;    // analysis input (natural layout)
  float* U;          // [L][J+1][N*N]; planes j >= j1 class-permuted (stride 2^j1)
  float* cr;         // c_{j1} out of the fine analysis / r_{j1} out of the coarse part
  const float* rin;  // r_{j1} read by the fine adjoint
  float* S;          // W_s^T U out of the fine adjoint (natural)
  float k;           // sigma * mu_s
  float rho;
  double* partials;  // NORM mode: one partial sum per block
};
size_t fine_smem_bytes(const Geom& g, int adjoint);
size_t coarse_smem_bytes(const Geom& g);
// host-only size estimates used to choose the split j1 (no CUDA calls)
size_t fine_smem_bytes(int gen, int j1, int adjoint);
size_t coarse_cl_smem_bytes(int n, int J, int gen, int j1, int cs);
size_t coarse_stream_smem_bytes(int n, int gen, int j1);
int coarse_cluster_size(int n, int J, int gen, int j1, size_t budget);
cudaError_t launch_fine_analysis(const Geom& g, const IuwtArgs& a, int mode, cudaStream_t s, int* nblocks);
cudaError_t launch_fine_adjoint(const Geom& g, const IuwtArgs& a, cudaStream_t s);
cudaError_t launch_coarse(const Geom& g, const float* c_in, float* r_out, float* U, float k, float rho, int mode,
                          double* partials, cudaStream_t s, int* nblocks);
// Opt the wavelet kernels into shared memory and pick g.cs for this device.
cudaError_t iuwt_configure(Geom& g);
// Vectorised generation-1 kernels of the pass (k_iuwt_vec.cu): 64 x 64 fine
// tiles with j1 in 1..3, coarse sub-images of 32 or 64 with 1..3 levels.
bool iuwt_vec_fine_ok(const Geom& g);
bool iuwt_vec_coarse_ok(const Geom& g);
cudaError_t launch_fine_analysis_vec(const Geom& g, const IuwtArgs& a, cudaStream_t s);
cudaError_t launch_fine_adjoint_vec(const Geom& g, const IuwtArgs& a, cudaStream_t s);
cudaError_t launch_coarse_vec(const Geom& g, const float* c_in, float* r_out, float* U, float k, float rho,
                              cudaStream_t s);
cudaError_t iuwt_vec_configure();
cudaError_t fft_configure(int n);

// ---- W_s as a union of eight orthonormal Daubechies bases (k_dwt.cu) ----
constexpr int kDbBases = 8;
// Daubechies lowpass filter with p vanishing moments (1 <= p <= 8), 2p taps,
// by spectral factorisation (host, double precision); false if p is out of range.
bool daubechies_lowpass(int p, double* h);
struct DwtArgs {
  const float* src;  // analysis input [L][N][N] (shared by the bases)
  float* U;          // coefficients / duals [L][8][N][N], Mallat layout per basis
  float* W1;         // scratch [L][8][N][N]
  float* W2;         // scratch [L][8][N][N]
  float* S;          // adjoint output [L][N][N]
  float k;           // sigma * mu_s (update mode)
  float rho;
};
// Upload the filters once per process and device.
cudaError_t dwt_configure();
// mode MODE_UPDATE: U <- rho sat(U + k W_s src) + (1 - rho) U; MODE_LINEAR: U = W_s src.
cudaError_t launch_dwt_analysis(const Geom& g, const DwtArgs& a, int mode, cudaStream_t s);
// S = W_s^T U.
cudaError_t launch_dwt_adjoint(const Geom& g, const DwtArgs& a, cudaStream_t s);
// sum |x| over n floats -> one partial per block (at most 1024).
cudaError_t launch_abs_sum(const float* x, size_t n, double* partials, int* nparts, cudaStream_t s);

// ---- spectral step (k_spectral.cu) ----
enum SpecMode { SPEC_UPDATE = 0, SPEC_NORM = 1, SPEC_TONLY = 2 };
struct SpecArgs {
  const float* D;    // analysis input
  float* V;          // dual variable (updated in place)
  float* T;          // W_lambda^T V out (unscaled)
  float k;           // sigma * mu_lambda
  float rho;
  const float* tw;   // FFT twiddles of length L (float2)
  const float* post; // DCT post-twiddles (float2) [L]
  const float* pre;  // inverse pre-twiddles (float2) [L]
  const float* invs; // 1 / (s_k L) [L]
  const float* dense;// dense orthonormal DCT matrix [L][L]
  double* partials;
};
bool spectral_uses_fft(int L);
cudaError_t spectral_configure(int L);
// Blocks of the pipelined spectral kernel that gave up a bounded wait since the
// last call (resets the count); -1 on a CUDA error.  Synchronises the device.
int spectral_take_timeouts();
cudaError_t launch_spectral(const SpecArgs& a, int npix, int L, int mode, cudaStream_t s, int* nblocks);

// ---- persistent batch pass (k_batch.cu) ----
// One cooperative launch runs one pass of Algorithm 1 over every cube of a
// batch: six stages (row FFTs, column filter, inverse rows + primal step,
// spatial analysis, coarse levels, spatial adjoint with the spectral step),
// each a work list over (cube, channel, tile) items, separated by grid
// barriers whose waits give up after `polls` polls and set *err.
constexpr int kMaxBatchCubes = 8;
constexpr int kBatchThreads = 512;
struct BatchCube {
  int n, L, J, j1;
  int spatial, spectral;
  float* spec;
  const float* Kp;
  const float* Kb;
  const float* twf;
  PrimalArgs pa;
  IuwtArgs ia;
  SpecArgs sa;
};
struct BatchArgs {
  int nc;
  BatchCube c[kMaxBatchCubes];
  unsigned* bar;     // [0] arrivals, [1] generation; zero before each launch
  int* err;          // set to 1 when a barrier wait gave up (sticky)
  long long polls;
};
// Whether the persistent kernel has a path for this cube geometry.
bool batch_cube_ok(const Geom& g, int spatial, int spectral);
// Dynamic shared memory the persistent kernel needs for these cubes.
size_t batch_smem_bytes(const BatchArgs& a);
cudaError_t batch_configure();
// Largest co-resident grid for smem bytes (0 if the kernel cannot run).
int batch_grid(size_t smem);
cudaError_t launch_batch_pass(const BatchArgs& a, size_t smem, int grid, cudaStream_t s);

// ---- misc (k_misc.cu) ----
cudaError_t launch_sum_partials(const double* partials, int n, double* out, cudaStream_t s);
cudaError_t launch_max_partials(const double* partials, int n, double* out, cudaStream_t s);
cudaError_t launch_dot(const float* a, const float* b, size_t n, double* partials, int* nparts, cudaStream_t s);
cudaError_t launch_scale(float* x, size_t n, const double* num, const double* den, cudaStream_t s);
cudaError_t launch_fill_random(float* x, size_t n, uint64_t seed, cudaStream_t s);
cudaError_t launch_permute_planes(const float* src, float* dst, int n, int L, int J, int j1, int to_class,
                                  cudaStream_t s);
cudaError_t launch_nonfinite_count(const float* x, size_t n, int* count, cudaStream_t s);

// How far ahead in launch order a block prefetches inputs into L2: the blocks
// of kernel fn resident on the device at once (one wave), times
// MUFFIN_L2_PREFETCH when that is set (0: no prefetch; 2: two waves ahead).
template <typename F>
inline int resident_blocks(F* fn, int nt, size_t smem) {
  static std::mutex mu;
  static std::map<const void*, int> known;
  static const int waves = [] {
    const char* e = getenv("MUFFIN_L2_PREFETCH");
    const int w = e ? atoi(e) : 1;
    return w < 0 ? 0 : (w > 4 ? 4 : w);
  }();
  if (waves == 0) return 0;
  std::lock_guard<std::mutex> lk(mu);
  const auto it = known.find(reinterpret_cast<const void*>(fn));
  if (it != known.end()) return it->second;
  int dev = 0, sms = 0, occ = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
      cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, fn, nt, smem) != cudaSuccess) {
    cudaGetLastError();
    return 0;
  }
  return known[reinterpret_cast<const void*>(fn)] = sms * occ * waves;
}

}  // namespace muffin
