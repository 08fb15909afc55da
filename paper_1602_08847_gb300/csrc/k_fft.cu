// FFT kernels of the data-fidelity gradient (Algorithm 1, first line; Eq. 8)
// and of the FP64 setup / objective paths.
//
// Hot path, FP32, per channel l:  grad_l = F^-1(K_l . F x_l) - b_l with
// K_l = w_l |hhat_l|^2 / N^2 (real, even) and b_l = w_l H_l^T y_l.
//   k_rows_fwd      two real rows -> one complex FFT -> two half-spectrum rows.
//                   The row spectrum is stored as N/2 complex numbers: bins
//                   1..N/2-1, with bin 0 packed as (DC, Nyquist) (both real).
//   k_cols_filter   column FFT, multiply by K, inverse column FFT, in place.
//                   The packed column 0 carries the DC and Nyquist columns as
//                   the real and imaginary parts of one complex sequence.
//   k_rows_inv      inverse row FFT of two rows at once, then the primal
//                   update of Algorithm 1 (second line; Eq. 10) in the
//                   epilogue: X~ = (X - tau (grad + mu_s S + mu_l T))_+,
//                   D = 2 X~ - X, X <- rho X~ + (1 - rho) X.
#include <cuda.h>   // CUtensorMap (the encoder is reached through the runtime's driver entry point)
#include <cstdlib>

#include "device.cuh"
#include "fft_blocks.cuh"
#include "internal.h"

namespace muffin {

// ------------------------------------------------------------------ FP32 rows forward
template <int N>
__global__ void __launch_bounds__(rows_pairs<N>() * (N / 8))
k_rows_fwd(const float* __restrict__ X, cpx<float>* __restrict__ spec, const cpx<float>* __restrict__ twg) {
  constexpr int PAIRS = rows_pairs<N>(), NP = fft_slots<N, 1>();
  __shared__ cpx<float> tw[N];
  __shared__ cpx<float> buf[PAIRS * NP];
  for (int i = threadIdx.x; i < N; i += blockDim.x) tw[i] = twg[i];
  rows_fwd_block<N, PAIRS>(X, spec, tw, buf, blockIdx.y, blockIdx.x);
}

// ------------------------------------------------------------------ FP32 column filter
template <int N>
__global__ void __launch_bounds__(cols_per_cta<N>() * (N / 8))
k_cols_filter(cpx<float>* __restrict__ spec, const float* __restrict__ Kp, const float* __restrict__ Kb,
              const cpx<float>* __restrict__ twg) {
  extern __shared__ __align__(16) unsigned char smraw[];
  cpx<float>* tw = reinterpret_cast<cpx<float>*>(smraw);
  cpx<float>* buf = tw + N;
  for (int i = threadIdx.x; i < N; i += blockDim.x) tw[i] = twg[i];
  cols_block<N, cols_per_cta<N>()>(spec, Kp, Kb, tw, buf, blockIdx.y, blockIdx.x);
}

// ------------------------------------------------------------------ column filter, pipelined (TMA)
// The column filter above as a persistent kernel: a block walks strips of C
// spectrum columns of one channel; the strip ([N][C] complex) and its
// multipliers ([N][C] floats) arrive by 2-D TMA copies into a double buffer,
// so the next strip's loads run under this strip's two FFTs, and the filtered
// strip leaves by TMA stores from the same buffer.  Bounded mbarrier waits: a
// block that gives up records it in g_fft_timeouts, waits (bounded) for its
// copies in flight and returns.
__device__ int g_fft_timeouts;
constexpr long long kFftPolls = 1LL << 22;

struct ColMaps {
  CUtensorMap spec;   // [L N rows][N floats], box [BR][2C]
  CUtensorMap k;      // [L N rows][N/2 floats], box [BR][C]
};

template <int N> __host__ __device__ constexpr int colt_c() { return N >= 512 ? 8 : 16; }
template <int N> __host__ __device__ constexpr int colt_br() { return N < 256 ? N : 256; }
template <int N> struct ColTma {
  static constexpr int C = colt_c<N>(), BR = colt_br<N>();
  static constexpr size_t SPEC = (size_t)N * C * sizeof(cpx<float>), KB = (size_t)N * C * sizeof(float);
  static constexpr size_t OFF_S = 0, OFF_K = 2 * SPEC, OFF_TW = OFF_K + 2 * KB;
  static constexpr size_t OFF_BAR = OFF_TW + (size_t)N * sizeof(cpx<float>);
  static constexpr size_t SMEM = OFF_BAR + 64 + 128;
};

template <int N>
__global__ void __launch_bounds__(colt_c<N>() * (N / 8), 1)
k_cols_tma(const __grid_constant__ ColMaps maps, const float* __restrict__ Kb, const cpx<float>* __restrict__ twg,
           int ntiles) {
  using G = ColTma<N>;
  constexpr int T8 = N / 8, C = G::C, BR = G::BR, H = N / 2, STRIPS = H / C;
  extern __shared__ __align__(16) unsigned char smraw[];
  unsigned char* sm = reinterpret_cast<unsigned char*>((reinterpret_cast<uintptr_t>(smraw) + 127) & ~(uintptr_t)127);
  cpx<float>* Sb = reinterpret_cast<cpx<float>*>(sm + G::OFF_S);
  float* Kbuf = reinterpret_cast<float*>(sm + G::OFF_K);
  cpx<float>* tw = reinterpret_cast<cpx<float>*>(sm + G::OFF_TW);
  const uint32_t bar0 = smem_addr(sm + G::OFF_BAR);
  const int tid = threadIdx.x, c = tid % C, t = tid / C;
  for (int i = tid; i < N; i += blockDim.x) tw[i] = twg[i];
  constexpr uint32_t kBytes = (uint32_t)(G::SPEC + G::KB);
  auto issue = [&](int tile, int s) {
    const int l = tile / STRIPS, strip = tile % STRIPS;
    const uint32_t bar = bar0 + 8 * s;
    mbar_expect(bar, kBytes);
#pragma unroll
    for (int r = 0; r < N / BR; ++r) {
      tma_load2(smem_addr(Sb + (size_t)s * N * C + (size_t)r * BR * C), &maps.spec, 2 * strip * C, l * N + r * BR, bar);
      tma_load2(smem_addr(Kbuf + (size_t)s * N * C + (size_t)r * BR * C), &maps.k, strip * C, l * N + r * BR, bar);
    }
  };
  uint32_t pend = 0, pend_ph = 0;   // thread 0: stages with a load in flight, and its phase parity
  if (tid == 0) {
    mbar_init(bar0, 1);
    mbar_init(bar0 + 8, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    for (int b = 0; b < 2; ++b)
      if ((int)blockIdx.x + b * (int)gridDim.x < ntiles) {
        issue(blockIdx.x + b * gridDim.x, b);
        pend |= 1u << b;
      }
  }
  __syncthreads();
  bool gave_up = false;
  int it = 0;
  for (int tile = blockIdx.x; tile < ntiles; tile += gridDim.x, ++it) {
    const int s = it & 1;
    const uint32_t ph = (uint32_t)(it >> 1) & 1u;
    const bool ok = mbar_try(bar0 + 8 * s, ph, kFftPolls);
    if (__syncthreads_or(!ok)) { gave_up = true; break; }
    if (tid == 0) pend &= ~(1u << s);
    const int l = tile / STRIPS, strip = tile % STRIPS;
    const int kx = strip * C + c;
    cpx<float>* buf = Sb + (size_t)s * N * C;
    const float* Kt = Kbuf + (size_t)s * N * C;
    cpx<float> v[8];
    float ka[8], kb[8];
#pragma unroll
    for (int q = 0; q < 8; ++q) {
      v[q] = buf[(t + q * T8) * C + c];
      ka[q] = Kt[(t + q * T8) * C + c];
      kb[q] = kx == 0 ? __ldg(Kb + (size_t)l * N + t + q * T8) : 0.0f;
    }
    fft_regs<float, N, -1, C>(v, buf + c, tw, t);
    __syncthreads();
#pragma unroll
    for (int q = 0; q < 8; ++q) buf[(t + q * T8) * C + c] = v[q];
    __syncthreads();
#pragma unroll
    for (int q = 0; q < 8; ++q) {
      const int pos = t + q * T8;
      if (kx == 0) {
        const cpx<float> zm = buf[((N - pos) & (N - 1)) * C + c];
        v[q] = add(scale(v[q], ka[q]), scale(conj(zm), kb[q]));
      } else {
        v[q] = scale(v[q], ka[q]);
      }
    }
    fft_regs<float, N, 1, C>(v, buf + c, tw, t);
    __syncthreads();
#pragma unroll
    for (int q = 0; q < 8; ++q) buf[(t + q * T8) * C + c] = v[q];
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    __syncthreads();
    if (tid == 0) {
#pragma unroll
      for (int r = 0; r < N / BR; ++r)
        tma_store2(&maps.spec, 2 * strip * C, l * N + r * BR, smem_addr(buf + (size_t)r * BR * C));
      asm volatile("cp.async.bulk.commit_group;" ::: "memory");
      const int next = tile + 2 * gridDim.x;
      if (next < ntiles) {
        asm volatile("cp.async.bulk.wait_group.read 0;" ::: "memory");
        issue(next, s);
        pend |= 1u << s;
        pend_ph = (pend_ph & ~(1u << s)) | ((((uint32_t)(it >> 1) + 1u) & 1u) << s);
      }
    }
  }
  if (tid == 0) {
    if (gave_up) {
      atomicAdd(&g_fft_timeouts, 1);
      for (int b = 0; b < 2; ++b)
        if ((pend >> b) & 1u) mbar_try(bar0 + 8 * b, (pend_ph >> b) & 1u, kFftPolls);
    }
    asm volatile("cp.async.bulk.wait_group 0;" ::: "memory");
  }
}

typedef CUresult (*FftEncodeFn)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

static FftEncodeFn fft_encoder() {
  static FftEncodeFn fn = nullptr;
  static bool tried = false;
  if (!tried) {
    tried = true;
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<FftEncodeFn>(p);
  }
  return fn;
}

// 2-D float32 map: rows x width floats (row pitch = width), box bh x bw.
static bool fft_map(CUtensorMap* m, const float* base, size_t rows, size_t width, int bw, int bh) {
  FftEncodeFn enc = fft_encoder();
  if (!enc) return false;
  const cuuint64_t dims[2] = {(cuuint64_t)width, (cuuint64_t)rows};
  const cuuint64_t strides[1] = {(cuuint64_t)width * sizeof(float)};
  const cuuint32_t box[2] = {(cuuint32_t)bw, (cuuint32_t)bh};
  const cuuint32_t estr[2] = {1, 1};
  return enc(m, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, const_cast<float*>(base), dims, strides, box, estr,
             CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
             CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

int fft_take_timeouts() {
  int v = 0, zero = 0;
  if (cudaMemcpyFromSymbol(&v, g_fft_timeouts, sizeof(int)) != cudaSuccess) return -1;
  if (v != 0 && cudaMemcpyToSymbol(g_fft_timeouts, &zero, sizeof(int)) != cudaSuccess) return -1;
  return v;
}

template <int N>
static cudaError_t cols_tma_n(float* spec, const float* Kp, const float* Kb, int L, const float* twf, cudaStream_t s) {
  using G = ColTma<N>;
  ColMaps maps;
  if (!fft_map(&maps.spec, spec, (size_t)L * N, N, 2 * G::C, G::BR) ||
      !fft_map(&maps.k, Kp, (size_t)L * N, N / 2, G::C, G::BR))
    return cudaErrorNotSupported;
  static int resident = 0;
  if (!resident) {
    int dev = 0, sms = 1, occ = 1;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_cols_tma<N>, G::C * (N / 8), G::SMEM) != cudaSuccess ||
        occ < 1)
      occ = 1;
    resident = (sms > 0 ? sms : 1) * occ;
  }
  const int ntiles = L * (N / 2 / G::C);
  k_cols_tma<N><<<ntiles < resident ? ntiles : resident, G::C * (N / 8), G::SMEM, s>>>(
      maps, Kb, reinterpret_cast<const cpx<float>*>(twf), ntiles);
  return cudaGetLastError();
}

// ------------------------------------------------------------------ FP32 rows inverse + primal
template <int N, int MODE>
__global__ void __launch_bounds__(rows_pairs<N>() * (N / 8), 2)
k_rows_inv(const cpx<float>* __restrict__ spec, PrimalArgs a, float* __restrict__ out,
           const cpx<float>* __restrict__ twg) {
  constexpr int PAIRS = rows_pairs<N>(), NP = fft_slots<N, 1>();
  __shared__ cpx<float> tw[N];
  __shared__ cpx<float> buf[PAIRS * NP];
  for (int i = threadIdx.x; i < N; i += blockDim.x) tw[i] = twg[i];
  rows_inv_block<N, PAIRS, MODE>(spec, a, out, tw, buf, blockIdx.y, blockIdx.x);
}

// ------------------------------------------------------------------ FP64 full complex FFT (setup, objective)
template <int N> __host__ __device__ constexpr int rows64_per_cta() { return (2048 / N) < 1 ? 1 : (2048 / N); }

template <int N, int DIR>
__global__ void __launch_bounds__(rows64_per_cta<N>() * (N / 8))
k_c2c_rows64(const void* __restrict__ in, int mode_in, cpx<double>* __restrict__ z, int nrows_total,
             const cpx<double>* __restrict__ twg) {
  constexpr int T8 = N / 8, R = rows64_per_cta<N>();
  extern __shared__ __align__(16) unsigned char smraw[];
  cpx<double>* tw = reinterpret_cast<cpx<double>*>(smraw);
  cpx<double>* buf = tw + N;
  const int f = threadIdx.x / T8, t = threadIdx.x % T8;
  for (int i = threadIdx.x; i < N; i += blockDim.x) tw[i] = twg[i];
  const int row = blockIdx.x * R + f;          // global row index l*N + y
  const bool ok = row < nrows_total;
  cpx<double> v[8];
#pragma unroll
  for (int q = 0; q < 8; ++q) {
    const int x = t + q * T8;
    v[q] = mk<double>(0.0, 0.0);
    if (ok) {
      if (mode_in == 0) {
        v[q] = reinterpret_cast<const cpx<double>*>(in)[(size_t)row * N + x];
      } else if (mode_in == 1) {
        // PSF given with its peak at (N/2, N/2): read it moved to (0, 0)
        const int l = row / N, y = row % N;
        const float* p = reinterpret_cast<const float*>(in) + (size_t)l * N * N;
        v[q] = mk<double>((double)p[((y + N / 2) & (N - 1)) * N + ((x + N / 2) & (N - 1))], 0.0);
      } else {
        v[q] = mk<double>((double)reinterpret_cast<const float*>(in)[(size_t)row * N + x], 0.0);
      }
    }
  }
  __syncthreads();
  fft_regs<double, N, DIR, 1>(v, buf + f * N, tw, t);
  if (ok) {
#pragma unroll
    for (int q = 0; q < 8; ++q) z[(size_t)row * N + t + q * T8] = v[q];
  }
}

template <int N> __host__ __device__ constexpr int cols64_per_cta() { return N >= 512 ? 4 : 8; }

// Column FFT of the full complex spectrum, in place.  With FID set (forward
// only) the epilogue also sums w_l |hhat z - yhat|^2 / (2 N^2) of the block.
template <int N, int DIR, int FID>
__global__ void __launch_bounds__(cols64_per_cta<N>() * (N / 8))
k_c2c_cols64(cpx<double>* __restrict__ z, const cpx<double>* __restrict__ twg, const cpx<double>* __restrict__ hhat,
             const cpx<double>* __restrict__ yhat, const double* __restrict__ w, double* __restrict__ partials) {
  constexpr int T8 = N / 8, C = cols64_per_cta<N>();
  extern __shared__ __align__(16) unsigned char smraw[];
  cpx<double>* tw = reinterpret_cast<cpx<double>*>(smraw);
  cpx<double>* buf = tw + N;
  __shared__ double red[32];
  const int c = threadIdx.x % C, t = threadIdx.x / C;
  for (int i = threadIdx.x; i < N; i += blockDim.x) tw[i] = twg[i];
  const int l = blockIdx.y;
  const int kx = blockIdx.x * C + c;
  const size_t base = (size_t)l * N * N;
  cpx<double> v[8];
#pragma unroll
  for (int q = 0; q < 8; ++q) v[q] = z[base + (size_t)(t + q * T8) * N + kx];
  __syncthreads();
  fft_regs<double, N, DIR, C>(v, buf + c, tw, t);
  if (FID) {
    double acc = 0.0;
#pragma unroll
    for (int q = 0; q < 8; ++q) {
      const size_t idx = base + (size_t)(t + q * T8) * N + kx;
      const cpx<double> r = sub(mul(hhat[idx], v[q]), yhat[idx]);
      acc += r.x * r.x + r.y * r.y;
    }
    const double tot = block_sum(acc, red);
    if (threadIdx.x == 0)
      partials[blockIdx.y * gridDim.x + blockIdx.x] = tot * w[l] * 0.5 / ((double)N * (double)N);
  } else {
#pragma unroll
    for (int q = 0; q < 8; ++q) z[base + (size_t)(t + q * T8) * N + kx] = v[q];
  }
}

__global__ void k_build_K(const cpx<double>* __restrict__ hhat, const double* __restrict__ w, float* __restrict__ Kp,
                          float* __restrict__ Kb, int n, int L) {
  const int H = n / 2;
  const size_t total = (size_t)L * n * H;
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < total; i += (size_t)gridDim.x * blockDim.x) {
    const int kx = (int)(i % H);
    const size_t lr = i / H;              // l * n + ky
    const int l = (int)(lr / n);
    const double s = w[l] / ((double)n * (double)n);
    const cpx<double> h0 = hhat[lr * n + kx];
    const double k0 = h0.x * h0.x + h0.y * h0.y;
    if (kx == 0) {
      const cpx<double> hn = hhat[lr * n + H];
      const double kn = hn.x * hn.x + hn.y * hn.y;
      Kp[i] = (float)(0.5 * (k0 + kn) * s);
      Kb[lr] = (float)(0.5 * (k0 - kn) * s);
    } else {
      Kp[i] = (float)(k0 * s);
    }
  }
}

__global__ void k_mul_conj(const cpx<double>* __restrict__ hhat, cpx<double>* __restrict__ z, size_t total) {
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < total; i += (size_t)gridDim.x * blockDim.x)
    z[i] = mul(conj(hhat[i]), z[i]);
}

__global__ void k_real_to_float(const cpx<double>* __restrict__ z, const double* __restrict__ w, float* __restrict__ out,
                                int n, size_t total) {
  const double inv = 1.0 / ((double)n * (double)n);
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < total; i += (size_t)gridDim.x * blockDim.x) {
    const int l = (int)(i / ((size_t)n * n));
    out[i] = (float)(z[i].x * inv * w[l]);
  }
}

__global__ void k_max_abs2(const cpx<double>* __restrict__ hhat, const double* __restrict__ w, int n, size_t total,
                           double* __restrict__ partials) {
  __shared__ double red[32];
  double m = 0.0;
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < total; i += (size_t)gridDim.x * blockDim.x) {
    const int l = (int)(i / ((size_t)n * n));
    const cpx<double> h = hhat[i];
    m = fmax(m, w[l] * (h.x * h.x + h.y * h.y));
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) m = fmax(m, __shfl_down_sync(0xffffffffu, m, o));
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = m;
  __syncthreads();
  if (threadIdx.x < 32) {
    m = threadIdx.x < (blockDim.x + 31) / 32 ? red[threadIdx.x] : 0.0;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) m = fmax(m, __shfl_down_sync(0xffffffffu, m, o));
    if (threadIdx.x == 0) partials[blockIdx.x] = m;
  }
}

// ------------------------------------------------------------------ launchers
#define MUFFIN_N_SWITCH(n, CALL) \
  switch (n) {                   \
    case 16: CALL(16); break;    \
    case 32: CALL(32); break;    \
    case 64: CALL(64); break;    \
    case 128: CALL(128); break;  \
    case 256: CALL(256); break;  \
    case 512: CALL(512); break;  \
    case 1024: CALL(1024); break;\
    default: return cudaErrorInvalidValue; \
  }

cudaError_t launch_rows_fwd(const float* X, float* spec, int n, int L, const float* twf, cudaStream_t s) {
#define CALL(NN)                                                                                   \
  {                                                                                                \
    dim3 grid((NN / 2) / rows_pairs<NN>(), L);                                                     \
    k_rows_fwd<NN><<<grid, rows_pairs<NN>() * (NN / 8), 0, s>>>(X, reinterpret_cast<cpx<float>*>(spec), \
                                                               reinterpret_cast<const cpx<float>*>(twf)); \
  }
  MUFFIN_N_SWITCH(n, CALL)
#undef CALL
  return cudaGetLastError();
}

template <int N> static cudaError_t cols_filter_n(float* spec, const float* Kp, const float* Kb, int L, const float* twf,
                                                  cudaStream_t s) {
  constexpr int C = cols_per_cta<N>();
  const size_t smem = (size_t)(N + N * C) * sizeof(cpx<float>);
  dim3 grid((N / 2) / C, L);
  k_cols_filter<N><<<grid, C * (N / 8), smem, s>>>(reinterpret_cast<cpx<float>*>(spec), Kp, Kb,
                                                   reinterpret_cast<const cpx<float>*>(twf));
  return cudaGetLastError();
}

cudaError_t launch_cols_filter(float* spec, const float* Kp, const float* Kb, int n, int L, const float* twf,
                               cudaStream_t s) {
  // the pipelined kernel for the larger planes (16-byte aligned arrays; MUFFIN_COLS_PLAIN: the plain one)
  if ((n == 256 || n == 512) && ((uintptr_t)spec & 15) == 0 && ((uintptr_t)Kp & 15) == 0 &&
      getenv("MUFFIN_COLS_PLAIN") == nullptr) {
    switch (n) {
      case 256: return cols_tma_n<256>(spec, Kp, Kb, L, twf, s);
      case 512: return cols_tma_n<512>(spec, Kp, Kb, L, twf, s);
    }
  }
#define CALL(NN) return cols_filter_n<NN>(spec, Kp, Kb, L, twf, s);
  MUFFIN_N_SWITCH(n, CALL)
#undef CALL
  return cudaErrorInvalidValue;
}

cudaError_t launch_rows_inv_primal(const float* spec, const PrimalArgs& a, int n, int L, const float* twf,
                                   cudaStream_t s) {
#define CALL(NN)                                                                                            \
  {                                                                                                         \
    dim3 grid((NN / 2) / rows_pairs<NN>(), L);                                                              \
    k_rows_inv<NN, 0><<<grid, rows_pairs<NN>() * (NN / 8), 0, s>>>(reinterpret_cast<const cpx<float>*>(spec), a, \
                                                                   nullptr, reinterpret_cast<const cpx<float>*>(twf)); \
  }
  MUFFIN_N_SWITCH(n, CALL)
#undef CALL
  return cudaGetLastError();
}

cudaError_t launch_rows_inv_plain(const float* spec, float* out, int n, int L, const float* twf, cudaStream_t s) {
  PrimalArgs a{};
#define CALL(NN)                                                                                            \
  {                                                                                                         \
    dim3 grid((NN / 2) / rows_pairs<NN>(), L);                                                              \
    k_rows_inv<NN, 1><<<grid, rows_pairs<NN>() * (NN / 8), 0, s>>>(reinterpret_cast<const cpx<float>*>(spec), a, \
                                                                   out, reinterpret_cast<const cpx<float>*>(twf)); \
  }
  MUFFIN_N_SWITCH(n, CALL)
#undef CALL
  return cudaGetLastError();
}

template <int N, int DIR> static cudaError_t rows64_n(const void* in, int mode_in, void* z, int L, const void* twd,
                                                      cudaStream_t s) {
  constexpr int R = rows64_per_cta<N>();
  const size_t smem = (size_t)(N + R * N) * sizeof(cpx<double>);
  const int rows = L * N;
  k_c2c_rows64<N, DIR><<<(rows + R - 1) / R, R * (N / 8), smem, s>>>(in, mode_in, reinterpret_cast<cpx<double>*>(z),
                                                                     rows, reinterpret_cast<const cpx<double>*>(twd));
  return cudaGetLastError();
}

cudaError_t launch_c2c_rows64(const void* in, int mode_in, void* z, int n, int L, int dir, const void* twd,
                              cudaStream_t s) {
#define CALL(NN) return dir < 0 ? rows64_n<NN, -1>(in, mode_in, z, L, twd, s) : rows64_n<NN, 1>(in, mode_in, z, L, twd, s);
  MUFFIN_N_SWITCH(n, CALL)
#undef CALL
  return cudaErrorInvalidValue;
}

template <int N, int DIR, int FID>
static cudaError_t cols64_n(void* z, int L, const void* twd, const void* hhat, const void* yhat, const double* w,
                            double* partials, int* nparts, cudaStream_t s) {
  constexpr int C = cols64_per_cta<N>();
  const size_t smem = (size_t)(N + N * C) * sizeof(cpx<double>);
  dim3 grid(N / C, L);
  if (nparts) *nparts = grid.x * grid.y;
  k_c2c_cols64<N, DIR, FID><<<grid, C * (N / 8), smem, s>>>(
      reinterpret_cast<cpx<double>*>(z), reinterpret_cast<const cpx<double>*>(twd),
      reinterpret_cast<const cpx<double>*>(hhat), reinterpret_cast<const cpx<double>*>(yhat), w, partials);
  return cudaGetLastError();
}

cudaError_t launch_c2c_cols64(void* z, int n, int L, int dir, const void* twd, cudaStream_t s) {
#define CALL(NN)                                                                                     \
  return dir < 0 ? cols64_n<NN, -1, 0>(z, L, twd, nullptr, nullptr, nullptr, nullptr, nullptr, s) \
                 : cols64_n<NN, 1, 0>(z, L, twd, nullptr, nullptr, nullptr, nullptr, nullptr, s);
  MUFFIN_N_SWITCH(n, CALL)
#undef CALL
  return cudaErrorInvalidValue;
}

cudaError_t launch_cols64_fidelity(void* z, const void* hhat, const void* yhat, const double* w, int n, int L,
                                   const void* twd, double* partials, int* nparts, cudaStream_t s) {
#define CALL(NN) return cols64_n<NN, -1, 1>(z, L, twd, hhat, yhat, w, partials, nparts, s);
  MUFFIN_N_SWITCH(n, CALL)
#undef CALL
  return cudaErrorInvalidValue;
}

cudaError_t launch_build_K(const void* hhat, const double* w, float* Kp, float* Kb, int n, int L, cudaStream_t s) {
  const size_t total = (size_t)L * n * (n / 2);
  const int blocks = (int)((total + 255) / 256 < 65535 ? (total + 255) / 256 : 65535);
  k_build_K<<<blocks, 256, 0, s>>>(reinterpret_cast<const cpx<double>*>(hhat), w, Kp, Kb, n, L);
  return cudaGetLastError();
}

cudaError_t launch_mul_conj(const void* hhat, void* z, int n, int L, cudaStream_t s) {
  const size_t total = (size_t)L * n * n;
  const int blocks = (int)((total + 255) / 256 < 65535 ? (total + 255) / 256 : 65535);
  k_mul_conj<<<blocks, 256, 0, s>>>(reinterpret_cast<const cpx<double>*>(hhat), reinterpret_cast<cpx<double>*>(z),
                                    total);
  return cudaGetLastError();
}

cudaError_t launch_real_to_float(const void* z, const double* w, float* out, int n, int L, cudaStream_t s) {
  const size_t total = (size_t)L * n * n;
  const int blocks = (int)((total + 255) / 256 < 65535 ? (total + 255) / 256 : 65535);
  k_real_to_float<<<blocks, 256, 0, s>>>(reinterpret_cast<const cpx<double>*>(z), w, out, n, total);
  return cudaGetLastError();
}

cudaError_t launch_max_abs2(const void* hhat, const double* w, int n, int L, double* partials, int* nparts,
                            cudaStream_t s) {
  const size_t total = (size_t)L * n * n;
  int blocks = (int)((total + 255) / 256);
  if (blocks > 1024) blocks = 1024;
  *nparts = blocks;
  k_max_abs2<<<blocks, 256, 0, s>>>(reinterpret_cast<const cpx<double>*>(hhat), w, n, total, partials);
  return cudaGetLastError();
}

// Shared-memory opt-in of the instantiations for side n.  Called once per
// context before any launch (and so before any stream capture).
template <int N> static cudaError_t configure_n() {
  cudaError_t e;
  if constexpr (N == 256 || N == 512) {
    if ((e = allow_max_dyn_smem(k_cols_tma<N>))) return e;
  }
  if ((e = allow_max_dyn_smem(k_cols_filter<N>))) return e;
  if ((e = allow_max_dyn_smem(k_c2c_rows64<N, -1>))) return e;
  if ((e = allow_max_dyn_smem(k_c2c_rows64<N, 1>))) return e;
  if ((e = allow_max_dyn_smem(k_c2c_cols64<N, -1, 0>))) return e;
  if ((e = allow_max_dyn_smem(k_c2c_cols64<N, 1, 0>))) return e;
  return allow_max_dyn_smem(k_c2c_cols64<N, -1, 1>);
}

cudaError_t fft_configure(int n) {
#define CALL(NN) return configure_n<NN>();
  MUFFIN_N_SWITCH(n, CALL)
#undef CALL
  return cudaErrorInvalidValue;
}

}  // namespace muffin
