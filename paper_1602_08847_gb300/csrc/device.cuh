// Device building blocks shared by the MUFFIN kernels: complex arithmetic,
// the in-register Stockham FFT, the B3 a trous stencil passes, the
// class-permuted plane layout and block reductions.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

namespace muffin {

// Dynamic shared memory a block may opt into on sm_100 / sm_103 (227 KB),
// static shared memory of the kernel included.
constexpr int kMaxDynSmem = 232448;

// Let kernel fn use as much dynamic shared memory as the device allows next to
// its static shared memory.  The largest size is set once for every context:
// a lower limit set for one context would break another.
template <typename F>
inline cudaError_t allow_max_dyn_smem(F* fn) {
  int dev = 0, optin = kMaxDynSmem;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if ((e = cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev)) != cudaSuccess) return e;
  cudaFuncAttributes fa;
  if ((e = cudaFuncGetAttributes(&fa, fn)) != cudaSuccess) return e;
  if ((e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, optin - (int)fa.sharedSizeBytes)))
    return e;
  // prefer the largest shared-memory carve-out so that several blocks fit per SM
  return cudaFuncSetAttribute(fn, cudaFuncAttributePreferredSharedMemoryCarveout, (int)cudaSharedmemCarveoutMaxShared);
}

// ----------------------------------------------------------------- L2 prefetch for the next wave
// Kernels that run one tile per block run in waves of `ahead` resident blocks
// (host: resident_blocks, internal.h).  A block first asks L2 for the inputs
// of the block `ahead` places later in launch order, the one that takes its
// place when this wave ends, so that the next wave's first loads find their
// lines in L2.  prefetch.global.L2 moves no data into the block: a wrong guess
// costs L2 bandwidth only.
__device__ __forceinline__ void pf_line(const float* p) { asm volatile("prefetch.global.L2 [%0];" ::"l"(p)); }

// A contiguous run of `bytes` (a multiple of 16; p 16-byte aligned) into L2 with
// one bulk prefetch.  (Worth it for long runs: the coarse kernel's 16 KB
// sub-images.  Row-sized runs of the fine kernels measured slower this way than
// as per-line prefetches.)
__device__ __forceinline__ void pf_bulk(const float* p, unsigned bytes) {
  asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(p), "r"(bytes) : "memory");
}

// Linear index of the block `ahead` places later in launch order, or -1.
__device__ __forceinline__ int pf_next(int ahead) {
  if (ahead <= 0) return -1;
  const int nb = gridDim.x * gridDim.y * gridDim.z;
  const int id = blockIdx.x + gridDim.x * (blockIdx.y + gridDim.y * blockIdx.z) + ahead;
  return id < nb ? id : -1;
}

// ----------------------------------------------------------------- complex
template <typename T> struct __align__(2 * sizeof(T)) cpx { T x, y; };

template <typename T> __device__ __forceinline__ cpx<T> mk(T a, T b) { cpx<T> r; r.x = a; r.y = b; return r; }
template <typename T> __device__ __forceinline__ cpx<T> add(cpx<T> a, cpx<T> b) { return mk<T>(a.x + b.x, a.y + b.y); }
template <typename T> __device__ __forceinline__ cpx<T> sub(cpx<T> a, cpx<T> b) { return mk<T>(a.x - b.x, a.y - b.y); }
template <typename T> __device__ __forceinline__ cpx<T> mul(cpx<T> a, cpx<T> b) {
  return mk<T>(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
template <typename T> __device__ __forceinline__ cpx<T> conj(cpx<T> a) { return mk<T>(a.x, -a.y); }
template <typename T> __device__ __forceinline__ cpx<T> scale(cpx<T> a, T s) { return mk<T>(a.x * s, a.y * s); }
// a * (dir * i): dir = -1 multiplies by -i, dir = +1 by +i
template <typename T, int DIR> __device__ __forceinline__ cpx<T> rot90(cpx<T> a) {
  return DIR < 0 ? mk<T>(a.y, -a.x) : mk<T>(-a.y, a.x);
}

// ----------------------------------------------------------------- FFT
// Radix plan for N = 2^m (8 <= N <= 1024): radix-8 passes first, then
// radix-4 passes; m = 3a + 2b.
template <int N> struct FftPlan {
  static constexpr int LOG = (N <= 1) ? 0 : 1 + FftPlan<N / 2>::LOG;
  static constexpr int P8 = LOG / 3 - (LOG % 3 == 1 ? 1 : 0);
  static constexpr int P4 = (LOG - 3 * P8) / 2;
  static constexpr int PASSES = P8 + P4;
  static constexpr int T8 = N / 8;   // threads per transform, 8 elements each
};
template <> struct FftPlan<1> { static constexpr int LOG = 0; };

// 4-point DFT in place, direction DIR (-1 forward, +1 inverse).
template <typename T, int DIR>
__device__ __forceinline__ void dft4(cpx<T>& a0, cpx<T>& a1, cpx<T>& a2, cpx<T>& a3) {
  cpx<T> t0 = add(a0, a2), t1 = sub(a0, a2), t2 = add(a1, a3), t3 = rot90<T, DIR>(sub(a1, a3));
  a0 = add(t0, t2); a1 = add(t1, t3); a2 = sub(t0, t2); a3 = sub(t1, t3);
}

// 8-point DFT of v[0..7] (natural order in and out): one radix-2 split into
// two 4-point DFTs with the eighth-root twiddles.
template <typename T, int DIR>
__device__ __forceinline__ void dft8(cpx<T> (&v)[8]) {
  const T s = (T)0.70710678118654752440;
  cpx<T> a0 = add(v[0], v[4]), a1 = add(v[1], v[5]), a2 = add(v[2], v[6]), a3 = add(v[3], v[7]);
  cpx<T> b0 = sub(v[0], v[4]), b1 = sub(v[1], v[5]), b2 = sub(v[2], v[6]), b3 = sub(v[3], v[7]);
  // b_q *= w^q with w = exp(DIR * 2 pi i / 8)
  b1 = mk<T>(s * (b1.x - DIR * b1.y), s * (b1.y + DIR * b1.x));
  b2 = rot90<T, DIR>(b2);
  b3 = mk<T>(s * (-b3.x - DIR * b3.y), s * (-b3.y + DIR * b3.x));
  dft4<T, DIR>(a0, a1, a2, a3);
  dft4<T, DIR>(b0, b1, b2, b3);
  v[0] = a0; v[1] = b0; v[2] = a1; v[3] = b1; v[4] = a2; v[5] = b2; v[6] = a3; v[7] = b3;
}

template <typename T, int DIR>
__device__ __forceinline__ cpx<T> twiddle(const cpx<T>* tw, int idx) {
  cpx<T> w = tw[idx];
  return DIR < 0 ? w : conj(w);
}

// Shared-memory slot of element i with PAD: one spare slot after every 8
// elements.  The first radix-8 pass writes 8 consecutive elements per thread,
// so neighbouring threads' writes are 8 elements apart; the spare slot moves
// them onto different banks, and runs of consecutive elements stay
// consecutive within each group of 8.
template <int PAD> __host__ __device__ __forceinline__ constexpr int fft_slot(int i) { return PAD ? i + (i >> 3) : i; }
template <int N, int PAD> __host__ __device__ constexpr int fft_slots() { return PAD ? N + N / 8 : N; }

// Length-N FFT (unnormalised, sign DIR) by the Stockham auto-sort scheme of
// Govindaraju et al. (SC'08), one thread per 8 elements.
// On entry thread t (0 <= t < N/8) holds v[q] = x[t + q N/8]; on exit it holds
// X[t + q N/8] in natural order.  Intermediate passes go through sm, where
// element i of this transform lives at sm[fft_slot<PAD>(i) * IS].
// tw[m] = exp(-2 pi i m / N).  Every thread of the block must call this the
// same number of times (it synchronises the whole block).
template <typename T, int N, int DIR, int IS, int PAD = 0>
__device__ __forceinline__ void fft_regs(cpx<T> (&v)[8], cpx<T>* sm, const cpx<T>* tw, int t) {
  using PL = FftPlan<N>;
  constexpr int T8 = PL::T8;
  int Ns = 1;
#pragma unroll
  for (int p = 0; p < PL::PASSES; ++p) {
    const bool last = (p == PL::PASSES - 1);
    if (p > 0) {
      __syncthreads();
#pragma unroll
      for (int q = 0; q < 8; ++q) v[q] = sm[fft_slot<PAD>(t + q * T8) * IS];
    }
    if (p < PL::P8) {
      const int k = t % Ns;
      const int step = N / (Ns * 8);
#pragma unroll
      for (int r = 1; r < 8; ++r) v[r] = mul(v[r], twiddle<T, DIR>(tw, r * k * step));
      dft8<T, DIR>(v);
      if (!last) {
        __syncthreads();
        const int base = (t - k) * 8 + k;
#pragma unroll
        for (int r = 0; r < 8; ++r) sm[fft_slot<PAD>(base + r * Ns) * IS] = v[r];
      }
      Ns *= 8;
    } else {
      const int step = N / (Ns * 4);
      const int j0 = t, j1 = t + T8;
      const int k0 = j0 % Ns, k1 = j1 % Ns;
#pragma unroll
      for (int r = 1; r < 4; ++r) {
        v[2 * r] = mul(v[2 * r], twiddle<T, DIR>(tw, r * k0 * step));
        v[2 * r + 1] = mul(v[2 * r + 1], twiddle<T, DIR>(tw, r * k1 * step));
      }
      dft4<T, DIR>(v[0], v[2], v[4], v[6]);
      dft4<T, DIR>(v[1], v[3], v[5], v[7]);
      if (!last) {
        __syncthreads();
        const int b0 = (j0 - k0) * 4 + k0, b1 = (j1 - k1) * 4 + k1;
#pragma unroll
        for (int r = 0; r < 4; ++r) {
          sm[fft_slot<PAD>(b0 + r * Ns) * IS] = v[2 * r];
          sm[fft_slot<PAD>(b1 + r * Ns) * IS] = v[2 * r + 1];
        }
      }
      Ns *= 4;
    }
  }
}

// ----------------------------------------------------------------- IUWT stencils
// B3 spline taps [1, 4, 6, 4, 1] / 16.
__device__ __forceinline__ float b3tap(int k) {
  return k == 2 ? 0.375f : ((k == 1 || k == 3) ? 0.25f : 0.0625f);
}

// Halo (in pixels) that each plane of the fine-scale recursions needs around
// an output tile, for generation GEN and j1 fine levels.
//   analysis:  c_j, j = 0..j1;  adjoint: r_j (j = 0..j1) and u_j (j < j1).
__host__ __device__ constexpr int halo_c(int gen, int j1, int j) {
  // gen1: c_j feeds c_{j+1}; gen2 also needs H c_{j1} on the tile for w_{j1-1}
  return gen == 1 ? ((1 << (j1 + 1)) - (1 << (j + 1)))
                  : ((1 << j1) + (1 << (j1 + 1)) - (1 << (j + 1)));
}
__host__ __device__ constexpr int halo_r(int j) { return (1 << (j + 1)) - 2; }
__host__ __device__ constexpr int halo_u(int gen, int j) {
  return gen == 1 ? halo_r(j + 1) : halo_r(j) + (1 << (j + 2));
}
__host__ __device__ constexpr int halo_max(int gen, int j1) {
  return j1 == 0 ? 0 : (gen == 1 ? (1 << (j1 + 1)) - 2 : 3 * (1 << j1) - 2);
}

// Address of pixel (gy, gx) of an N x N plane stored class-permuted with
// stride s = 2^lgs: the s*s sub-lattices {(gy, gx) : gy = cy mod s, gx = cx
// mod s} are stored one after another, each as an (N/s) x (N/s) row-major
// image.  lgs = 0 is the natural layout.
__device__ __forceinline__ int class_index(int gy, int gx, int n, int lgs) {
  const int s = 1 << lgs, m = n >> lgs;
  return (((gy & (s - 1)) * s + (gx & (s - 1))) * m + (gy >> lgs)) * m + (gx >> lgs);
}

// ----------------------------------------------------------------- reductions
template <typename T>
__device__ __forceinline__ T warp_sum(T v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  return v;
}

// Sum over the block; the result is valid in thread 0.  scratch >= 32 doubles.
__device__ __forceinline__ double block_sum(double v, double* scratch) {
  const int tid = threadIdx.x + blockDim.x * (threadIdx.y + blockDim.y * threadIdx.z);
  const int nth = blockDim.x * blockDim.y * blockDim.z;
  v = warp_sum(v);
  __syncthreads();
  if ((tid & 31) == 0) scratch[tid >> 5] = v;
  __syncthreads();
  double r = 0.0;
  if (tid < 32) {
    r = (tid < (nth + 31) / 32) ? scratch[tid] : 0.0;
    r = warp_sum(r);
  }
  return r;
}

__device__ __forceinline__ float sat1(float u) { return fminf(fmaxf(u, -1.0f), 1.0f); }

// ----------------------------------------------------------------- TMA and mbarriers
__device__ __forceinline__ uint32_t smem_addr(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

// Wait for phase `parity` of the mbarrier at shared address bar, at most
// `limit` polls (each try_wait may suspend for a bounded time); false if it
// gave up.
__device__ __forceinline__ bool mbar_try(uint32_t bar, uint32_t parity, long long limit) {
  uint32_t done = 0;
  for (long long it = 0; it < limit && !done; ++it)
    asm volatile("{\n.reg .pred p;\nmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\nselp.u32 %0, 1, 0, p;\n}\n"
                 : "=r"(done)
                 : "r"(bar), "r"(parity)
                 : "memory");
  return done != 0;
}

__device__ __forceinline__ void mbar_init(uint32_t bar, int count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_expect(uint32_t bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
}

// 2-D tiled TMA copies; map is the address of a CUtensorMap kernel parameter.
__device__ __forceinline__ void tma_load2(uint32_t dst, const void* map, int x, int y, uint32_t bar) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];" ::"r"(dst),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(bar)
      : "memory");
}
__device__ __forceinline__ void tma_store2(const void* map, int x, int y, uint32_t src) {
  asm volatile("cp.async.bulk.tensor.2d.global.shared::cta.bulk_group [%0, {%1, %2}], [%3];" ::"l"(
                   reinterpret_cast<uint64_t>(map)),
               "r"(x), "r"(y), "r"(src)
               : "memory");
}

}  // namespace muffin
