// Spectral l1 term of the objective without any device allocation.
//
// Some callers cannot allocate device memory at all: code running inside a
// host framework that owns every device byte through its own pool, a plugin
// that is handed fixed buffers, or a memory-capped service whose budget is
// already spent on the cubes.  This entry point serves them.  It evaluates
// sum_n ||W_lambda x^n||_1 (the orthonormal DCT along channels of every pixel
// spectrum, then the l1 norm) with the same kernel as muffin_objective, but
// its scratch -- the per-block partial sums and the DCT tables -- lives in
// one file-scope __device__ array of fixed size instead of a caller
// workspace.  The caller passes only the input cube and the output slot.
#include <cmath>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <string>
#include <vector>

#include "internal.h"
#include "muffin.h"

using namespace muffin;

namespace {

// Layout of the static scratch (bytes, each piece 256-byte aligned).
constexpr size_t kMaxPix = (size_t)1 << 20;       // up to 1024 x 1024 pixels
constexpr int kMaxChan = 256;                      // up to 256 channels
constexpr size_t kPartOff = 0;                                          // doubles, one per block
constexpr size_t kPartBytes = ((kMaxPix + 31) / 32) * sizeof(double);   // 256 KiB
constexpr size_t kTwOff = kPartOff + kPartBytes;                        // float2[L]
constexpr size_t kPostOff = kTwOff + kMaxChan * 8;                      // float2[L]
constexpr size_t kPreOff = kPostOff + kMaxChan * 8;                     // float2[L]
constexpr size_t kInvsOff = kPreOff + kMaxChan * 8;                     // float[L]
constexpr size_t kDenseOff = kInvsOff + kMaxChan * 4;                   // float[L][L]
constexpr size_t kScratchBytes = kDenseOff + (size_t)kMaxChan * kMaxChan * 4;   // ~515 KiB

// Held by every GPU that loads the library until the process exits.
static __device__ __align__(256) unsigned char g_scratch[kScratchBytes];

thread_local std::string g_err;
std::mutex g_mu;
void* g_addr[64] = {};   // device address of g_scratch, per device ordinal

int err(int code, const std::string& m) {
  g_err = m;
  return code;
}

}  // namespace

extern "C" {

const char* muffin_noalloc_last_error(void) { return g_err.c_str(); }

int muffin_spectral_l1_noalloc(const float* d_x, int n_pix, int nchan, double* d_out, cudaStream_t stream) {
  if (!d_x || !d_out) return err(MUFFIN_ERR_ARG, "NULL input or output pointer");
  if (n_pix < 1 || (size_t)n_pix > kMaxPix)
    return err(MUFFIN_ERR_ARG, "n_pix must be in [1, 1048576] (the static scratch holds partial sums for 2^20 pixels)");
  if (nchan < 1 || nchan > kMaxChan)
    return err(MUFFIN_ERR_ARG, "nchan must be in [1, 256] (the static scratch holds DCT tables for 256 channels)");
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return err(MUFFIN_ERR_CUDA, std::string("cudaGetDevice: ") + cudaGetErrorString(e));
  if (dev < 0 || dev >= 64) return err(MUFFIN_ERR_ARG, "device ordinal >= 64");
  char* base = nullptr;
  {
    // once per device, with that device current: the device address of the
    // array (its name in host code is only a host-side stand-in)
    std::lock_guard<std::mutex> lock(g_mu);
    if (!g_addr[dev]) {
      void* p = nullptr;
      e = cudaGetSymbolAddress(&p, g_scratch);
      if (e != cudaSuccess) return err(MUFFIN_ERR_CUDA, std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(e));
      g_addr[dev] = p;
    }
    base = static_cast<char*>(g_addr[dev]);
  }
  if ((e = spectral_configure(nchan)) != cudaSuccess)
    return err(MUFFIN_ERR_CUDA, std::string("kernel configuration: ") + cudaGetErrorString(e));
  // DCT tables for this channel count, computed in FP64 on the host
  const int L = nchan;
  const double pi = 3.14159265358979323846;
  std::vector<float> tw(2 * L), post(2 * L), pre(2 * L), invs(L), dense((size_t)L * L);
  for (int k = 0; k < L; ++k) {
    const double a = -2.0 * pi * k / L;
    tw[2 * k] = (float)std::cos(a); tw[2 * k + 1] = (float)std::sin(a);
    const double sk = k == 0 ? std::sqrt(1.0 / L) : std::sqrt(2.0 / L);
    const double b = pi * k / (2.0 * L);
    post[2 * k] = (float)(sk * std::cos(-b)); post[2 * k + 1] = (float)(sk * std::sin(-b));
    pre[2 * k] = (float)std::cos(b); pre[2 * k + 1] = (float)std::sin(b);
    invs[k] = (float)(1.0 / (sk * L));
    for (int l = 0; l < L; ++l) dense[(size_t)k * L + l] = (float)(sk * std::cos(pi * (2 * l + 1) * k / (2.0 * L)));
  }
  struct Piece { size_t off; const void* src; size_t bytes; };
  const Piece pieces[] = {{kTwOff, tw.data(), tw.size() * 4}, {kPostOff, post.data(), post.size() * 4},
                          {kPreOff, pre.data(), pre.size() * 4}, {kInvsOff, invs.data(), invs.size() * 4},
                          {kDenseOff, dense.data(), dense.size() * 4}};
  for (const Piece& pc : pieces) {
    // pageable source: the copy is staged before the call returns
    e = cudaMemcpyAsync(base + pc.off, pc.src, pc.bytes, cudaMemcpyHostToDevice, stream);
    if (e != cudaSuccess) return err(MUFFIN_ERR_CUDA, std::string("table upload: ") + cudaGetErrorString(e));
  }
  SpecArgs sa{};
  sa.D = d_x;
  sa.tw = reinterpret_cast<const float*>(base + kTwOff);
  sa.post = reinterpret_cast<const float*>(base + kPostOff);
  sa.pre = reinterpret_cast<const float*>(base + kPreOff);
  sa.invs = reinterpret_cast<const float*>(base + kInvsOff);
  sa.dense = reinterpret_cast<const float*>(base + kDenseOff);
  // every block writes its own partial sum, so nothing needs clearing first
  sa.partials = reinterpret_cast<double*>(base + kPartOff);
  int nblocks = 0;
  if ((e = launch_spectral(sa, n_pix, L, SPEC_NORM, stream, &nblocks)) != cudaSuccess)
    return err(MUFFIN_ERR_CUDA, std::string("spectral kernel: ") + cudaGetErrorString(e));
  if ((e = launch_sum_partials(sa.partials, nblocks, d_out, stream)) != cudaSuccess)
    return err(MUFFIN_ERR_CUDA, std::string("reduction: ") + cudaGetErrorString(e));
  return MUFFIN_OK;
}

}  // extern "C"
