// Host runtime of libmuffin: parameter checks, workspace layout, set-up
// (Fourier multipliers, H^T y, operator norms, step sizes), the per-pass
// kernel sequence of Algorithm 1 captured once in a CUDA graph, the FP64
// objective, state save / restore and per-stage timing.
#include "muffin.h"
#include "internal.h"

#include <cmath>
#include <cstdlib>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

using namespace muffin;

namespace {

thread_local std::string g_init_error;
constexpr int kNumStages = 7;
constexpr int kSideStreams = 4;    // graph branches of one pass: up to 3 group branches and the spectral step
const char* kStageNames[kNumStages] = {"iuwt_fine_adjoint", "fft_rows_fwd", "fft_cols_filter", "fft_rows_inv_primal",
                                       "iuwt_fine_analysis", "iuwt_coarse", "spectral_dct"};

bool is_pow2(int v) { return v > 0 && (v & (v - 1)) == 0; }

// Split j1 (levels below it run on halo tiles, the others on class
// sub-images).  Measured on GB300: the largest split whose coarse sub-image
// fits one block within 110 KB wins (fewer barriers, no cluster exchange);
// failing that, the smallest split that fits a cluster, then the streaming
// kernel.  -1 if nothing fits.
int auto_j1(int n, int J, int gen) {
  if (J == 0) return 0;
  const int top = J < 3 ? J : 3;
  for (int j1 = top; j1 >= 0; --j1) {
    if (j1 > 0 && n < 64) continue;
    if (J > j1 && coarse_cl_smem_bytes(n, J, gen, j1, 1) <= 110 * 1024) return j1;
  }
  for (size_t budget : {(size_t)110 * 1024, (size_t)220 * 1024}) {
    for (int j1 = 0; j1 <= top; ++j1) {
      if (j1 > 0 && n < 64) break;
      if (J == j1 || coarse_cluster_size(n, J, gen, j1, budget) > 0) return j1;
    }
  }
  for (int j1 = 0; j1 <= top; ++j1) {
    if (j1 > 0 && n < 64) break;
    if (J == j1 || coarse_stream_smem_bytes(n, gen, j1) <= 200 * 1024) return j1;
  }
  return -1;
}

bool split_fits(int n, int J, int gen, int j1) {
  if (J == j1) return true;
  return coarse_cluster_size(n, J, gen, j1, 220 * 1024) > 0 || coarse_stream_smem_bytes(n, gen, j1) <= 220 * 1024;
}

int check(const muffin_params* p, std::string* why) {
  auto fail = [&](const char* m) { if (why) *why = m; return (int)MUFFIN_ERR_ARG; };
  if (!p) return fail("params is NULL");
  if (p->nx != p->ny) return fail("nx != ny: only square images are supported");
  if (!is_pow2(p->nx) || p->nx < 16 || p->nx > 1024) return fail("N must be a power of two in [16, 1024]");
  if (p->nchan < 1 || p->nchan > 512) return fail("nchan must be in [1, 512]");
  if (p->nscales < 0 || (1 << p->nscales) >= p->nx) return fail("nscales J must satisfy 0 <= J and 2^J < N");
  if (p->iuwt_gen != 1 && p->iuwt_gen != 2) return fail("iuwt_gen must be 1 or 2");
  if (p->dictionary != 0 && p->dictionary != 1) return fail("dictionary must be 0 (IUWT) or 1 (union of bases)");
  if (p->dictionary == 1 && p->nscales < 1) return fail("the union of bases needs nscales J >= 1 levels");
  if (!(p->mu_s >= 0.0) || !std::isfinite(p->mu_s) || !(p->mu_l >= 0.0) || !std::isfinite(p->mu_l))
    return fail("mu_s and mu_l must be finite and >= 0");
  if (!std::isfinite(p->tau) || !std::isfinite(p->sigma) || !std::isfinite(p->rho)) return fail("non-finite step size");
  if (p->rho >= 2.0) return fail("rho must be < 2");
  if (p->h_chan_weight) {
    for (int l = 0; l < p->nchan; ++l)
      if (!(p->h_chan_weight[l] > 0.0) || !std::isfinite(p->h_chan_weight[l])) return fail("channel weights must be finite and > 0");
  }
  if (p->dictionary == 1) return MUFFIN_OK;   // no wavelet tiling to choose
  int j1 = p->fine_levels;
  if (j1 < 0) {
    j1 = auto_j1(p->nx, p->nscales, p->iuwt_gen);
    if (j1 < 0) return fail("no wavelet tiling fits shared memory");
  } else {
    const int top = p->nscales < 3 ? p->nscales : 3;
    if (j1 > top) return fail("fine_levels must be <= min(J, 3)");
    if (j1 > 0 && p->nx < 64) return fail("fine_levels > 0 needs N >= 64");
    if (!split_fits(p->nx, p->nscales, p->iuwt_gen, j1))
      return fail("fine_levels too small: coarse sub-image does not fit shared memory");
  }
  return MUFFIN_OK;
}

// Default pass plan: the whole cube as one group, one branch.
int default_group(const muffin_params*) { return 0; }
int default_branches(const muffin_params*) { return 1; }

struct Layout {
  size_t X, U, V, y, b, Kp, Kb, spec, S, T, D, cr, hhat, yhat, z64, pw, partials, scal;
  size_t W1, W2, W3;   // union of bases: [L][8][N][N] scratch each
  size_t twf, twd, twL, post, pre, invs, dense, w;
  size_t total;
  int max_parts;
  int j1;
};

Layout make_layout(const muffin_params* p) {
  Layout Lo{};
  const size_t n = p->nx, L = p->nchan, J = p->nscales, P = n * n;
  const bool uni = p->dictionary == 1;
  const size_t planes = uni ? (size_t)kDbBases : J + 1;
  Lo.j1 = uni ? 0 : (p->fine_levels >= 0 ? p->fine_levels : auto_j1(p->nx, p->nscales, p->iuwt_gen));
  size_t off = 0;
  auto take = [&](size_t bytes) { off = (off + 255) & ~(size_t)255; const size_t o = off; off += bytes; return o; };
  Lo.X = take(L * P * 4);
  Lo.U = take(L * planes * P * 4);
  Lo.V = take(L * P * 4);
  Lo.y = take(L * P * 4);
  Lo.b = take(L * P * 4);
  Lo.Kp = take(L * n * (n / 2) * 4);
  Lo.Kb = take(L * n * 4);
  Lo.spec = take(L * P * 4);
  Lo.S = take(L * P * 4);
  Lo.T = take(L * P * 4);
  Lo.D = take(L * P * 4);
  Lo.cr = take(L * P * 4);
  Lo.hhat = take(L * P * 16);
  Lo.yhat = take(L * P * 16);
  Lo.z64 = take(L * P * 16);
  Lo.pw = take((uni ? 2 + 3 * (size_t)kDbBases : J + 4) * P * 4);
  Lo.W1 = take(uni ? L * kDbBases * P * 4 : 0);
  Lo.W2 = take(uni ? L * kDbBases * P * 4 : 0);
  Lo.W3 = take(uni ? L * kDbBases * P * 4 : 0);
  size_t mp = 1024;
  mp = std::max(mp, (n / 64) * (n / 64) * L);
  mp = std::max(mp, (size_t)64 * 8 * L);   // coarse blocks for any split j1 <= 3 and cluster <= 8
  mp = std::max(mp, (P + 31) / 32);
  mp = std::max(mp, (n / 4) * L);
  mp = std::max(mp, (size_t)4096);
  Lo.max_parts = (int)mp;
  Lo.partials = take(mp * 8);
  Lo.scal = take(64 * 8);
  Lo.twf = take(n * 8);
  Lo.twd = take(n * 16);
  Lo.twL = take(L * 8);
  Lo.post = take(L * 8);
  Lo.pre = take(L * 8);
  Lo.invs = take(L * 4);
  Lo.dense = take(L * L * 4);
  Lo.w = take(L * 8);
  Lo.total = (off + 255) & ~(size_t)255;
  return Lo;
}

}  // namespace

struct muffin_ctx {
  muffin_params p;
  Geom g;
  Layout lo;
  cudaStream_t stream = nullptr;
  cudaStream_t cap = nullptr;
  char* ws = nullptr;
  std::vector<double> w;
  int state = 0;          // 0 initialised, 1 PSF set
  long long iter = 0;
  double mu_s, mu_l, tau, sigma, rho;
  double beta = 0, beta_closed = 0, ws_norm2 = 1, l_norm2 = 0;
  bool tau_auto = true;
  bool split_auto = false;   // choose the wavelet split by timing at the first set_psf
  bool tuned = false;
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  unsigned version = 0;    // bumped whenever the pass changes (step sizes, weights, tiling)
  std::string err;
  // pass plan: channels per group (the FFT and wavelet kernels of one group run
  // back to back, so that its row spectra and c_j1 / r_j1 stay in L2) and the
  // number of graph branches the groups alternate between
  int group = 0, branches = 1;
  cudaStream_t side[kSideStreams] = {};
  std::vector<cudaEvent_t> ev;     // fork, per-group "D written", per-branch join

  template <typename T> T* at(size_t off) const { return reinterpret_cast<T*>(ws + off); }
  float* X() const { return at<float>(lo.X); }
  float* U() const { return at<float>(lo.U); }
  float* V() const { return at<float>(lo.V); }
  size_t P() const { return (size_t)g.n * g.n; }
  size_t vox() const { return (size_t)g.L * P(); }
  double* partials() const { return at<double>(lo.partials); }
  double* scal() const { return at<double>(lo.scal); }
  // W_s^T U as the primal step reads it
  const float* S_ptr() const { return (g.J == 0 && g.dict == 0) ? U() : at<float>(lo.S); }
  size_t planes() const { return g.dict ? (size_t)kDbBases : (size_t)g.J + 1; }
  DwtArgs dwt(const float* src) const {
    DwtArgs d{};
    d.src = src;
    d.U = U();
    d.W1 = at<float>(lo.W1);
    d.W2 = at<float>(lo.W2);
    d.S = at<float>(lo.S);
    d.k = (float)(sigma * mu_s);
    d.rho = (float)rho;
    return d;
  }
};

#define CK(call)                                                                       \
  do {                                                                                 \
    cudaError_t e_ = (call);                                                           \
    if (e_ != cudaSuccess) return fail(ctx, MUFFIN_ERR_CUDA, #call, cudaGetErrorString(e_)); \
  } while (0)

static int fail(muffin_ctx* ctx, int code, const char* what, const char* detail = nullptr) {
  std::string m = what;
  if (detail) { m += ": "; m += detail; }
  if (ctx) ctx->err = m; else g_init_error = m;
  return code;
}

static void drop_graph(muffin_ctx* ctx) {
  if (ctx->exec) cudaGraphExecDestroy(ctx->exec);
  if (ctx->graph) cudaGraphDestroy(ctx->graph);
  ctx->exec = nullptr;
  ctx->graph = nullptr;
  ++ctx->version;
}

static void compute_steps(muffin_ctx* ctx) {
  ctx->l_norm2 = ctx->mu_s * ctx->mu_s * ctx->ws_norm2 + ctx->mu_l * ctx->mu_l;
  if (ctx->tau_auto) ctx->tau = 0.99 / (0.5 * ctx->beta + ctx->sigma * ctx->l_norm2);
}

// ----------------------------------------------------------------- one pass of Algorithm 1
struct StageTimer {
  std::vector<cudaEvent_t>* ev;
  std::vector<int>* stage;
  cudaStream_t s;
  void mark(int k) {
    cudaEvent_t e;
    cudaEventCreate(&e);
    cudaEventRecord(e, s);
    ev->push_back(e);
    stage->push_back(k);
  }
};

// Channel groups and branches of one pass (see the context's plan).
static void pass_plan(const muffin_ctx* ctx, bool timed, int* G, int* ngroups, int* nb) {
  const Geom& g = ctx->g;
  // the union-of-bases kernels take the whole cube in one launch
  *G = (timed || g.dict || ctx->group <= 0 || ctx->group >= g.L) ? g.L : ctx->group;
  *ngroups = (g.L + *G - 1) / *G;
  int b = ctx->branches < 1 ? 1 : ctx->branches;
  if (b > kSideStreams - 1) b = kSideStreams - 1;
  if (b > *ngroups) b = *ngroups;
  *nb = timed ? 1 : b;
}

// One pass of Algorithm 1.  Per channel group: the gradient FFTs ending in the
// primal step (Eqs. 8, 10), the spatial analysis with the dual update (Eq. 11)
// and the spatial adjoint W_s^T U of the updated duals, which the next pass's
// primal step reads (Eq. 9).  The spectral step (Eqs. 13-14 and the next
// pass's T) needs every channel of a pixel: it waits for every group's D and
// runs on its own branch, beside the remaining wavelet kernels.  Timed passes
// (tm) run everything in order on s, one group.
static int enqueue_pass(muffin_ctx* ctx, cudaStream_t s, StageTimer* tm) {
  const Geom& g = ctx->g;
  const Layout& lo = ctx->lo;
  const bool spatial = ctx->mu_s != 0.0, spectral = ctx->mu_l != 0.0;
  const size_t P = ctx->P();
  int G, ngroups, nb;
  pass_plan(ctx, tm != nullptr, &G, &ngroups, &nb);
  const bool fork = !tm && (nb > 1 || spectral);
  auto mark = [&](int k) { if (tm) tm->mark(k); };
  mark(-1);
  // events: [0] fork, [1 .. ngroups] D of group written, then one join per branch
  const size_t nev = 1 + (size_t)ngroups + kSideStreams;
  while (ctx->ev.size() < nev) {
    cudaEvent_t e;
    CK(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
    ctx->ev.push_back(e);
  }
  cudaStream_t br[kSideStreams];
  br[0] = s;
  for (int b = 1; b < nb; ++b) br[b] = ctx->side[b - 1];
  if (fork) {
    CK(cudaEventRecord(ctx->ev[0], s));
    for (int b = 1; b < nb; ++b) CK(cudaStreamWaitEvent(br[b], ctx->ev[0], 0));
  }
  const float k_s = (float)(ctx->sigma * ctx->mu_s), rho = (float)ctx->rho;
  for (int gi = 0; gi < ngroups; ++gi) {
    const int b = gi % nb;
    cudaStream_t st = br[b];
    const int l0 = gi * G, Lg = G < g.L - l0 ? G : g.L - l0;
    Geom gg = g;
    gg.L = Lg;
    const size_t o = (size_t)l0 * P;
    float* spec = ctx->at<float>(lo.spec) + (size_t)b * G * P;
    float* cr = ctx->at<float>(lo.cr) + (size_t)b * G * P;
    CK(launch_rows_fwd(ctx->X() + o, spec, g.n, Lg, ctx->at<float>(lo.twf), st));
    mark(1);
    CK(launch_cols_filter(spec, ctx->at<float>(lo.Kp) + (size_t)l0 * g.n * (g.n / 2),
                          ctx->at<float>(lo.Kb) + (size_t)l0 * g.n, g.n, Lg, ctx->at<float>(lo.twf), st));
    mark(2);
    PrimalArgs pa{};
    pa.b = ctx->at<float>(lo.b) + o;
    pa.S = spatial ? ((g.J == 0 && g.dict == 0) ? ctx->U() + o : ctx->at<float>(lo.S) + o) : nullptr;
    pa.T = spectral ? ctx->at<float>(lo.T) + o : nullptr;
    pa.X = ctx->X() + o;
    pa.D = ctx->at<float>(lo.D) + o;
    pa.tau = (float)ctx->tau;
    pa.mu_s = (float)ctx->mu_s;
    pa.mu_l = (float)ctx->mu_l;
    pa.rho = rho;
    CK(launch_rows_inv_primal(spec, pa, g.n, Lg, ctx->at<float>(lo.twf), st));
    mark(3);
    if (fork && spectral) CK(cudaEventRecord(ctx->ev[1 + gi], st));
    if (!spatial) continue;
    if (g.dict) {
      DwtArgs da = ctx->dwt(ctx->at<float>(lo.D));
      CK(launch_dwt_analysis(g, da, MODE_UPDATE, st));
      mark(4);
      CK(launch_dwt_adjoint(g, ctx->dwt(nullptr), st));
      mark(0);
      continue;
    }
    IuwtArgs ia{};
    ia.D = ctx->at<float>(lo.D) + o;
    ia.U = ctx->U() + o * ctx->planes();
    ia.cr = cr;
    ia.rin = cr;
    ia.S = ctx->at<float>(lo.S) + o;
    ia.k = k_s;
    ia.rho = rho;
    if (g.j1 > 0 || g.J == 0) {
      CK(launch_fine_analysis(gg, ia, MODE_UPDATE, st, nullptr));
      mark(4);
    }
    if (g.J > g.j1) {
      CK(launch_coarse(gg, g.j1 > 0 ? cr : ia.D, g.j1 > 0 ? cr : ia.S, ia.U, k_s, rho, MODE_UPDATE, nullptr, st,
                       nullptr));
      mark(5);
    }
    if (g.J > 0 && g.j1 > 0) {
      CK(launch_fine_adjoint(gg, ia, st));
      mark(0);
    }
  }
  if (spectral) {
    cudaStream_t sp = s;
    if (fork) {
      sp = ctx->side[kSideStreams - 1];
      for (int gi = 0; gi < ngroups; ++gi) CK(cudaStreamWaitEvent(sp, ctx->ev[1 + gi], 0));
    }
    SpecArgs sa{};
    sa.D = ctx->at<float>(lo.D);
    sa.V = ctx->V();
    sa.T = ctx->at<float>(lo.T);
    sa.k = (float)(ctx->sigma * ctx->mu_l);
    sa.rho = rho;
    sa.tw = ctx->at<float>(lo.twL);
    sa.post = ctx->at<float>(lo.post);
    sa.pre = ctx->at<float>(lo.pre);
    sa.invs = ctx->at<float>(lo.invs);
    sa.dense = ctx->at<float>(lo.dense);
    CK(launch_spectral(sa, (int)P, g.L, SPEC_UPDATE, sp, nullptr));
    mark(6);
    if (fork) {
      CK(cudaEventRecord(ctx->ev[1 + ngroups], sp));
      CK(cudaStreamWaitEvent(s, ctx->ev[1 + ngroups], 0));
    }
  }
  if (fork) {
    for (int b = 1; b < nb; ++b) {
      CK(cudaEventRecord(ctx->ev[2 + ngroups + b], br[b]));
      CK(cudaStreamWaitEvent(s, ctx->ev[2 + ngroups + b], 0));
    }
  }
  return MUFFIN_OK;
}

// T = W_lambda^T V and S = W_s^T U from the stored duals (after a state load).
static int refresh_adjoints(muffin_ctx* ctx) {
  const Geom& g = ctx->g;
  const Layout& lo = ctx->lo;
  SpecArgs sa{};
  sa.D = ctx->at<float>(lo.D);
  sa.V = ctx->V();
  sa.T = ctx->at<float>(lo.T);
  sa.tw = ctx->at<float>(lo.twL);
  sa.post = ctx->at<float>(lo.post);
  sa.pre = ctx->at<float>(lo.pre);
  sa.invs = ctx->at<float>(lo.invs);
  sa.dense = ctx->at<float>(lo.dense);
  sa.rho = 1.0f;
  CK(launch_spectral(sa, (int)ctx->P(), g.L, SPEC_TONLY, ctx->stream, nullptr));
  if (g.dict) {
    CK(launch_dwt_adjoint(g, ctx->dwt(nullptr), ctx->stream));
    return MUFFIN_OK;
  }
  if (g.J > g.j1) {
    float* rout = g.j1 > 0 ? ctx->at<float>(lo.cr) : ctx->at<float>(lo.S);
    CK(launch_coarse(g, nullptr, rout, ctx->U(), 0.f, 1.f, MODE_ADJ, nullptr, ctx->stream, nullptr));
  }
  if (g.J > 0 && g.j1 > 0) {
    IuwtArgs ia{};
    ia.U = ctx->U();
    ia.rin = ctx->at<float>(lo.cr);
    ia.S = ctx->at<float>(lo.S);
    CK(launch_fine_adjoint(g, ia, ctx->stream));
  }
  return MUFFIN_OK;
}

static void host_tables(const muffin_ctx* ctx, std::vector<char>& blob, const Layout& lo, size_t base) {
  const int n = ctx->g.n, L = ctx->g.L;
  auto put = [&](size_t off, const void* src, size_t bytes) { std::memcpy(blob.data() + (off - base), src, bytes); };
  const double pi = 3.14159265358979323846;
  std::vector<float> twf(2 * n);
  std::vector<double> twd(2 * n);
  for (int m = 0; m < n; ++m) {
    const double a = -2.0 * pi * m / n;
    twd[2 * m] = std::cos(a); twd[2 * m + 1] = std::sin(a);
    twf[2 * m] = (float)twd[2 * m]; twf[2 * m + 1] = (float)twd[2 * m + 1];
  }
  put(lo.twf, twf.data(), twf.size() * 4);
  put(lo.twd, twd.data(), twd.size() * 8);
  std::vector<float> twL(2 * L), post(2 * L), pre(2 * L), invs(L), dense((size_t)L * L);
  for (int k = 0; k < L; ++k) {
    const double a = -2.0 * pi * k / L;
    twL[2 * k] = (float)std::cos(a); twL[2 * k + 1] = (float)std::sin(a);
    const double sk = k == 0 ? std::sqrt(1.0 / L) : std::sqrt(2.0 / L);
    const double b = pi * k / (2.0 * L);
    post[2 * k] = (float)(sk * std::cos(-b)); post[2 * k + 1] = (float)(sk * std::sin(-b));
    pre[2 * k] = (float)std::cos(b); pre[2 * k + 1] = (float)std::sin(b);
    invs[k] = (float)(1.0 / (sk * L));
    for (int l = 0; l < L; ++l) dense[(size_t)k * L + l] = (float)(sk * std::cos(pi * (2 * l + 1) * k / (2.0 * L)));
  }
  put(lo.twL, twL.data(), twL.size() * 4);
  put(lo.post, post.data(), post.size() * 4);
  put(lo.pre, pre.data(), pre.size() * 4);
  put(lo.invs, invs.data(), invs.size() * 4);
  put(lo.dense, dense.data(), dense.size() * 4);
  put(lo.w, ctx->w.data(), ctx->w.size() * 8);
}

// Time one spatial half-pass (fine adjoint, fine analysis, coarse levels) of
// the split in g on the context's buffers; milliseconds per pass.
static int time_split(muffin_ctx* ctx, const Geom& g, float* ms) {
  const Layout& lo = ctx->lo;
  cudaStream_t s = ctx->stream;
  IuwtArgs ia{};
  ia.D = ctx->at<float>(lo.D);
  ia.U = ctx->U();
  ia.cr = ctx->at<float>(lo.cr);
  ia.rin = ctx->at<float>(lo.cr);
  ia.S = ctx->at<float>(lo.S);
  ia.k = 0.25f;
  ia.rho = 1.0f;
  cudaEvent_t e0, e1;
  CK(cudaEventCreate(&e0));
  CK(cudaEventCreate(&e1));
  const int reps = 3;
  for (int it = 0; it < reps + 1; ++it) {
    if (it == 1) CK(cudaEventRecord(e0, s));
    if (g.j1 > 0) CK(launch_fine_adjoint(g, ia, s));
    if (g.j1 > 0 || g.J == 0) CK(launch_fine_analysis(g, ia, MODE_UPDATE, s, nullptr));
    if (g.J > g.j1)
      CK(launch_coarse(g, g.j1 > 0 ? ia.cr : ia.D, g.j1 > 0 ? ia.cr : ia.S, ia.U, ia.k, ia.rho, MODE_UPDATE, nullptr, s,
                       nullptr));
  }
  CK(cudaEventRecord(e1, s));
  CK(cudaEventSynchronize(e1));
  CK(cudaEventElapsedTime(ms, e0, e1));
  *ms /= reps;
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  return MUFFIN_OK;
}

// Pick the fastest wavelet split for this cube by timing every valid one.  The
// dual state is still zero at the first set_psf, so the class-permuted layout
// of U may change; the planes the trials touch are cleared afterwards.
static int autotune_split(muffin_ctx* ctx) {
  const Geom base = ctx->g;
  const int top = base.J < 3 ? base.J : 3;
  float best = 0.0f;
  Geom best_g = base;
  bool any = false;
  for (int j1 = 0; j1 <= top; ++j1) {
    if (j1 > 0 && base.n < 64) continue;
    if (!split_fits(base.n, base.J, base.gen, j1)) continue;
    Geom g = base;
    g.j1 = j1;
    if (iuwt_configure(g) != cudaSuccess) { cudaGetLastError(); continue; }
    float ms = 0.0f;
    const int r = time_split(ctx, g, &ms);
    if (r != MUFFIN_OK) return r;
    if (!any || ms < best) { best = ms; best_g = g; any = true; }
  }
  // then the block shapes of the vectorised kernels for that split: 256 or 512 threads
  // (different work runs per thread), fine and coarse kernels each
  if (any && best_g.vec && getenv("MUFFIN_FINE_THREADS") == nullptr && getenv("MUFFIN_COARSE_THREADS") == nullptr) {
    for (int fnt : {256, 512}) {
      for (int cnt : {256, 512}) {
        if (fnt == best_g.fnt && cnt == best_g.cnt) continue;
        Geom g = best_g;
        g.fnt = fnt;
        g.cnt = cnt;
        float ms = 0.0f;
        const int r = time_split(ctx, g, &ms);
        if (r != MUFFIN_OK) return r;
        if (ms < best) { best = ms; best_g = g; }
      }
    }
  }
  if (any) ctx->g = best_g;
  cudaError_t e = iuwt_configure(ctx->g);
  if (e != cudaSuccess) return fail(ctx, MUFFIN_ERR_CUDA, "wavelet configuration", cudaGetErrorString(e));
  const Layout& lo = ctx->lo;
  CK(cudaMemsetAsync(ctx->U(), 0, (size_t)ctx->vox() * ctx->planes() * 4, ctx->stream));
  CK(cudaMemsetAsync(ctx->at<float>(lo.S), 0, ctx->vox() * 4, ctx->stream));
  CK(cudaMemsetAsync(ctx->at<float>(lo.cr), 0, ctx->vox() * 4, ctx->stream));
  return MUFFIN_OK;
}

// ----------------------------------------------------------------- C ABI
extern "C" {

size_t muffin_workspace_bytes(const muffin_params* p) {
  if (check(p, nullptr) != MUFFIN_OK) return 0;
  return make_layout(p).total;
}

int muffin_check_params(const muffin_params* p, char* h_msg, size_t msg_len) {
  std::string why;
  const int r = check(p, &why);
  if (h_msg && msg_len) {
    std::snprintf(h_msg, msg_len, "%s", r == MUFFIN_OK ? "ok" : why.c_str());
  }
  return r;
}

int muffin_init(muffin_ctx** out, const muffin_params* p, const float* d_dirty, void* d_workspace, size_t ws_bytes,
                cudaStream_t stream) {
  muffin_ctx* ctx = nullptr;
  if (!out) return fail(nullptr, MUFFIN_ERR_ARG, "ctx out-pointer is NULL");
  *out = nullptr;
  std::string why;
  if (check(p, &why) != MUFFIN_OK) return fail(nullptr, MUFFIN_ERR_ARG, why.c_str());
  if (!d_dirty || !d_workspace) return fail(nullptr, MUFFIN_ERR_ARG, "NULL dirty cube or workspace");
  if (((uintptr_t)d_workspace & 255) != 0) return fail(nullptr, MUFFIN_ERR_ARG, "workspace must be 256-byte aligned");
  const Layout lo = make_layout(p);
  if (ws_bytes < lo.total) return fail(nullptr, MUFFIN_ERR_NOMEM, "workspace smaller than muffin_workspace_bytes()");
  ctx = new muffin_ctx();
  ctx->p = *p;
  ctx->p.h_chan_weight = nullptr;
  ctx->lo = lo;
  ctx->g = Geom{p->nx, p->nchan, p->nscales, p->iuwt_gen, lo.j1, 0, p->dictionary};
  ctx->stream = stream;
  ctx->ws = reinterpret_cast<char*>(d_workspace);
  ctx->w.assign(p->nchan, 1.0);
  if (p->h_chan_weight) for (int l = 0; l < p->nchan; ++l) ctx->w[l] = p->h_chan_weight[l];
  ctx->mu_s = p->mu_s;
  ctx->mu_l = p->mu_l;
  ctx->sigma = p->sigma > 0 ? p->sigma : 1.0;
  ctx->rho = p->rho > 0 ? p->rho : 1.0;
  ctx->tau_auto = !(p->tau > 0);
  ctx->split_auto = p->dictionary == 0 && p->fine_levels < 0 && p->nscales > 0 &&
                    getenv("MUFFIN_NO_AUTOTUNE") == nullptr;
  ctx->tau = p->tau > 0 ? p->tau : 0.0;
  if (ctx->p.power_iters <= 0) ctx->p.power_iters = 40;
  auto bail = [&](int code) {
    if (ctx->cap) cudaStreamDestroy(ctx->cap);
    for (cudaStream_t x : ctx->side) if (x) cudaStreamDestroy(x);
    g_init_error = ctx->err;
    delete ctx;
    return code;
  };
  cudaError_t e;
  if ((e = cudaStreamCreateWithFlags(&ctx->cap, cudaStreamNonBlocking))) { fail(ctx, MUFFIN_ERR_CUDA, "cudaStreamCreate", cudaGetErrorString(e)); return bail(MUFFIN_ERR_CUDA); }
  for (int b = 0; b < kSideStreams; ++b)
    if ((e = cudaStreamCreateWithFlags(&ctx->side[b], cudaStreamNonBlocking))) {
      fail(ctx, MUFFIN_ERR_CUDA, "cudaStreamCreate", cudaGetErrorString(e));
      return bail(MUFFIN_ERR_CUDA);
    }
  // pass plan (channels per group, graph branches); MUFFIN_GROUP / MUFFIN_BRANCHES override
  ctx->group = default_group(p);
  ctx->branches = default_branches(p);
  if (const char* v = getenv("MUFFIN_GROUP")) ctx->group = atoi(v);
  if (const char* v = getenv("MUFFIN_BRANCHES")) ctx->branches = atoi(v);
  if ((e = fft_configure(ctx->g.n)) || (ctx->g.dict == 0 && (e = iuwt_configure(ctx->g))) ||
      (ctx->g.dict == 1 && (e = dwt_configure())) || (e = spectral_configure(ctx->g.L))) {
    fail(ctx, MUFFIN_ERR_CUDA, "kernel configuration", cudaGetErrorString(e));
    return bail(MUFFIN_ERR_CUDA);
  }
  // zero everything (X = U = V = 0 and every derived buffer), then the dirty cube and the tables
  if ((e = cudaMemsetAsync(ctx->ws, 0, lo.total, stream))) { fail(ctx, MUFFIN_ERR_CUDA, "cudaMemsetAsync", cudaGetErrorString(e)); return bail(MUFFIN_ERR_CUDA); }
  if ((e = cudaMemcpyAsync(ctx->at<float>(lo.y), d_dirty, ctx->vox() * 4, cudaMemcpyDeviceToDevice, stream))) {
    fail(ctx, MUFFIN_ERR_CUDA, "copy of the dirty cube", cudaGetErrorString(e));
    return bail(MUFFIN_ERR_CUDA);
  }
  const size_t tbase = lo.twf, tend = lo.w + ctx->w.size() * 8;
  std::vector<char> blob(tend - tbase, 0);
  host_tables(ctx, blob, lo, tbase);
  if ((e = cudaMemcpyAsync(ctx->ws + tbase, blob.data(), blob.size(), cudaMemcpyHostToDevice, stream))) {
    fail(ctx, MUFFIN_ERR_CUDA, "table upload", cudaGetErrorString(e));
    return bail(MUFFIN_ERR_CUDA);
  }
  int* cnt = reinterpret_cast<int*>(ctx->scal() + 63);
  int h_cnt = 0;
  if ((e = launch_nonfinite_count(ctx->at<float>(lo.y), ctx->vox(), cnt, stream)) ||
      (e = cudaMemcpyAsync(&h_cnt, cnt, sizeof(int), cudaMemcpyDeviceToHost, stream)) || (e = cudaStreamSynchronize(stream))) {
    fail(ctx, MUFFIN_ERR_CUDA, "init", cudaGetErrorString(e));
    return bail(MUFFIN_ERR_CUDA);
  }
  if (h_cnt) { fail(ctx, MUFFIN_ERR_NONFINITE, "dirty cube holds NaN or Inf"); return bail(MUFFIN_ERR_NONFINITE); }
  *out = ctx;
  return MUFFIN_OK;
}

int muffin_set_psf(muffin_ctx* ctx, const float* d_psf) {
  if (!ctx) return fail(nullptr, MUFFIN_ERR_ARG, "ctx is NULL");
  if (!d_psf) return fail(ctx, MUFFIN_ERR_ARG, "psf is NULL");
  const Geom& g = ctx->g;
  const Layout& lo = ctx->lo;
  cudaStream_t s = ctx->stream;
  const int n = g.n, L = g.L;
  const size_t P = ctx->P(), V = ctx->vox();
  double* sc = ctx->scal();
  int* cnt = reinterpret_cast<int*>(sc + 63);
  int h_cnt = 0;
  CK(cudaMemsetAsync(cnt, 0, sizeof(int), s));
  CK(launch_nonfinite_count(d_psf, V, cnt, s));
  CK(cudaMemcpyAsync(&h_cnt, cnt, sizeof(int), cudaMemcpyDeviceToHost, s));
  CK(cudaStreamSynchronize(s));
  if (h_cnt) return fail(ctx, MUFFIN_ERR_NONFINITE, "psf holds NaN or Inf");
  if (ctx->split_auto && !ctx->tuned) {
    const int r = autotune_split(ctx);
    if (r != MUFFIN_OK) return r;
    ctx->tuned = true;
  }
  void* hh = ctx->ws + lo.hhat;
  void* yh = ctx->ws + lo.yhat;
  void* z = ctx->ws + lo.z64;
  const void* twd = ctx->ws + lo.twd;
  const double* w = ctx->at<double>(lo.w);
  // hhat_l = DFT of the PSF moved to the origin; yhat_l = DFT of y_l (FP64)
  CK(launch_c2c_rows64(d_psf, 1, hh, n, L, -1, twd, s));
  CK(launch_c2c_cols64(hh, n, L, -1, twd, s));
  CK(launch_c2c_rows64(ctx->at<float>(lo.y), 2, yh, n, L, -1, twd, s));
  CK(launch_c2c_cols64(yh, n, L, -1, twd, s));
  CK(launch_build_K(hh, w, ctx->at<float>(lo.Kp), ctx->at<float>(lo.Kb), n, L, s));
  // b_l = w_l H_l^T y_l = w_l IDFT(conj(hhat) yhat)
  CK(cudaMemcpyAsync(z, yh, V * 16, cudaMemcpyDeviceToDevice, s));
  CK(launch_mul_conj(hh, z, n, L, s));
  CK(launch_c2c_cols64(z, n, L, 1, twd, s));
  CK(launch_c2c_rows64(z, 0, z, n, L, 1, twd, s));
  CK(launch_real_to_float(z, w, ctx->at<float>(lo.b), n, L, s));
  int np = 0;
  CK(launch_max_abs2(hh, w, n, L, ctx->partials(), &np, s));
  CK(launch_max_partials(ctx->partials(), np, sc + 0, s));
  // beta: power method on the block-diagonal H^T H (K already holds w_l / N^2)
  float* pv = reinterpret_cast<float*>(z);
  float* pw = pv + V;
  float* spec = ctx->at<float>(lo.spec);
  const float* twf = ctx->at<float>(lo.twf);
  CK(launch_fill_random(pv, V, 0x5eedULL, s));
  CK(launch_dot(pv, pv, V, ctx->partials(), &np, s));
  CK(launch_sum_partials(ctx->partials(), np, sc + 1, s));
  CK(launch_scale(pv, V, nullptr, sc + 1, s));
  for (int it = 0; it < ctx->p.power_iters; ++it) {
    CK(launch_rows_fwd(pv, spec, n, L, twf, s));
    CK(launch_cols_filter(spec, ctx->at<float>(lo.Kp), ctx->at<float>(lo.Kb), n, L, twf, s));
    CK(launch_rows_inv_plain(spec, pw, n, L, twf, s));
    CK(launch_dot(pv, pw, V, ctx->partials(), &np, s));
    CK(launch_sum_partials(ctx->partials(), np, sc + 2, s));
    CK(launch_dot(pw, pw, V, ctx->partials(), &np, s));
    CK(launch_sum_partials(ctx->partials(), np, sc + 1, s));
    CK(launch_scale(pw, V, nullptr, sc + 1, s));
    std::swap(pv, pw);
  }
  // ||W_s||^2: power method on W_s^T W_s over one N x N plane
  if (g.dict) {
    Geom g1 = g;
    g1.L = 1;
    float* x = ctx->at<float>(lo.pw);
    DwtArgs da{};
    da.src = x;
    da.U = x + P;
    da.S = da.U + (size_t)kDbBases * P;
    da.W1 = da.S + P;
    da.W2 = da.W1 + (size_t)kDbBases * P;
    da.k = 1.f;
    da.rho = 1.f;
    float* St = da.S;
    CK(launch_fill_random(x, P, 0x5eed2ULL, s));
    CK(launch_dot(x, x, P, ctx->partials(), &np, s));
    CK(launch_sum_partials(ctx->partials(), np, sc + 4, s));
    CK(launch_scale(x, P, nullptr, sc + 4, s));
    for (int it = 0; it < ctx->p.power_iters; ++it) {
      CK(launch_dwt_analysis(g1, da, MODE_LINEAR, s));
      CK(launch_dwt_adjoint(g1, da, s));
      CK(launch_dot(x, St, P, ctx->partials(), &np, s));
      CK(launch_sum_partials(ctx->partials(), np, sc + 3, s));
      CK(launch_dot(St, St, P, ctx->partials(), &np, s));
      CK(launch_sum_partials(ctx->partials(), np, sc + 4, s));
      CK(cudaMemcpyAsync(x, St, P * 4, cudaMemcpyDeviceToDevice, s));
      CK(launch_scale(x, P, nullptr, sc + 4, s));
    }
  } else if (g.J > 0) {
    Geom g1 = g;
    g1.L = 1;
    float* x = ctx->at<float>(lo.pw);
    float* Ut = x + P;
    float* crt = Ut + (size_t)(g.J + 1) * P;
    float* St = crt + P;
    IuwtArgs ia{};
    ia.D = x; ia.U = Ut; ia.cr = crt; ia.rin = crt; ia.S = St; ia.k = 1.f; ia.rho = 1.f;
    CK(launch_fill_random(x, P, 0x5eed2ULL, s));
    CK(launch_dot(x, x, P, ctx->partials(), &np, s));
    CK(launch_sum_partials(ctx->partials(), np, sc + 4, s));
    CK(launch_scale(x, P, nullptr, sc + 4, s));
    for (int it = 0; it < ctx->p.power_iters; ++it) {
      if (g1.j1 > 0) CK(launch_fine_analysis(g1, ia, MODE_LINEAR, s, nullptr));
      if (g1.J > g1.j1)
        CK(launch_coarse(g1, g1.j1 > 0 ? crt : x, g1.j1 > 0 ? crt : St, Ut, 1.f, 1.f, MODE_LINEAR, nullptr, s, nullptr));
      if (g1.j1 > 0) CK(launch_fine_adjoint(g1, ia, s));
      CK(launch_dot(x, St, P, ctx->partials(), &np, s));
      CK(launch_sum_partials(ctx->partials(), np, sc + 3, s));
      CK(launch_dot(St, St, P, ctx->partials(), &np, s));
      CK(launch_sum_partials(ctx->partials(), np, sc + 4, s));
      CK(cudaMemcpyAsync(x, St, P * 4, cudaMemcpyDeviceToDevice, s));
      CK(launch_scale(x, P, nullptr, sc + 4, s));
    }
  }
  double h[4] = {0, 0, 0, 0};
  CK(cudaMemcpyAsync(h, sc, 4 * sizeof(double), cudaMemcpyDeviceToHost, s));
  CK(cudaStreamSynchronize(s));
  ctx->beta_closed = h[0];
  ctx->beta = 1.01 * h[2];
  ctx->ws_norm2 = g.J > 0 ? 1.01 * h[3] : 1.0;
  if (!std::isfinite(ctx->beta) || !(ctx->beta > 0)) return fail(ctx, MUFFIN_ERR_NONFINITE, "power method for beta failed");
  compute_steps(ctx);
  drop_graph(ctx);
  ctx->state = 1;
  return MUFFIN_OK;
}

int muffin_iterate(muffin_ctx* ctx, int n_iter) {
  if (!ctx) return fail(nullptr, MUFFIN_ERR_ARG, "ctx is NULL");
  if (n_iter < 0) return fail(ctx, MUFFIN_ERR_ARG, "n_iter < 0");
  if (ctx->state < 1) return fail(ctx, MUFFIN_ERR_STATE, "muffin_set_psf must come before muffin_iterate");
  if (n_iter == 0) return MUFFIN_OK;
  if (!ctx->exec) {
    CK(cudaStreamBeginCapture(ctx->cap, cudaStreamCaptureModeThreadLocal));
    const int r = enqueue_pass(ctx, ctx->cap, nullptr);
    cudaGraph_t gr = nullptr;
    const cudaError_t e = cudaStreamEndCapture(ctx->cap, &gr);
    if (r != MUFFIN_OK) { if (gr) cudaGraphDestroy(gr); return r; }
    if (e != cudaSuccess) return fail(ctx, MUFFIN_ERR_CUDA, "cudaStreamEndCapture", cudaGetErrorString(e));
    ctx->graph = gr;
    CK(cudaGraphInstantiate(&ctx->exec, ctx->graph, 0));
  }
  for (int i = 0; i < n_iter; ++i) CK(cudaGraphLaunch(ctx->exec, ctx->stream));
  ctx->iter += n_iter;
  return MUFFIN_OK;
}

int muffin_iterate_timed(muffin_ctx* ctx, int n_iter, double* h_ms, int n_stages) {
  if (!ctx) return fail(nullptr, MUFFIN_ERR_ARG, "ctx is NULL");
  if (ctx->state < 1) return fail(ctx, MUFFIN_ERR_STATE, "muffin_set_psf must come before muffin_iterate_timed");
  if (n_iter < 0 || (n_stages > 0 && !h_ms)) return fail(ctx, MUFFIN_ERR_ARG, "bad n_iter or h_ms");
  std::vector<cudaEvent_t> ev;
  std::vector<int> st;
  StageTimer tm{&ev, &st, ctx->stream};
  int r = MUFFIN_OK;
  for (int i = 0; i < n_iter && r == MUFFIN_OK; ++i) r = enqueue_pass(ctx, ctx->stream, &tm);
  cudaError_t e = cudaStreamSynchronize(ctx->stream);
  for (int k = 0; k < n_stages; ++k) h_ms[k] = 0.0;
  for (size_t i = 1; i < ev.size() && e == cudaSuccess; ++i) {
    if (st[i] < 0) continue;
    float ms = 0.f;
    e = cudaEventElapsedTime(&ms, ev[i - 1], ev[i]);
    if (st[i] < n_stages) h_ms[st[i]] += ms;
  }
  for (auto x : ev) cudaEventDestroy(x);
  if (r != MUFFIN_OK) return r;
  if (e != cudaSuccess) return fail(ctx, MUFFIN_ERR_CUDA, "timed iteration", cudaGetErrorString(e));
  ctx->iter += n_iter;
  return MUFFIN_OK;
}

int muffin_objective(muffin_ctx* ctx, double* h_obj, double* h_terms) {
  if (!ctx) return fail(nullptr, MUFFIN_ERR_ARG, "ctx is NULL");
  if (ctx->state < 1) return fail(ctx, MUFFIN_ERR_STATE, "muffin_set_psf must come before muffin_objective");
  if (!h_obj) return fail(ctx, MUFFIN_ERR_ARG, "h_obj is NULL");
  const Geom& g = ctx->g;
  const Layout& lo = ctx->lo;
  cudaStream_t s = ctx->stream;
  double* sc = ctx->scal();
  void* z = ctx->ws + lo.z64;
  int np = 0;
  CK(cudaMemsetAsync(sc + 10, 0, 4 * sizeof(double), s));
  CK(launch_c2c_rows64(ctx->X(), 2, z, g.n, g.L, -1, ctx->ws + lo.twd, s));
  CK(launch_cols64_fidelity(z, ctx->ws + lo.hhat, ctx->ws + lo.yhat, ctx->at<double>(lo.w), g.n, g.L,
                            ctx->ws + lo.twd, ctx->partials(), &np, s));
  CK(launch_sum_partials(ctx->partials(), np, sc + 10, s));
  IuwtArgs ia{};
  ia.D = ctx->X();
  ia.U = ctx->U();
  ia.cr = ctx->at<float>(lo.D);   // c_{j1} of X goes to scratch, not to the state
  ia.partials = ctx->partials();
  if (g.dict) {
    DwtArgs da = ctx->dwt(ctx->X());
    da.U = ctx->at<float>(lo.W3);      // W_s X into scratch, not into the state
    CK(launch_dwt_analysis(g, da, MODE_LINEAR, s));
    CK(launch_abs_sum(da.U, (size_t)kDbBases * ctx->vox(), ctx->partials(), &np, s));
    CK(launch_sum_partials(ctx->partials(), np, sc + 11, s));
  } else if (g.j1 > 0 || g.J == 0) {
    CK(launch_fine_analysis(g, ia, MODE_NORM, s, &np));
    CK(launch_sum_partials(ctx->partials(), np, sc + 11, s));
  }
  if (!g.dict && g.J > g.j1) {
    const float* cin = g.j1 > 0 ? ctx->at<float>(lo.D) : ctx->X();
    CK(launch_coarse(g, cin, nullptr, ctx->U(), 0.f, 1.f, MODE_NORM, ctx->partials(), s, &np));
    CK(launch_sum_partials(ctx->partials(), np, sc + 12, s));
  }
  SpecArgs sa{};
  sa.D = ctx->X();
  sa.tw = ctx->at<float>(lo.twL);
  sa.post = ctx->at<float>(lo.post);
  sa.pre = ctx->at<float>(lo.pre);
  sa.invs = ctx->at<float>(lo.invs);
  sa.dense = ctx->at<float>(lo.dense);
  sa.partials = ctx->partials();
  CK(launch_spectral(sa, (int)ctx->P(), g.L, SPEC_NORM, s, &np));
  CK(launch_sum_partials(ctx->partials(), np, sc + 13, s));
  double h[4];
  CK(cudaMemcpyAsync(h, sc + 10, sizeof(h), cudaMemcpyDeviceToHost, s));
  CK(cudaStreamSynchronize(s));
  // a block of the pipelined spectral kernel that gave up a bounded wait left its tiles unwritten
  const int to = spectral_take_timeouts(), tf = fft_take_timeouts();
  if (to < 0 || tf < 0) return fail(ctx, MUFFIN_ERR_CUDA, "reading the pipelined kernels' wait status");
  if (to > 0 || tf > 0)
    return fail(ctx, MUFFIN_ERR_TIMEOUT, "a block of a pipelined (TMA) kernel gave up a bounded wait; the state is incomplete");
  const double data = h[0], sp = ctx->mu_s * (h[1] + h[2]), sl = ctx->mu_l * h[3];
  *h_obj = data + sp + sl;
  if (h_terms) { h_terms[0] = data; h_terms[1] = sp; h_terms[2] = sl; }
  if (!std::isfinite(*h_obj)) return fail(ctx, MUFFIN_ERR_NONFINITE, "objective is not finite");
  return MUFFIN_OK;
}

int muffin_get_cube(muffin_ctx* ctx, float* d_x) {
  if (!ctx || !d_x) return fail(ctx, MUFFIN_ERR_ARG, "NULL argument");
  CK(cudaMemcpyAsync(d_x, ctx->X(), ctx->vox() * 4, cudaMemcpyDeviceToDevice, ctx->stream));
  return MUFFIN_OK;
}

int muffin_set_cube(muffin_ctx* ctx, const float* d_x) {
  if (!ctx || !d_x) return fail(ctx, MUFFIN_ERR_ARG, "NULL argument");
  CK(cudaMemcpyAsync(ctx->X(), d_x, ctx->vox() * 4, cudaMemcpyDeviceToDevice, ctx->stream));
  return MUFFIN_OK;
}

int muffin_get_state(muffin_ctx* ctx, float* d_x, float* d_u, float* d_v, long long* h_iter) {
  if (!ctx || !d_x || !d_u || !d_v) return fail(ctx, MUFFIN_ERR_ARG, "NULL argument");
  const Geom& g = ctx->g;
  CK(cudaMemcpyAsync(d_x, ctx->X(), ctx->vox() * 4, cudaMemcpyDeviceToDevice, ctx->stream));
  if (g.dict) CK(cudaMemcpyAsync(d_u, ctx->U(), ctx->vox() * kDbBases * 4, cudaMemcpyDeviceToDevice, ctx->stream));
  else CK(launch_permute_planes(ctx->U(), d_u, g.n, g.L, g.J, g.j1, 0, ctx->stream));
  CK(cudaMemcpyAsync(d_v, ctx->V(), ctx->vox() * 4, cudaMemcpyDeviceToDevice, ctx->stream));
  if (h_iter) *h_iter = ctx->iter;
  return MUFFIN_OK;
}

int muffin_set_state(muffin_ctx* ctx, const float* d_x, const float* d_u, const float* d_v, long long iter) {
  if (!ctx || !d_x || !d_u || !d_v) return fail(ctx, MUFFIN_ERR_ARG, "NULL argument");
  if (ctx->state < 1) return fail(ctx, MUFFIN_ERR_STATE, "muffin_set_psf must come before muffin_set_state");
  const Geom& g = ctx->g;
  CK(cudaMemcpyAsync(ctx->X(), d_x, ctx->vox() * 4, cudaMemcpyDeviceToDevice, ctx->stream));
  if (g.dict) CK(cudaMemcpyAsync(ctx->U(), d_u, ctx->vox() * kDbBases * 4, cudaMemcpyDeviceToDevice, ctx->stream));
  else CK(launch_permute_planes(d_u, ctx->U(), g.n, g.L, g.J, g.j1, 1, ctx->stream));
  CK(cudaMemcpyAsync(ctx->V(), d_v, ctx->vox() * 4, cudaMemcpyDeviceToDevice, ctx->stream));
  const int r = refresh_adjoints(ctx);
  if (r != MUFFIN_OK) return r;
  ctx->iter = iter;
  return MUFFIN_OK;
}

int muffin_set_mu(muffin_ctx* ctx, double mu_s, double mu_l) {
  if (!ctx) return fail(nullptr, MUFFIN_ERR_ARG, "ctx is NULL");
  if (!(mu_s >= 0) || !(mu_l >= 0) || !std::isfinite(mu_s) || !std::isfinite(mu_l))
    return fail(ctx, MUFFIN_ERR_ARG, "mu_s and mu_l must be finite and >= 0");
  ctx->mu_s = mu_s;
  ctx->mu_l = mu_l;
  if (ctx->state >= 1) compute_steps(ctx);
  drop_graph(ctx);
  return MUFFIN_OK;
}

int muffin_step_sizes(const muffin_ctx* ctx, double* tau, double* sigma, double* rho, double* beta, double* l_norm2,
                      double* beta_closed, double* ws_norm2) {
  if (!ctx) return MUFFIN_ERR_ARG;
  if (ctx->state < 1) return MUFFIN_ERR_STATE;
  if (tau) *tau = ctx->tau;
  if (sigma) *sigma = ctx->sigma;
  if (rho) *rho = ctx->rho;
  if (beta) *beta = ctx->beta;
  if (l_norm2) *l_norm2 = ctx->l_norm2;
  if (beta_closed) *beta_closed = ctx->beta_closed;
  if (ws_norm2) *ws_norm2 = ctx->ws_norm2;
  return MUFFIN_OK;
}

int muffin_num_stages(void) { return kNumStages; }

const char* muffin_stage_name(int k) { return (k >= 0 && k < kNumStages) ? kStageNames[k] : ""; }

double muffin_stage_bytes(const muffin_ctx* ctx, int k) {
  if (!ctx) return 0.0;
  const Geom& g = ctx->g;
  const double V = (double)ctx->vox();
  const bool sp = ctx->mu_s != 0.0, sl = ctx->mu_l != 0.0;
  if (g.dict) {
    // union of bases: the adjoint reads the eight planes of U and writes
    // W_s^T U once; the analysis reads D and reads and writes U
    switch (k) {
      case 0: return sp ? V * (4.0 * kDbBases + 4.0) : 0.0;
      case 4: return sp ? V * (4.0 + 8.0 * kDbBases) : 0.0;
      case 5: return 0.0;
    }
  }
  switch (k) {
    case 0: return (sp && g.J > 0 && g.j1 > 0) ? 4.0 * V * (g.j1 + 2) : 0.0;
    case 1: return 8.0 * V;
    case 2: return 8.0 * V + 4.0 * (double)g.L * g.n * (g.n / 2 + 1);
    case 3: return V * (4 + 4 + (sp ? 4 : 0) + (sl ? 4 : 0) + 8 + 4);
    case 4:
      if (!sp || !(g.j1 > 0 || g.J == 0)) return 0.0;
      return V * (4.0 + 8.0 * g.j1 + (g.J == g.j1 ? 8.0 : 4.0));
    case 5: return (sp && g.J > g.j1) ? V * (4.0 + 8.0 * (g.J - g.j1 + 1) + 4.0) : 0.0;
    case 6: return sl ? 16.0 * V : 0.0;
  }
  return 0.0;
}

int muffin_kernels_per_iteration(const muffin_ctx* ctx) {
  if (!ctx) return 0;
  int G, ngroups, nb;
  pass_plan(ctx, false, &G, &ngroups, &nb);
  int per_group = 0;
  for (int k = 0; k < kNumStages; ++k) per_group += (k != 6 && muffin_stage_bytes(ctx, k) > 0) ? 1 : 0;
  int n = ngroups * per_group + (muffin_stage_bytes(ctx, 6) > 0 ? 1 : 0);
  if (ctx->g.dict && ctx->mu_s != 0.0) n += 3 * ctx->g.J - 2;   // 2J adjoint and J analysis kernels, not 2
  return n;
}

int muffin_set_plan(muffin_ctx* ctx, int channels_per_group, int branches) {
  if (!ctx) return fail(nullptr, MUFFIN_ERR_ARG, "ctx is NULL");
  if (channels_per_group < 0 || branches < 1 || branches > kSideStreams - 1)
    return fail(ctx, MUFFIN_ERR_ARG, "channels_per_group must be >= 0 and branches in [1, 3]");
  ctx->group = channels_per_group;
  ctx->branches = branches;
  drop_graph(ctx);
  return MUFFIN_OK;
}

int muffin_plan(const muffin_ctx* ctx, int* channels_per_group, int* branches) {
  if (!ctx) return MUFFIN_ERR_ARG;
  int G, ngroups, nb;
  pass_plan(ctx, false, &G, &ngroups, &nb);
  if (channels_per_group) *channels_per_group = G;
  if (branches) *branches = nb;
  return MUFFIN_OK;
}

int muffin_block_threads(const muffin_ctx* ctx, int* fine_threads, int* coarse_threads) {
  if (!ctx) return MUFFIN_ERR_ARG;
  if (fine_threads) *fine_threads = ctx->g.fnt;
  if (coarse_threads) *coarse_threads = ctx->g.cnt;
  return MUFFIN_OK;
}

int muffin_tiling(const muffin_ctx* ctx, int* fine_levels, int* cluster) {
  if (!ctx) return MUFFIN_ERR_ARG;
  if (fine_levels) *fine_levels = ctx->g.j1;
  if (cluster) *cluster = ctx->g.cs;
  return MUFFIN_OK;
}

const char* muffin_last_error(const muffin_ctx* ctx) { return ctx ? ctx->err.c_str() : g_init_error.c_str(); }

void muffin_destroy(muffin_ctx* ctx) {
  if (!ctx) return;
  drop_graph(ctx);
  if (ctx->cap) cudaStreamDestroy(ctx->cap);
  for (cudaStream_t x : ctx->side) if (x) cudaStreamDestroy(x);
  for (cudaEvent_t e : ctx->ev) cudaEventDestroy(e);
  delete ctx;
}

}  // extern "C"

// ----------------------------------------------------------------- batches of cubes
struct muffin_batch {
  std::vector<muffin_ctx*> ctx;
  std::vector<unsigned> version;
  std::vector<cudaStream_t> side;
  std::vector<cudaEvent_t> done;
  cudaStream_t stream = nullptr, cap = nullptr;
  cudaEvent_t fork = nullptr;
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  int mode = 0;                 // 0: graph branches, 1: one persistent launch per pass
  long long polls = 1LL << 22;  // bound of the persistent kernel's barrier waits
  std::string err;
};

static int bfail(muffin_batch* b, int code, const char* what, const char* detail = nullptr);

// Arguments of one cube for the persistent batch kernel (the pass of enqueue_pass, whole cube).
static void batch_cube_of(const muffin_ctx* ctx, BatchCube* c) {
  const Geom& g = ctx->g;
  const Layout& lo = ctx->lo;
  const bool spatial = ctx->mu_s != 0.0, spectral = ctx->mu_l != 0.0;
  *c = BatchCube{};
  c->n = g.n; c->L = g.L; c->J = g.J; c->j1 = g.j1;
  c->spatial = spatial ? 1 : 0;
  c->spectral = spectral ? 1 : 0;
  c->spec = ctx->at<float>(lo.spec);
  c->Kp = ctx->at<float>(lo.Kp);
  c->Kb = ctx->at<float>(lo.Kb);
  c->twf = ctx->at<float>(lo.twf);
  PrimalArgs& pa = c->pa;
  pa.b = ctx->at<float>(lo.b);
  pa.S = spatial ? ctx->at<float>(lo.S) : nullptr;
  pa.T = spectral ? ctx->at<float>(lo.T) : nullptr;
  pa.X = ctx->X();
  pa.D = ctx->at<float>(lo.D);
  pa.tau = (float)ctx->tau;
  pa.mu_s = (float)ctx->mu_s;
  pa.mu_l = (float)ctx->mu_l;
  pa.rho = (float)ctx->rho;
  IuwtArgs& ia = c->ia;
  ia.D = ctx->at<float>(lo.D);
  ia.U = ctx->U();
  ia.cr = ctx->at<float>(lo.cr);
  ia.rin = ctx->at<float>(lo.cr);
  ia.S = ctx->at<float>(lo.S);
  ia.k = (float)(ctx->sigma * ctx->mu_s);
  ia.rho = (float)ctx->rho;
  SpecArgs& sa = c->sa;
  sa.D = ctx->at<float>(lo.D);
  sa.V = ctx->V();
  sa.T = ctx->at<float>(lo.T);
  sa.k = (float)(ctx->sigma * ctx->mu_l);
  sa.rho = (float)ctx->rho;
  sa.tw = ctx->at<float>(lo.twL);
  sa.post = ctx->at<float>(lo.post);
  sa.pre = ctx->at<float>(lo.pre);
  sa.invs = ctx->at<float>(lo.invs);
  sa.dense = ctx->at<float>(lo.dense);
}

// The barrier words and the error word of the persistent kernel live in the
// first context's scalar area (doubles 48 and 49).
static unsigned* batch_bar(const muffin_batch* b) { return reinterpret_cast<unsigned*>(b->ctx[0]->scal() + 48); }
static int* batch_errw(const muffin_batch* b) { return reinterpret_cast<int*>(b->ctx[0]->scal() + 49); }

static int batch_args(muffin_batch* b, BatchArgs* a, size_t* smem, int* grid) {
  if ((int)b->ctx.size() > kMaxBatchCubes) return bfail(b, MUFFIN_ERR_ARG, "the persistent batch takes at most 8 cubes");
  *a = BatchArgs{};
  a->nc = (int)b->ctx.size();
  for (int i = 0; i < a->nc; ++i) {
    const muffin_ctx* c = b->ctx[i];
    if (!batch_cube_ok(c->g, c->mu_s != 0.0, c->mu_l != 0.0))
      return bfail(b, MUFFIN_ERR_ARG, "a cube of the batch has no path in the persistent kernel",
                   "generation 1 IUWT, N in {128, 256, 512, 1024}, wavelet split 1..3 with coarse sub-images of "
                   "32, 64 or 128 and at most 3 coarse levels");
    batch_cube_of(c, &a->c[i]);
  }
  a->bar = batch_bar(b);
  a->err = batch_errw(b);
  a->polls = b->polls;
  *smem = batch_smem_bytes(*a);
  *grid = batch_grid(*smem);
  if (*grid <= 0) return bfail(b, MUFFIN_ERR_ARG, "the persistent batch kernel does not fit on this device");
  return MUFFIN_OK;
}

static int bfail(muffin_batch* b, int code, const char* what, const char* detail) {
  std::string m = what;
  if (detail) { m += ": "; m += detail; }
  if (b) b->err = m; else g_init_error = m;
  return code;
}

#define BCK(call)                                                                        \
  do {                                                                                   \
    cudaError_t e_ = (call);                                                             \
    if (e_ != cudaSuccess) return bfail(b, MUFFIN_ERR_CUDA, #call, cudaGetErrorString(e_)); \
  } while (0)

static void batch_drop_graph(muffin_batch* b) {
  if (b->exec) cudaGraphExecDestroy(b->exec);
  if (b->graph) cudaGraphDestroy(b->graph);
  b->exec = nullptr;
  b->graph = nullptr;
}

// One pass of every cube: parallel branches of one graph (mode 0), or one
// persistent cooperative launch (mode 1) after clearing its barrier words.
static int batch_capture(muffin_batch* b) {
  batch_drop_graph(b);
  if (b->mode == 1) {
    BatchArgs a;
    size_t smem = 0;
    int grid = 0;
    const int r = batch_args(b, &a, &smem, &grid);
    if (r != MUFFIN_OK) return r;
    BCK(cudaStreamBeginCapture(b->cap, cudaStreamCaptureModeThreadLocal));
    cudaError_t e = cudaMemsetAsync(a.bar, 0, 2 * sizeof(unsigned), b->cap);
    if (e == cudaSuccess) e = launch_batch_pass(a, smem, grid, b->cap);
    cudaGraph_t gr = nullptr;
    const cudaError_t e2 = cudaStreamEndCapture(b->cap, &gr);
    if (e != cudaSuccess || e2 != cudaSuccess) {
      if (gr) cudaGraphDestroy(gr);
      return bfail(b, MUFFIN_ERR_CUDA, "capture of the persistent batch pass", cudaGetErrorString(e != cudaSuccess ? e : e2));
    }
    b->graph = gr;
    BCK(cudaGraphInstantiate(&b->exec, b->graph, 0));
    for (size_t i = 0; i < b->ctx.size(); ++i) b->version[i] = b->ctx[i]->version;
    return MUFFIN_OK;
  }
  BCK(cudaStreamBeginCapture(b->cap, cudaStreamCaptureModeThreadLocal));
  int r = MUFFIN_OK;
  std::string why;
  cudaError_t e = cudaEventRecord(b->fork, b->cap);
  for (size_t i = 0; i < b->ctx.size() && e == cudaSuccess && r == MUFFIN_OK; ++i) {
    e = cudaStreamWaitEvent(b->side[i], b->fork, 0);
    if (e == cudaSuccess) r = enqueue_pass(b->ctx[i], b->side[i], nullptr);
    if (r != MUFFIN_OK) why = b->ctx[i]->err;
    if (e == cudaSuccess && r == MUFFIN_OK) e = cudaEventRecord(b->done[i], b->side[i]);
    if (e == cudaSuccess && r == MUFFIN_OK) e = cudaStreamWaitEvent(b->cap, b->done[i], 0);
  }
  cudaGraph_t gr = nullptr;
  const cudaError_t e2 = cudaStreamEndCapture(b->cap, &gr);
  if (r != MUFFIN_OK || e != cudaSuccess || e2 != cudaSuccess) {
    if (gr) cudaGraphDestroy(gr);
    if (r != MUFFIN_OK) return bfail(b, r, "capture of a cube's pass", why.c_str());
    return bfail(b, MUFFIN_ERR_CUDA, "batch capture", cudaGetErrorString(e != cudaSuccess ? e : e2));
  }
  b->graph = gr;
  BCK(cudaGraphInstantiate(&b->exec, b->graph, 0));
  for (size_t i = 0; i < b->ctx.size(); ++i) b->version[i] = b->ctx[i]->version;
  return MUFFIN_OK;
}

extern "C" {

int muffin_batch_create(muffin_batch** out, muffin_ctx* const* ctxs, int n, cudaStream_t stream) {
  if (!out || !ctxs || n < 1) return bfail(nullptr, MUFFIN_ERR_ARG, "batch needs an out-pointer and n >= 1 contexts");
  *out = nullptr;
  for (int i = 0; i < n; ++i) {
    if (!ctxs[i]) return bfail(nullptr, MUFFIN_ERR_ARG, "NULL context in batch");
    if (ctxs[i]->state < 1) return bfail(nullptr, MUFFIN_ERR_STATE, "every context of a batch needs muffin_set_psf first");
    for (int k = 0; k < i; ++k)
      if (ctxs[k] == ctxs[i]) return bfail(nullptr, MUFFIN_ERR_ARG, "a context appears twice in the batch");
  }
  muffin_batch* b = new muffin_batch();
  b->stream = stream;
  b->ctx.assign(ctxs, ctxs + n);
  b->version.assign(n, ~0u);
  b->side.assign(n, nullptr);
  b->done.assign(n, nullptr);
  cudaError_t e = cudaStreamCreateWithFlags(&b->cap, cudaStreamNonBlocking);
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&b->fork, cudaEventDisableTiming);
  for (int i = 0; i < n && e == cudaSuccess; ++i) {
    e = cudaStreamCreateWithFlags(&b->side[i], cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&b->done[i], cudaEventDisableTiming);
  }
  if (e != cudaSuccess) {
    muffin_batch_destroy(b);
    return bfail(nullptr, MUFFIN_ERR_CUDA, "batch streams", cudaGetErrorString(e));
  }
  *out = b;
  return MUFFIN_OK;
}

int muffin_batch_iterate(muffin_batch* b, int n_iter) {
  if (!b) return bfail(nullptr, MUFFIN_ERR_ARG, "batch is NULL");
  if (n_iter < 0) return bfail(b, MUFFIN_ERR_ARG, "n_iter < 0");
  if (n_iter == 0) return MUFFIN_OK;
  bool stale = !b->exec;
  for (size_t i = 0; i < b->ctx.size(); ++i) stale = stale || b->version[i] != b->ctx[i]->version;
  if (stale) {
    const int r = batch_capture(b);
    if (r != MUFFIN_OK) return r;
  }
  for (int i = 0; i < n_iter; ++i) BCK(cudaGraphLaunch(b->exec, b->stream));
  for (muffin_ctx* c : b->ctx) c->iter += n_iter;
  return MUFFIN_OK;
}

int muffin_batch_set_mode(muffin_batch* b, int mode) {
  if (!b) return bfail(nullptr, MUFFIN_ERR_ARG, "batch is NULL");
  if (mode != 0 && mode != 1) return bfail(b, MUFFIN_ERR_ARG, "mode must be 0 (graph branches) or 1 (persistent launch)");
  if (mode == 1) {
    cudaError_t e = batch_configure();
    if (e != cudaSuccess) return bfail(b, MUFFIN_ERR_CUDA, "persistent batch kernel", cudaGetErrorString(e));
    BatchArgs a;
    size_t smem = 0;
    int grid = 0;
    const int r = batch_args(b, &a, &smem, &grid);
    if (r != MUFFIN_OK) return r;
    // clear the error word once (it is sticky until muffin_batch_check)
    BCK(cudaMemsetAsync(batch_errw(b), 0, sizeof(int), b->stream));
  }
  b->mode = mode;
  batch_drop_graph(b);
  return MUFFIN_OK;
}

int muffin_batch_mode(const muffin_batch* b) { return b ? b->mode : -1; }

int muffin_batch_set_wait_limit(muffin_batch* b, long long polls) {
  if (!b) return bfail(nullptr, MUFFIN_ERR_ARG, "batch is NULL");
  b->polls = polls < 0 ? (1LL << 22) : polls;
  batch_drop_graph(b);
  return MUFFIN_OK;
}

int muffin_batch_check(muffin_batch* b) {
  if (!b) return bfail(nullptr, MUFFIN_ERR_ARG, "batch is NULL");
  BCK(cudaStreamSynchronize(b->stream));
  if (b->mode != 1) return MUFFIN_OK;
  int h = 0;
  BCK(cudaMemcpy(&h, batch_errw(b), sizeof(int), cudaMemcpyDeviceToHost));
  if (h != 0) {
    BCK(cudaMemset(batch_errw(b), 0, sizeof(int)));
    return bfail(b, MUFFIN_ERR_TIMEOUT,
                 "a grid barrier of the persistent batch pass gave up its bounded wait; the blocks skipped the "
                 "remaining stages, so the state of the batch's cubes is incomplete");
  }
  return MUFFIN_OK;
}

const char* muffin_batch_last_error(const muffin_batch* b) { return b ? b->err.c_str() : g_init_error.c_str(); }

void muffin_batch_destroy(muffin_batch* b) {
  if (!b) return;
  batch_drop_graph(b);
  for (cudaStream_t s : b->side) if (s) cudaStreamDestroy(s);
  for (cudaEvent_t e : b->done) if (e) cudaEventDestroy(e);
  if (b->fork) cudaEventDestroy(b->fork);
  if (b->cap) cudaStreamDestroy(b->cap);
  delete b;
}

}  // extern "C"
